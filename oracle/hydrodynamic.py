"""Navier-Stokes (Chapman-Enskog) reference profiles of the gravity-driven
channel between walls at different temperatures (Sec. V, "Different wall
temperatures: hydrodynamic regime").

Test infrastructure only (see the package docstring).

Coordinates as in the solver: walls at x = 0 (left, T_L = the paper's T_+)
and x = L (right, T_R = T_-), acceleration a_x = -g.  In the paper's
coordinate x' = x - L/2:

  - Fourier's law with kappa = 3 tau n T / 2 and tau = Kn / n (Eq.
    "eq:NS_q_def") makes the heat flux constant with kappa proportional to T,
    so T^2 is linear: T(x') = sqrt(A x' + B), A = (T_-^2 - T_+^2)/L,
    B = (T_-^2 + T_+^2)/2 (Eq. "eq:NS_temp");
  - q = 3 Kn (T_+^2 - T_-^2) / (4 L) (Eq. "eq:NS_q");
  - hydrostatic balance d(nT)/dx = -g n then gives Eq. "eq:NS_n",
    n = g N exp[-g L (2T - T_- - T_+) / (T_-^2 - T_+^2)] / (2 T sinh(g L / (T_+ + T_-))),
    which for T_+ = T_- = T_w is the barometric profile of Eq. "eq:iso_n",
    n = g N exp(-g x / T_w) / (2 T_w sinh(g L / 2 T_w)) (x measured from the
    channel centre there).

The profiles hold to first order in Kn away from the walls' Knudsen layers;
the paper compares them with runs at Kn = 1e-3.
"""
from __future__ import annotations

import math

import numpy as np


def ns_profiles(x, L: float, g: float, T_left: float, T_right: float, N: float = 1.0):
    """n(x), T(x) and the constant q of the Navier-Stokes solution with N
    particles per unit cross-section (one momentum axis, m = 1)."""
    x = np.asarray(x, dtype=np.float64)
    xp = x - L / 2.0
    Tp, Tm = T_left, T_right
    A = (Tm * Tm - Tp * Tp) / L
    B = (Tm * Tm + Tp * Tp) / 2.0
    T = np.sqrt(A * xp + B)
    if g == 0.0:
        # the g -> 0 limit of Eq. "eq:NS_n" (sinh z ~ z): n T constant
        n = N * (Tp + Tm) / (2.0 * L * T)
    elif Tm == Tp:
        n = g * N * np.exp(-g * xp / Tp) / (2.0 * Tp * math.sinh(g * L / (2.0 * Tp)))
    else:
        n = (g * N * np.exp(-g * L * (2.0 * T - Tm - Tp) / (Tm * Tm - Tp * Tp))
             / (2.0 * T * math.sinh(g * L / (Tp + Tm))))
    return n, T


def ns_heat_flux(L: float, Kn: float, T_left: float, T_right: float) -> float:
    """q of Eq. "eq:NS_q" (constant across the channel)."""
    return 3.0 * Kn * (T_left ** 2 - T_right ** 2) / (4.0 * L)


__all__ = ["ns_profiles", "ns_heat_flux"]
