"""Stationary free-streaming (ballistic) solution between diffuse walls under
constant gravity (Sec. V, "Ballistic regime: analytic analysis"): the
reference profiles of the paper's convergence test.

Test infrastructure only (see the package docstring).

Coordinates as in the solver: walls at x = 0 (left, temperature T_L) and x = L
(right, T_R); the acceleration is a_x = -g, so the potential V(x) = g x (m = 1)
is largest at the right wall.  In the paper's coordinate x' = x - L/2 the
solution Eq. "eq:f_bal" reads

    f(x, p) = A_+(x) exp(-p^2 / 2T_L)   for p > -c(x),
              A_-(x) exp(-p^2 / 2T_R)   for p < -c(x),
    c(x) = sqrt(g (L - 2x')),
    A_+ = n_+ exp(-g (L + 2x') / 2T_L) / sqrt(2 pi T_L),
    A_- = n_- exp( g (L - 2x') / 2T_R) / sqrt(2 pi T_R):

particles with p > -c left the left wall (those with -c < p < 0 turn back
before reaching the right wall), the others the right wall.  Zero net mass
flux fixes n_- sqrt(T_R) = n_+ exp(-g L / T_L) sqrt(T_L) (Eq. "eq:bal_npnm"),
and the particle number N = int_0^L n dx fixes n_+.

The moments are written out from that distribution with the truncated
Gaussian integrals (erf / exp closed forms); N is matched by adaptive
quadrature over x (scipy).  ``epsilon`` is the relative error of the paper's
convergence test (Eq. "eq:epsmax").
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad


def _gauss_moments(a: float, b: float, T: float):
    """int_a^b p^k exp(-p^2 / 2T) dp for k = 0, 1, 2 (a or b may be +-inf)."""
    s = math.sqrt(2.0 * T)
    ea = 0.0 if math.isinf(a) else math.exp(-a * a / (2.0 * T))
    eb = 0.0 if math.isinf(b) else math.exp(-b * b / (2.0 * T))
    erfa = -1.0 if a == -math.inf else (1.0 if a == math.inf else math.erf(a / s))
    erfb = -1.0 if b == -math.inf else (1.0 if b == math.inf else math.erf(b / s))
    I0 = math.sqrt(math.pi * T / 2.0) * (erfb - erfa)
    I1 = T * (ea - eb)
    aea = 0.0 if math.isinf(a) else a * ea
    beb = 0.0 if math.isinf(b) else b * eb
    I2 = T * I0 + T * (aea - beb)
    return I0, I1, I2


def _moments_at(x: float, L: float, g: float, TL: float, TR: float, n_plus: float):
    xp = x - L / 2.0
    n_minus = n_plus * math.exp(-g * L / TL) * math.sqrt(TL / TR)
    c = math.sqrt(max(g * (L - 2.0 * xp), 0.0))
    Ap = n_plus * math.exp(-g * (L + 2.0 * xp) / (2.0 * TL)) / math.sqrt(2.0 * math.pi * TL)
    Am = n_minus * math.exp(g * (L - 2.0 * xp) / (2.0 * TR)) / math.sqrt(2.0 * math.pi * TR)
    p0, p1, p2 = _gauss_moments(-c, math.inf, TL)
    m0, m1, m2 = _gauss_moments(-math.inf, -c, TR)
    n = Ap * p0 + Am * m0
    j = Ap * p1 + Am * m1
    e = Ap * p2 + Am * m2
    return n, j, e


def ballistic_profiles(x, L: float, g: float, T_left: float, T_right: float, N: float = 1.0):
    """n(x), u(x), T(x) of the ballistic solution with particle number N
    (one momentum axis: T = int (p - u)^2 f dp / n)."""
    if g == 0.0:
        raise ValueError("g > 0 (the g -> 0 limit is the free-molecular state)")
    N1 = quad(lambda s: _moments_at(s, L, g, T_left, T_right, 1.0)[0], 0.0, L, epsabs=1e-14, epsrel=1e-13,
              limit=200)[0]
    n_plus = N / N1
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.array([_moments_at(float(s), L, g, T_left, T_right, n_plus) for s in x])
    n, j, e = out[:, 0], out[:, 1], out[:, 2]
    u = j / n
    T = e / n - u * u
    return n, u, T


def epsilon(M, M_ref) -> float:
    """The paper's relative error of a profile (Eq. "eq:epsmax"): the largest
    deviation over the spread of M, the spread bounded below by 0.1."""
    M, M_ref = np.asarray(M, dtype=np.float64), np.asarray(M_ref, dtype=np.float64)
    return float(np.abs(M - M_ref).max() / max(M.max() - M.min(), 0.1))


__all__ = ["ballistic_profiles", "epsilon"]
