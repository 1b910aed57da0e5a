"""Seeded synthetic workloads: plain parameter sets and random draws.

This module holds no arithmetic of the method.  It is the one piece shared by
the CUDA path's callers and the oracle's tests: each workload is a dict of
``hlb_config`` fields, plus the seeded draws that some workloads need (the
batched instances, perturbations of an initial state).

Notation follows the paper: Qx = half-range order per half (2 Qx values of
p_x), Qy / Qz = full-range orders (0 = axis absent), Kn = Knudsen number,
(ax, ay, az) = F/m the acceleration; "gravity g at angle theta to the wall
normal" is a = -g (cos theta, sin theta, 0) (the potential V = m g x of Eq.
"eq:V" gives F = -m g).
"""
from __future__ import annotations

import math

import numpy as np

UPWIND2, WENO5 = 0, 1
FP64, FP32, FP32_TF32X3, FP32_BF16SPLIT = 0, 1, 2, 3   # FP32 state; force term on the tensor cores
X_HALF, X_FULL, X_LAGUERRE = 0, 1, 2   # along p_x: half-range Hermite (HHLB), Gauss-Hermite (HLB),
                                       # half-range Gauss-Laguerre

# Every workload is a plain dict of hlb_config fields (see include/hlb.h).
_BASE = dict(Qx=4, Qy=0, Qz=0, Nx_eq=-1, Ny_eq=-1, Nz_eq=-1, nx=64, ny=1,
             Lx=1.0, Ly=1.0, stretch_A=0.0, advection=WENO5, precision=FP32,
             cfl=0.5, dt=0.0, T_left=1.0, T_right=1.0, ax=0.0, ay=0.0, az=0.0,
             Kn=math.inf, x_basis=X_HALF)


def make(**kw) -> dict:
    unknown = set(kw) - set(_BASE)
    if unknown:
        raise KeyError(f"unknown config fields {sorted(unknown)}")
    d = dict(_BASE)
    d.update(kw)
    return d


def gravity(g: float, theta_deg: float):
    t = math.radians(theta_deg)
    return dict(ax=-g * math.cos(t), ay=-g * math.sin(t))


# --- the five synthetic workloads ------------------------------------------
# 1D channel, plain method in FP64: HHLB(3;4) x GH(4), upwind2, barometric.
CHANNEL_1D_FP64 = make(Qx=4, Qy=4, nx=64, advection=UPWIND2, precision=FP64,
                       Kn=0.1, ax=-0.1, T_left=1.0, T_right=1.0)
CHANNEL_1D_FP64_STEPS = 10_000

# 1D channel, unequal walls, stretched grid, WENO5, four Knudsen numbers.
def channel_1d_stretched(Kn: float, precision: int = FP32) -> dict:
    return make(Qx=8, Qy=8, nx=512, stretch_A=0.9, T_left=0.5, T_right=1.5,
                Kn=Kn, advection=WENO5, precision=precision, **gravity(0.5, 30.0))
CHANNEL_1D_STRETCHED_KN = (0.01, 0.1, 1.0, 10.0)

# The paper's ballistic runs (Sec. V): the HHLB(20;200) model (Qx = 200 per
# half, 400 velocities, equilibrium order N = 20), N_x = 24 cells stretched with
# A = 0.99, dt = 1e-4, WENO5, FP64, no collisions, gravity g towards the left
# wall, wall temperatures T_+- = 1 -+ Delta T (T_+ = 1.4, T_- = 0.6 at
# Delta T = -0.4).  The paper's figure sweeps g in {0.1, 1} x Delta T in
# {0.6, 0.3, 0, -0.4}: eight independent instances.
def hhlb_ballistic(g: float, dT: float, Qx: int = 200, Nx_eq: int = 20) -> dict:
    return make(Qx=Qx, Nx_eq=Nx_eq, nx=24, stretch_A=0.99, Lx=1.0, advection=WENO5, precision=FP64,
                dt=1e-4, Kn=math.inf, ax=-g, T_left=1.0 - dT, T_right=1.0 + dT)
HHLB_BALLISTIC_G = (0.1, 1.0)
HHLB_BALLISTIC_DT = (0.6, 0.3, 0.0, -0.4)
HHLB_BALLISTIC_SET = [hhlb_ballistic(g, dT) for g in HHLB_BALLISTIC_G for dT in HHLB_BALLISTIC_DT]

# 2D box 256 x 256, Qx = 16 per half x Qy = 16 (512 velocities).
BOX_2D = make(Qx=16, Qy=16, nx=256, ny=256, Lx=1.0, Ly=1.0, T_left=1.0,
              T_right=1.2, Kn=0.05, advection=WENO5, precision=FP32,
              **gravity(0.2, 45.0))
BOX_2D_STEPS = 2000

# Large 2D channel 1024 x 512, 16 x 8 x 8 = 1024 velocities, about 537M values.
LARGE_2D = make(Qx=8, Qy=8, Qz=8, nx=1024, ny=512, Lx=1.0, Ly=0.5,
                T_left=1.0, T_right=2.0, Kn=0.5, ax=-0.3, ay=-0.3, az=0.0,
                advection=WENO5, precision=FP32)
LARGE_2D_STEPS = 500


def scaled(base: dict, **kw) -> dict:
    """A smaller case of a workload: same velocity set and physics, new sizes."""
    d = dict(base)
    d.update(kw)
    return d


# --- seeded draws -------------------------------------------------------------
_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma, then mix."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """U[0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


BATCH_SEED = 170803249
BATCH_STEPS = 5000


def batched_instances(ninst: int = 4096, seed: int = BATCH_SEED):
    """Independent 1D channels, drawn in this order per instance:
    nx = round(exp U[ln 32, ln 1024]); Qx uniform in {4, 8, 16}, Qy = Qx;
    Kn = exp U[ln 0.01, ln 10]; g ~ U[0, 1]; theta ~ U[0, 90] degrees;
    T_left = 1, T_right = exp U[ln 1/2, ln 2].  Uniform grid, WENO5, CFL 0.5.
    """
    rng = SplitMix64(seed)
    out = []
    for _ in range(ninst):
        nx = int(round(math.exp(math.log(32) + rng.uniform() * (math.log(1024) - math.log(32)))))
        Q = (4, 8, 16)[min(2, int(rng.uniform() * 3))]
        Kn = math.exp(math.log(0.01) + rng.uniform() * (math.log(10) - math.log(0.01)))
        g = rng.uniform()
        theta = 90.0 * rng.uniform()
        TR = math.exp(math.log(0.5) + rng.uniform() * (math.log(2) - math.log(0.5)))
        out.append(make(Qx=Q, Qy=Q, nx=nx, Kn=Kn, T_left=1.0, T_right=TR,
                        advection=WENO5, precision=FP32, **gravity(g, theta)))
    return out


def perturbation(shape, seed: int, amplitude: float = 0.05) -> np.ndarray:
    """Multiplicative factors 1 + amplitude * U(-1, 1), FP64, seeded."""
    rng = np.random.default_rng(seed)
    return 1.0 + amplitude * rng.uniform(-1.0, 1.0, size=shape)
