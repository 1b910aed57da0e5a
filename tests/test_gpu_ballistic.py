"""The paper's ballistic convergence test (Sec. V, Eq. "eq:epsmax") on the GPU.

The HHLB(20;200) model (Q_x = 200 per half, N = 20), 24 cells stretched with
A = 0.99, dt = 1e-4, WENO-5, FP64, no collisions, for the eight (g, Delta T)
cases of the paper's figure, as the instances of one handle.  From n = 1,
T = 1 at rest, 2.5e5 steps (t = 25): every profile must lie within the
paper's 1 % criterion of the free-streaming solution (Eqs. "eq:f_bal",
"eq:bal_npnm"; oracle/ballistic.py), and be stationary (n and T moved by less
than 0.1 % of their spread over the last 5e4 steps).  Measured: eps_max from
0.07 % (g = 1, Delta T = 0) to 0.96 % (g = 0.1, Delta T = -0.4); about 90 s of
GPU time.
"""
import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


def test_hhlb_20_200_ballistic_profiles_within_one_percent():
    from oracle.ballistic import ballistic_profiles, epsilon
    from oracle.solver import grid_x
    from paper_1708_03249_gb300 import hlb
    cfgs = W.HHLB_BALLISTIC_SET
    nx = cfgs[0]["nx"]
    _, xc, _ = grid_x(nx, 1.0, cfgs[0]["stretch_A"])
    stream = torch.cuda.Stream()
    with hlb.Handle(cfgs, stream=stream.cuda_stream) as h:
        h.init_equilibrium(1.0, 0.0, 0.0, 1.0)
        h.step(200_000)
        n20, _, T20, _ = h.moments()
        h.step(50_000)
        n, _, T, _ = h.moments()
        N, _ = h.diag()
    assert np.isfinite(n).all() and np.isfinite(T).all()
    np.testing.assert_allclose(N, 1.0, rtol=1e-10)          # one particle per unit length, conserved
    worst = []
    for i, c in enumerate(cfgs):
        sl = slice(nx * i, nx * (i + 1))
        rn, _, rT = ballistic_profiles(xc, 1.0, -c["ax"], c["T_left"], c["T_right"], N=1.0)
        eps = max(epsilon(n[sl], rn), epsilon(T[sl], rT))
        worst.append(eps)
        for M, M20 in ((n[sl], n20[sl]), (T[sl], T20[sl])):
            assert np.abs(M - M20).max() < 1e-3 * max(M.max() - M.min(), 0.1)
    assert max(worst) < 0.01, worst
