"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Each case starts both sides from the same state (the library's own
equilibrium times seeded perturbation factors) and compares, after a number
of RK-3 steps, the full state element by element and the macroscopic
moments.  Tolerances:
  FP64 path: |f - f_ref| <= 1e-10 max|f_ref| at Q <= 8; 5e-8 at Q = 16 (the
             per-node equilibrium recurrence loses up to 1e-8 there);
  FP32 path: moment errors err(M) <= 1e-5 with
             err(M) = max|M - M_ref| / max(max|M_ref|, s_M), s_n = max n,
             s_u = sqrt(max T), s_T = max T, s_q = max n T^{3/2};
             per-velocity |f_v - f_ref,v| <= 2e-5 max_nodes |f_ref,v|.
"""
import math

import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stream():
    return torch.cuda.current_stream().cuda_stream


def moment_errors(mom, ref):
    n, u, T, q = mom
    rn, ru, rT, rq = ref
    sT = np.abs(rT).max()
    return {
        "n": np.abs(n - rn).max() / np.abs(rn).max(),
        "u": np.abs(u - ru).max() / max(np.abs(ru).max(), math.sqrt(sT)),
        "T": np.abs(T - rT).max() / sT,
        "q": np.abs(q - rq).max() / max(np.abs(rq).max(), np.abs(rn).max() * sT ** 1.5),
    }


def run_pair(cfg, steps, seed=1, amp=0.05, init=(1.0, 0.0, 0.0, 1.0), graphs=True, stochastic=None,
             persistent=None):
    from oracle.solver import Solver, config_from
    from paper_1708_03249_gb300 import hlb
    cfgs = cfg if isinstance(cfg, list) else [cfg]
    h = hlb.Handle(cfgs, stream=_stream())
    h.set_options(use_graphs=graphs)
    if stochastic is not None:
        h.set_rounding(stochastic)
    if persistent is not None:
        h.set_persistent(persistent)
    h.init_equilibrium(*init)
    f0 = h.get_state().astype(np.float64)
    f0 = f0 * W.perturbation(f0.shape, seed=seed, amplitude=amp)
    h.set_state(f0)
    f0 = h.get_state().astype(np.float64)          # exactly what the device holds
    h.step(steps)
    got = h.get_state().astype(np.float64)
    mom = h.moments()
    N, res = h.diag()
    refs, off = [], 0
    for i, c in enumerate(cfgs):
        s = Solver(config_from(c))
        assert h.dt(i) == pytest.approx(s.dt, rel=1e-14)
        size = s.f.size
        s.f = f0[off:off + size].reshape(s.f.shape).copy()
        s.step(steps)
        refs.append(s)
        off += size
    h.close()
    return got, mom, N, refs


def _oracle_moments(refs):
    parts = [s.moments() for s in refs]
    n = np.concatenate([p[0].reshape(-1) for p in parts])
    u = np.concatenate([p[1].reshape(-1, 3) for p in parts])
    T = np.concatenate([p[2].reshape(-1) for p in parts])
    q = np.concatenate([p[3].reshape(-1) for p in parts])
    return n, u, T, q


def _check_fp64(got, refs, tol):
    ref = np.concatenate([s.f.reshape(-1) for s in refs])
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < tol, err


def _check_fp32(got, mom, refs, ftol=2e-5, mtol=1e-5, bulk=1e-6):
    """FP32 path vs FP64 oracle: moments, the max-norm of the state, and each
    velocity whose largest value exceeds ``bulk`` times the state's maximum
    against its own scale (the far tails of the Q = 16 sets, weights down to
    1e-15, are covered by the max-norm: the FP64 equilibrium recurrence keeps
    them to ~1e-4 of their own size only)."""
    errs = moment_errors(mom, _oracle_moments(refs))
    assert max(errs.values()) < mtol, errs
    off = 0
    for s in refs:
        ref = s.f.reshape(-1, s.vs.V)
        g = got[off:off + ref.size].reshape(ref.shape)
        gmax = np.abs(ref).max()
        assert np.abs(g - ref).max() < ftol * gmax
        scale = np.abs(ref).max(axis=0)
        sel = scale >= bulk * gmax
        rel = (np.abs(g - ref)[:, sel] / scale[sel]).max()
        assert rel < ftol, (rel, int(np.argmax((np.abs(g - ref)[:, sel] / scale[sel]).max(axis=0))))
        off += ref.size


def test_fp32_weno_extreme_ratios_stay_finite():
    # A jump of 30 orders of magnitude between neighbouring cells: sigma^2 of
    # the flat side underflows FP32; the weights must still follow Tab. "weno".
    cfg = W.make(Qx=4, Qy=4, nx=16, advection=W.WENO5, precision=W.FP32, Kn=math.inf)
    from oracle.solver import Solver, config_from
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.init_equilibrium()
        f = h.get_state().reshape(1, 16, -1).astype(np.float64)
        f[:, :8] *= 1e-30
        h.set_state(f.reshape(-1))
        f0 = h.get_state().astype(np.float64)
        h.step(3)
        got = h.get_state().astype(np.float64)
    assert np.isfinite(got).all()
    s = Solver(config_from(cfg))
    s.f = f0.reshape(s.f.shape).copy()
    s.step(3)
    ref = s.f.reshape(-1)
    assert np.abs(got - ref).max() < 2e-6 * np.abs(ref).max()


# --- FP64 ------------------------------------------------------------------------
def test_fp64_channel_upwind2():
    cfg = W.scaled(W.CHANNEL_1D_FP64, nx=24)
    got, mom, N, refs = run_pair(cfg, 40)
    _check_fp64(got, refs, 1e-11)
    assert N[0] == pytest.approx(refs[0].total_number(), rel=1e-12)


def test_fp64_channel_eager_equals_graph():
    cfg = W.scaled(W.CHANNEL_1D_FP64, nx=16)
    a, *_ = run_pair(cfg, 37, graphs=True)
    b, *_ = run_pair(cfg, 37, graphs=False)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("adv", [W.UPWIND2, W.WENO5])
def test_fp64_2d_stretched_all_forces(adv):
    cfg = W.make(Qx=3, Qy=4, Qz=2, nx=10, ny=6, Ly=0.6, stretch_A=0.7, advection=adv,
                 precision=W.FP64, T_left=0.7, T_right=1.6, ax=-0.4, ay=0.3, az=0.2, Kn=0.2)
    got, mom, N, refs = run_pair(cfg, 12, init=(1.0, 0.1, -0.05, 1.1))
    _check_fp64(got, refs, 1e-10)


def test_fp64_collisionless_free_molecular():
    cfg = W.make(Qx=4, nx=12, advection=W.WENO5, precision=W.FP64, T_left=0.8, T_right=1.7)
    got, mom, N, refs = run_pair(cfg, 60)
    _check_fp64(got, refs, 1e-10)


def test_fp64_q16():
    cfg = W.make(Qx=16, Qy=4, nx=8, advection=W.WENO5, precision=W.FP64, T_left=1.0, T_right=1.2,
                 Kn=0.05, **W.gravity(0.2, 45.0))
    got, mom, N, refs = run_pair(cfg, 4)
    _check_fp64(got, refs, 5e-8)


# --- the HHLB(20;200) model of the ballistic runs (Sec. V) -----------------------
# 400 velocities, K^h read from global memory (400 x 400 FP64), each node's
# velocities split over several CTAs; the oracle takes the stored 40-digit
# order-200 tables.  Tolerance: the library's K^h differs from the oracle's
# by 1.5e-12 of each column's largest entry, which moves (K f)_k by up to
# 7e-11 of max f at the slowest velocity; times g dt per stage.
@pytest.mark.parametrize("g,dT", [(1.0, -0.4), (0.1, 0.6)])
def test_fp64_hhlb_20_200_ballistic(g, dT):
    cfg = W.hhlb_ballistic(g, dT)
    got, mom, N, refs = run_pair(cfg, 40)
    _check_fp64(got, refs, 1e-11)
    assert N[0] == pytest.approx(refs[0].total_number(), rel=1e-12)
    errs = moment_errors(mom, _oracle_moments(refs))
    assert max(errs.values()) < 1e-11, errs


def test_fp64_hhlb_20_200_paper_set_in_one_handle():
    # the eight (g, Delta T) cases of the paper's figure as instances of one
    # group: 192 nodes x 400 velocities in one launch per stage
    got, mom, N, refs = run_pair(W.HHLB_BALLISTIC_SET, 12)
    _check_fp64(got, refs, 1e-11)


@pytest.mark.parametrize("Qx,Qy,Nx_eq,adv", [(200, 4, 12, W.WENO5), (200, 0, 12, W.UPWIND2),
                                              (200, 0, 20, W.WENO5), (200, 4, 20, W.UPWIND2),
                                              (16, 0, 15, W.WENO5)])
def test_fp64_high_order_collisional(Qx, Qy, Nx_eq, adv):
    # BGK at the order-200 set (the oracle's stored tables; no mpmath on
    # every machine), also with a p_y axis (1600 velocities, 19 CTAs per
    # node).  Up to N = 12 the per-node equilibrium recurrence on the device
    # is accurate to ~3^N eps; above it (N = 20: the paper's HHLB(20;200), and
    # N = 15 at Q = 16 on the marching path) the coefficients G^{+-} come from
    # the quadrature kernel.
    cfg = W.make(Qx=Qx, Qy=Qy, Nx_eq=Nx_eq, nx=16, stretch_A=0.8, advection=adv, precision=W.FP64,
                 T_left=0.8, T_right=1.3, Kn=0.3, dt=2e-4, **W.gravity(0.5, 30.0))
    got, mom, N, refs = run_pair(cfg, 10, init=(1.0, 0.05, 0.0, 1.0))
    _check_fp64(got, refs, 1e-9)


# --- FP32 ------------------------------------------------------------------------
@pytest.mark.parametrize("Kn", W.CHANNEL_1D_STRETCHED_KN)
def test_fp32_stretched_channel(Kn):
    cfg = W.scaled(W.channel_1d_stretched(Kn), nx=32)
    got, mom, N, refs = run_pair(cfg, 30)
    _check_fp32(got, mom, refs)


@pytest.mark.parametrize("TL,TR", [(0.5, 2.0), (1.0, 0.5)])
def test_fp32_channel_q16(TL, TR):
    # order 15 along p_x: the per-node equilibrium runs in double-float
    cfg = W.make(Qx=16, Qy=16, nx=48, advection=W.WENO5, precision=W.FP32, T_left=TL, T_right=TR,
                 Kn=0.1, **W.gravity(0.7, 60.0))
    got, mom, N, refs = run_pair(cfg, 20, init=(1.0, 0.1, -0.1, 0.9))
    _check_fp32(got, mom, refs)


def test_fp32_box_2d_q16():
    cfg = W.scaled(W.BOX_2D, nx=12, ny=6)
    got, mom, N, refs = run_pair(cfg, 4)
    _check_fp32(got, mom, refs)


@pytest.mark.parametrize("adv", [W.WENO5, W.UPWIND2])
def test_fp32_large_2d_1024_velocities(adv):
    cfg = W.scaled(W.LARGE_2D, nx=12, ny=6, Ly=6 / 12, advection=adv)
    got, mom, N, refs = run_pair(cfg, 4)
    _check_fp32(got, mom, refs)


@pytest.mark.parametrize("nx", [13, 31, 55])
def test_fp32_2d_ragged_pairs(nx):
    # The pair kernel advances two cells per iteration: segments of odd length
    # (nx = 13: one segment; 31, 55: a full segment of 24 and a ragged one)
    # end on a single cell.  Stretched grid, walls at different temperatures,
    # forces along p_x and p_y.
    cfg = W.make(Qx=4, Qy=4, nx=nx, ny=5, Ly=0.25, stretch_A=0.6, advection=W.WENO5, precision=W.FP32,
                 T_left=0.8, T_right=1.4, ax=-0.3, ay=0.2, Kn=0.1)
    got, mom, N, refs = run_pair(cfg, 6, init=(1.0, 0.05, -0.03, 1.0))
    _check_fp32(got, mom, refs)


@pytest.mark.parametrize("adv", [W.WENO5, W.UPWIND2])
def test_fp32_2d_q8_16x8(adv):
    cfg = W.make(Qx=8, Qy=8, nx=27, ny=6, Ly=0.3, advection=adv, precision=W.FP32,
                 T_left=1.0, T_right=2.0, ax=-0.3, ay=-0.3, Kn=0.5)
    got, mom, N, refs = run_pair(cfg, 4)
    _check_fp32(got, mom, refs)


@pytest.mark.parametrize("Qx,Qy,nx", [(16, 0, 31), (4, 0, 31), (8, 8, 55), (4, 4, 13), (16, 16, 23)])
def test_fp32_1d_shapes_ragged(Qx, Qy, nx):
    # 1D FP32: the line kernel (four cells per iteration; whole-warp slabs:
    # 32 x 1, 16 x 8, 8 x 4, and 32 x 16 with the force term on the tensor
    # cores) and the scalar kernel (8 x 1); lengths that are not a multiple of
    # four end a segment on a partial iteration
    cfg = W.make(Qx=Qx, Qy=Qy, nx=nx, advection=W.WENO5, precision=W.FP32, T_left=0.7, T_right=1.3,
                 Kn=0.2, **(W.gravity(0.4, 30.0) if Qy else {"ax": -0.4}))
    got, mom, N, refs = run_pair(cfg, 10, init=(1.0, 0.05, 0.0, 1.0))
    _check_fp32(got, mom, refs)


@pytest.mark.parametrize("adv", [W.WENO5, W.UPWIND2])
def test_fp32_1d_q16_tensor_core_force(adv):
    # 32 x 16 slabs: a K f by three TF32 products on the tensor cores; a strong
    # oblique force so that the force term carries the update
    cfg = W.make(Qx=16, Qy=16, nx=42, advection=adv, precision=W.FP32, T_left=0.8, T_right=1.6,
                 Kn=0.3, **W.gravity(0.9, 35.0))
    got, mom, N, refs = run_pair(cfg, 8, init=(1.0, 0.1, 0.05, 1.1))
    _check_fp32(got, mom, refs)


# The force term a . K f on the tensor cores, as a runtime option: three TF32
# products (HLB_FP32_TF32X3) or the six leading products of a three-term bf16
# split (HLB_FP32_BF16SPLIT), FP32 accumulation, in the 2D pair kernel and the
# 1D line kernel, for both slab shapes that tile into 16 x 8 x 8 blocks; a
# strong oblique force so that K carries the update.
_TC_CASES = {
    "pair_16x8": lambda p: W.make(Qx=8, Qy=8, nx=27, ny=6, Ly=0.3, precision=p, T_left=1.0, T_right=2.0,
                                  Kn=0.5, **W.gravity(0.9, 40.0)),
    "pair_32x16": lambda p: W.make(Qx=16, Qy=16, nx=14, ny=6, Ly=6 / 14, precision=p, T_left=1.0, T_right=1.2,
                                   Kn=0.05, **W.gravity(0.9, 45.0)),
    "line_16x8": lambda p: W.make(Qx=8, Qy=8, nx=43, precision=p, T_left=0.7, T_right=1.4, Kn=0.3,
                                  **W.gravity(0.9, 30.0)),
    "line_32x16": lambda p: W.make(Qx=16, Qy=16, nx=42, precision=p, T_left=0.8, T_right=1.6, Kn=0.3,
                                   **W.gravity(0.9, 35.0)),
}


@pytest.mark.parametrize("prec", [W.FP32_TF32X3, W.FP32_BF16SPLIT])
@pytest.mark.parametrize("case", sorted(_TC_CASES))
@pytest.mark.parametrize("adv", [W.WENO5, W.UPWIND2])
def test_fp32_tensor_core_force_forms(case, prec, adv):
    from paper_1708_03249_gb300 import hlb
    cfg = dict(_TC_CASES[case](prec), advection=adv)
    with hlb.Handle(cfg, stream=_stream()) as h:
        assert h.force_form(0) == (1 if prec == W.FP32_TF32X3 else 2)
    got, mom, N, refs = run_pair(cfg, 6, init=(1.0, 0.1, 0.05, 1.1))
    _check_fp32(got, mom, refs)


def test_fp32_force_forms_agree():
    # The three FP32 forms of the force term on one state: they differ only
    # by FP32 rounding of the contraction (all within a few ulps of the state).
    from paper_1708_03249_gb300 import hlb
    outs = []
    for prec in (W.FP32, W.FP32_TF32X3, W.FP32_BF16SPLIT):
        cfg = _TC_CASES["pair_32x16"](prec)
        with hlb.Handle(cfg, stream=_stream()) as h:
            h.init_equilibrium(1.0, 0.1, 0.05, 1.1)
            f = h.get_state().astype(np.float64) * W.perturbation(h.values, seed=21)
            h.set_state(f)
            h.step(5)
            outs.append(h.get_state().astype(np.float64))
    scale = np.abs(outs[0]).max()
    for o in outs[1:]:
        assert np.abs(o - outs[0]).max() < 2e-6 * scale


def test_default_force_forms():
    # HLB_FP32 leaves the choice to the library (the measured faster form):
    # the tensor cores for the 1D kernel's 32 x 16 slabs and the 2D kernel's
    # 16 x 8 slabs with upwind2, FMAs elsewhere; FP64 and slabs that do not
    # tile use FMAs whatever was asked.
    from paper_1708_03249_gb300 import hlb
    cases = [(_TC_CASES["line_32x16"](W.FP32), 1), (_TC_CASES["pair_16x8"](W.FP32), 0),
             (dict(_TC_CASES["pair_16x8"](W.FP32), advection=W.UPWIND2), 1),
             (_TC_CASES["line_16x8"](W.FP32), 0), (W.make(Qx=4, Qy=4, nx=16, precision=W.FP32_TF32X3), 0),
             (W.make(Qx=8, Qy=8, nx=16, precision=W.FP64), 0)]
    for cfg, form in cases:
        with hlb.Handle(cfg, stream=_stream()) as h:
            assert h.force_form(0) == form, cfg


@pytest.mark.parametrize("Qx,Qy,ny,prec,adv", [(16, 8, 1, W.FP32, W.WENO5), (8, 4, 5, W.FP32, W.WENO5),
                                                (32, 16, 1, W.FP32, W.UPWIND2), (8, 4, 1, W.FP64, W.UPWIND2)])
def test_full_range_x_models(Qx, Qy, ny, prec, adv):
    # HLB(N; Q) along p_x (Gauss-Hermite of order Qx, K^H without the jump
    # term): the line kernel (16 x 8, and 32 x 16 with the tensor-core force
    # term), the pair kernel (8 x 4) and the FP64 kernel, against the oracle
    cfg = W.make(Qx=Qx, Qy=Qy, nx=23, ny=ny, Ly=0.25, advection=adv, precision=prec, T_left=0.8, T_right=1.4,
                 Kn=0.4, x_basis=W.X_FULL, **W.gravity(0.5, 30.0))
    got, mom, N, refs = run_pair(cfg, 6, init=(1.0, 0.05, 0.0, 1.0))
    if prec == W.FP64:
        _check_fp64(got, refs, 1e-10)
    else:
        _check_fp32(got, mom, refs)


@pytest.mark.parametrize("Qx,Qy,ny,prec,adv", [(4, 4, 1, W.FP32, W.WENO5), (8, 8, 4, W.FP32, W.WENO5),
                                                (4, 4, 1, W.FP64, W.UPWIND2)])
def test_half_range_laguerre_models(Qx, Qy, ny, prec, adv):
    # Half-range Gauss-Laguerre along p_x (K^L of Eq. "eq:hh_Kk_L"): the line
    # kernel (8 x 4), the pair kernel (16 x 8) and the FP64 kernel, with the
    # library's equilibrium recurrence (omega(0) = 1, no 1/a term) for the
    # node pass and the walls, against the oracle's moment projection
    cfg = W.make(Qx=Qx, Qy=Qy, nx=19, ny=ny, Ly=0.2, advection=adv, precision=prec, T_left=0.9, T_right=1.3,
                 Kn=0.3, x_basis=W.X_LAGUERRE, **W.gravity(0.4, 20.0))
    got, mom, N, refs = run_pair(cfg, 5, init=(1.0, 0.05, 0.0, 1.0))
    if prec == W.FP64:
        _check_fp64(got, refs, 1e-10)
    else:
        _check_fp32(got, mom, refs)


def test_laguerre_initial_equilibrium_matches_oracle():
    from oracle.model import VelocitySet
    from paper_1708_03249_gb300 import hlb
    cfg = W.make(Qx=8, Qy=4, nx=7, precision=W.FP64, x_basis=W.X_LAGUERRE, Kn=1.0)
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.init_equilibrium(1.2, -0.3, 0.1, 0.8)
        got = h.get_state().reshape(7, -1)
    ref = VelocitySet(8, 4, x_laguerre=True).equilibrium(np.float64(1.2), -0.3, 0.1, 0.0, np.float64(0.8)).reshape(-1)
    np.testing.assert_allclose(got, np.broadcast_to(ref, got.shape), atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("Qx,Qy,nx,ny,adv,prec", [
    (8, 8, 6, 1, W.WENO5, W.FP32),      # shortest WENO-5 channel: line kernel, one partial iteration
    (8, 8, 6, 5, W.WENO5, W.FP32),      # pair kernel at the fewest rows it takes (5: two strips, one ragged)
    (8, 8, 6, 3, W.WENO5, W.FP32),      # ny = 3: the generic per-node kernel (halo wraps more than once)
    (4, 4, 3, 1, W.UPWIND2, W.FP64),    # shortest upwind2 channel, FP64
    (4, 4, 3, 1, W.UPWIND2, W.FP32),    # ... FP32 (scalar kernel: 8 x 4 slabs)
])
def test_minimum_sizes(Qx, Qy, nx, ny, adv, prec):
    # The smallest grids each kernel accepts: wall ghosts and periodic halos
    # overlap the interior everywhere.
    cfg = W.make(Qx=Qx, Qy=Qy, nx=nx, ny=ny, Ly=0.1 * ny, advection=adv, precision=prec, T_left=0.9,
                 T_right=1.2, Kn=0.4, **W.gravity(0.3, 40.0))
    got, mom, N, refs = run_pair(cfg, 4, init=(1.0, 0.05, 0.0, 1.0))
    if prec == W.FP64:
        _check_fp64(got, refs, 1e-10)
    else:
        _check_fp32(got, mom, refs)


def test_fp32_collisionless_2d_with_force():
    # Kn = +inf (no BGK term, 1/tau = 0 in the factor lines) with an oblique force
    cfg = W.make(Qx=8, Qy=8, nx=20, ny=6, Ly=0.3, precision=W.FP32, T_left=0.8, T_right=1.5,
                 Kn=math.inf, **W.gravity(0.5, 30.0))
    got, mom, N, refs = run_pair(cfg, 6)
    _check_fp32(got, mom, refs)


def test_rest_state_is_a_fixed_point():
    # No force, walls at the gas temperature, f = the rest Maxwellian: the
    # half-range quadrature represents it exactly, every flux balances and the
    # BGK term vanishes, so the state stays put (up to FP32 rounding) on the 2D
    # pair kernel, 1024 velocities.
    from paper_1708_03249_gb300 import hlb
    cfg = W.scaled(W.LARGE_2D, nx=64, ny=16, ax=0.0, ay=0.0, az=0.0, T_left=1.3, T_right=1.3)
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.init_equilibrium(1.0, 0.0, 0.0, 1.3)
        f0 = h.get_state().astype(np.float64)
        h.step(20)
        f1 = h.get_state().astype(np.float64)
    assert np.abs(f1 - f0).max() < 1e-5 * np.abs(f0).max()


def test_fp32_batched_mixed_instances():
    insts = W.batched_instances(6)
    insts = [W.scaled(c, nx=min(c["nx"], 40)) for c in insts]
    got, mom, N, refs = run_pair(insts, 6)
    _check_fp32(got, mom, refs)
    for i, s in enumerate(refs):
        assert N[i] == pytest.approx(s.total_number(), rel=2e-6)


@pytest.mark.parametrize("persistent", [True, False])
def test_fp32_particle_number_conserved(persistent):
    # N = int n dx is conserved by the scheme (flux telescoping, wall balance,
    # K column sums, BGK mass); in FP32 only rounding noise may move it.  Over
    # 3000 steps a bias of one ulp-fraction per step (e.g. RK-3 weights that
    # do not sum to 1 after rounding: 2^-25 per step, 9e-5 here) shows.
    from paper_1708_03249_gb300 import hlb
    cfg = W.scaled(W.channel_1d_stretched(0.1), nx=64)
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.set_persistent(persistent)
        h.init_equilibrium()
        N0 = h.diag()[0][0]
        h.step(3000)
        N1, r = h.diag()
    assert N1[0] == pytest.approx(N0, rel=2e-6)
    assert r[0] > 0


def test_fp32_full_size_large_2d_sampled_nodes():
    # The bench's workload at full size (1024 x 512 x 1024 velocities), one RK-3
    # step from a perturbed equilibrium, checked on sampled nodes: the oracle
    # steps a 19 x 19 window around each sample (the RK-3 stencil reaches 9
    # cells), whose centre is then exact.
    from oracle.solver import Solver, config_from
    from paper_1708_03249_gb300 import hlb
    cfg = W.LARGE_2D
    nx, ny = cfg["nx"], cfg["ny"]
    with hlb.Handle(cfg, stream=_stream()) as h:
        V = h.values // h.nodes
        h.init_equilibrium(1.0, 0.05, -0.02, 1.2)
        f = h.get_state().reshape(ny, nx, V).astype(np.float64)
        f *= W.perturbation(f.shape, seed=21, amplitude=0.02)
        f = f.astype(np.float32)
        h.set_state(f)
        N0 = h.diag()[0][0]
        h.step(1)
        got = h.get_state().reshape(ny, nx, V)
        N1 = h.diag()[0][0]
        dt = h.dt()
    assert N1 == pytest.approx(N0, rel=1e-5)
    rng = np.random.default_rng(5)
    samples = [(0, 3), (nx - 1, 100), (4, 511), (nx - 6, 0)] + \
              [(int(rng.integers(9, nx - 9)), int(rng.integers(0, ny))) for _ in range(3)]
    for (x, y) in samples:
        x0 = min(max(x - 9, 0), nx - 19)
        ys = [(y + k) % ny for k in range(-9, 10)]
        win = f[ys][:, x0:x0 + 19].astype(np.float64)
        wc = dict(cfg, nx=19, ny=19, Ly=19 * cfg["Ly"] / ny, Lx=19 * cfg["Lx"] / nx, dt=dt)
        s = Solver(config_from(wc))
        s.f = win.reshape(s.f.shape)
        s.step(1)
        ref = s.f[9, x - x0].reshape(-1)
        g = got[y, x].astype(np.float64)
        err = np.abs(g - ref).max() / np.abs(ref).max()
        assert err < 2e-6, (x, y, err)


def test_fp64_channel_full_length_barometric():
    # The FP64 channel at its full length (64 cells, 10^4 RK-3 steps, CUDA-graph
    # replay) from n = 1, u = 0, T = 1, against the oracle run alike; the
    # result is the near-steady barometric state of Sec. V, log n linear in x
    # with slope -g/T away from the walls.
    from oracle.solver import Solver, config_from
    from paper_1708_03249_gb300 import hlb
    cfg = W.CHANNEL_1D_FP64
    steps = W.CHANNEL_1D_FP64_STEPS
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.init_equilibrium(1.0, 0.0, 0.0, 1.0)
        f0 = h.get_state().astype(np.float64)
        h.step(steps)
        got = h.get_state().astype(np.float64)
        n, u, T, q = h.moments()
    s = Solver(config_from(cfg))
    s.f = f0.reshape(s.f.shape).copy()
    s.step(steps)
    ref = s.f.reshape(-1)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    g = -cfg["ax"]
    x = (np.arange(cfg["nx"]) + 0.5) / cfg["nx"]
    inner = slice(8, cfg["nx"] - 8)
    slope = np.polyfit(x[inner], np.log(n[inner]), 1)[0]
    assert slope == pytest.approx(-g / T[inner].mean(), rel=2e-3)


@pytest.mark.parametrize("cfg", [W.scaled(W.LARGE_2D, nx=12, ny=6, Ly=6 / 12),
                                 W.make(Qx=16, Qy=16, nx=40, precision=W.FP32)])
def test_fp32_moment_sums_are_compensated(cfg):
    # Every node holds 1 in one aligned block of four velocities and 1e-8 in all
    # others.  A plain FP32 running sum that has reached 4 drops each later
    # 4e-8 partial (below half an ulp of 4), a relative loss of ~1e-7 in n; the
    # compensated sums (running sum and error term, lanes and warp tree) keep
    # them, so n agrees with the exact FP64 sum of the same values to rounding.
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(cfg, stream=_stream()) as h:
        V = h.values // h.nodes
        f = np.full((h.nodes, V), 1e-8, dtype=np.float32)
        rng = np.random.default_rng(11)
        blocks = rng.integers(0, V // 4, size=h.nodes)
        for k in range(4):
            f[np.arange(h.nodes), 4 * blocks + k] = 1.0
        h.set_state(f.reshape(-1))
        n, u, T, q = h.moments()
    exact = f.astype(np.float64).sum(axis=1)
    err = np.abs(n - exact).max() / exact.max()
    assert err < 1e-9, err


def test_fp32_moments_of_a_given_state():
    # The moments of a given FP32 state against the FP64 moments of the very
    # same values: what remains is the FP32 rounding of the velocity table and
    # of the per-term products, well below the 1e-5 bar.
    from oracle.solver import Solver, config_from
    from paper_1708_03249_gb300 import hlb
    cfg = W.scaled(W.LARGE_2D, nx=12, ny=6, Ly=6 / 12)
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.init_equilibrium(1.0, 0.3, -0.2, 1.4)
        f = h.get_state().astype(np.float64)
        f = (f * W.perturbation(f.shape, seed=7, amplitude=0.3)).astype(np.float32)
        h.set_state(f)
        mom = h.moments()
    s = Solver(config_from(cfg))
    s.f = f.astype(np.float64).reshape(s.f.shape)
    errs = moment_errors(mom, _oracle_moments([s]))
    assert max(errs.values()) < 2e-7, errs


# --- stochastic rounding of the FP32 stage outputs (hlb_set_rounding) ----------
_SR_PHYS = dict(Kn=0.2, T_left=1.0, T_right=1.4, advection=W.WENO5, precision=W.FP32, **W.gravity(0.4, 35.0))
_SR_CASES = {
    "pair_2d_16x8": (dict(Qx=8, Qy=8, nx=40, ny=6, Ly=0.3, stretch_A=0.5), None),
    "line_1d_16x8": (dict(Qx=8, Qy=8, nx=60), False),
    "persistent_1d_16x8": (dict(Qx=8, Qy=8, nx=60), True),
    "line_1d_32x16": (dict(Qx=16, Qy=16, nx=40), False),     # FMA force term with stochastic rounding
    "march_scalar_8x1": (dict(Qx=4, Qy=0, nx=40), None),
    "generic_8x2": (dict(Qx=4, Qy=2, nx=40), None),
}


@pytest.mark.parametrize("case", sorted(_SR_CASES))
def test_fp32_stochastic_rounding_parity(case):
    # every kind of FP32 stage kernel with stochastically rounded outputs, at
    # the FP32 bar against the oracle
    kw, persistent = _SR_CASES[case]
    cfg = W.make(**kw, **_SR_PHYS)
    got, mom, N, refs = run_pair(cfg, 20, stochastic=True, persistent=persistent)
    _check_fp32(got, mom, refs)
    assert N[0] == pytest.approx(refs[0].total_number(), rel=1e-6)


def test_fp32_stochastic_rounding_is_deterministic_and_takes_effect():
    # the random numbers are a hash of address, stage and values: two runs
    # give the same bits, and they differ from round-to-nearest in the last place
    from paper_1708_03249_gb300 import hlb
    cfgs = [W.make(Qx=8, Qy=8, nx=40, ny=6, Ly=0.3, **_SR_PHYS), W.make(Qx=8, Qy=8, nx=60, **_SR_PHYS)]
    out = []
    for stochastic in (True, True, False):
        with hlb.Handle(cfgs, stream=_stream()) as h:
            h.set_rounding(stochastic)
            h.init_equilibrium(1.0, 0.02, 0.0, 1.1)
            h.step(5)
            out.append(h.get_state())
    np.testing.assert_array_equal(out[0], out[1])
    diff = out[0] != out[2]
    assert 0.01 < diff.mean() < 0.9
    rel = np.abs(out[0][diff].astype(np.float64) - out[2][diff]) / np.abs(out[2][diff])
    assert rel.max() < 1e-5
    with hlb.Handle(cfgs[0]) as h:
        with pytest.raises(hlb.HlbError):
            lib = hlb.lib()
            hlb._check(lib.hlb_set_rounding(h._h, 2))


def test_double_float_erf_and_exp_of_the_node_pass():
    # the double-float exp(-z^2) and erf(z) that start the FP32 groups' half-
    # range recurrence at orders up to 10, against FP64 (Python's math module):
    # the recurrence grows an error about threefold per order, so 3^10 x their
    # error must stay below FP32 resolution
    from paper_1708_03249_gb300 import hlb
    z = np.concatenate([np.linspace(0.0, 2.5, 501), -np.linspace(1e-3, 2.5, 97), [1e-8, 1e-4, 0.05]])
    zd = torch.from_numpy(z).cuda()
    e_out = torch.zeros_like(zd)
    x_out = torch.zeros_like(zd)
    torch.cuda.synchronize()
    hlb.df_special_check(zd.data_ptr(), z.size, e_out.data_ptr(), x_out.data_ptr())
    got_erf, got_exp = e_out.cpu().numpy(), x_out.cpu().numpy()
    ref_erf = np.array([math.erf(v) for v in z])
    ref_exp = np.array([math.exp(-v * v) for v in z])
    err_exp = np.abs(got_exp / ref_exp - 1.0).max()
    nz = ref_erf != 0.0
    err_erf = np.abs(got_erf[nz] / ref_erf[nz] - 1.0).max()
    assert err_exp < 1e-13 and err_erf < 1e-13, (err_exp, err_erf)
    assert got_erf[z == 0.0].max() == 0.0
    assert 3.0 ** 10 * max(err_exp, err_erf) < 2.0 ** -24
