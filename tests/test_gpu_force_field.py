"""Per-node acceleration fields (hlb_set_force_field) against the FP64 oracle.

The oracle applies the force term of App. A node by node with a(node) = the
uniform acceleration plus the field (its pins: the per-node homogeneous closed
form and the barometric residual in a potential, tests/test_oracle_solver.py).
Here the CUDA path runs the same seeded state and fields through every kind of
stage kernel (2D pair kernel, 1D line kernel with FMA and tensor-core force
terms, FP64 kernel) and is compared element by element with the tolerances of
the parity tests (FP32: moments within 1e-5, every bulk velocity within 2e-5
of its own scale; FP64: 1e-10 of the state's maximum).  Also: removing the
field restores the field-free step bit for bit, and a constant field equals
the same uniform acceleration within FP32 rounding.
"""
import math

import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _potential_field(cfg, seed):
    """a = -grad V of a smooth seeded potential V(x, y) on the instance's cell
    centres (uniform grid in x on [0, Lx], periodic in y)."""
    rng = np.random.default_rng(seed)
    nx, ny = cfg["nx"], cfg.get("ny", 1)
    x = (np.arange(nx) + 0.5) / nx * cfg["Lx"]
    y = (np.arange(ny) + 0.5) / ny * cfg.get("Ly", 1.0)
    X, Y = np.meshgrid(x, y)                                     # (ny, nx)
    c1, c2, c3 = rng.uniform(0.1, 0.3, 3)
    ky = 2 * np.pi / cfg.get("Ly", 1.0)
    ax = -(c1 + 2 * np.pi * c2 * np.cos(2 * np.pi * X / cfg["Lx"]) * (1 + 0.3 * np.sin(ky * Y)))
    ay = -(c2 * np.sin(2 * np.pi * X / cfg["Lx"]) * 0.3 * ky * np.cos(ky * Y)) if ny > 1 else np.zeros_like(X)
    az = c3 * np.cos(np.pi * X / cfg["Lx"])
    return ax, ay, az


def _moment_errors(mom, ref):
    n, u, T, q = mom
    rn, ru, rT, rq = ref
    sT = np.abs(rT).max()
    return {"n": np.abs(n - rn).max() / np.abs(rn).max(),
            "u": np.abs(u - ru).max() / max(np.abs(ru).max(), math.sqrt(sT)),
            "T": np.abs(T - rT).max() / sT,
            "q": np.abs(q - rq).max() / max(np.abs(rq).max(), np.abs(rn).max() * sT ** 1.5)}


def _run(cfg, steps, fields, seed=5):
    from oracle.solver import Solver, config_from
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.init_equilibrium(1.0, 0.05, 0.0, 1.0)
        f0 = h.get_state().astype(np.float64) * W.perturbation(h.values, seed=seed, amplitude=0.05)
        h.set_state(f0)
        f0 = h.get_state().astype(np.float64)
        if fields is not None:
            h.set_force_field(0, *[a.reshape(-1) for a in fields])
        h.step(steps)
        got = h.get_state().astype(np.float64)
        mom = h.moments()
    oc = config_from(cfg)
    if fields is not None:
        oc.ax_field, oc.ay_field, oc.az_field = fields
    s = Solver(oc)
    s.f = f0.reshape(s.f.shape).copy()
    s.step(steps)
    return got, mom, s


def _check(cfg, got, mom, s):
    ref = s.f.reshape(-1, s.vs.V)
    g = got.reshape(ref.shape)
    if cfg["precision"] == W.FP64:
        assert np.abs(g - ref).max() < 1e-10 * np.abs(ref).max()
        return
    n, u, T, q = s.moments()
    errs = _moment_errors(mom, (n.reshape(-1), u.reshape(-1, 3), T.reshape(-1), q.reshape(-1)))
    assert max(errs.values()) < 1e-5, errs
    scale = np.abs(ref).max(axis=0)
    sel = scale >= 1e-6 * np.abs(ref).max()
    assert (np.abs(g - ref)[:, sel] / scale[sel]).max() < 2e-5


CASES = {
    "2d_fp32_pair_16x8": W.make(Qx=8, Qy=8, nx=27, ny=6, Ly=0.3, precision=W.FP32, T_left=1.0, T_right=1.5,
                                ax=-0.2, ay=0.1, Kn=0.5),
    "1d_fp32_line_16x8": W.make(Qx=8, Qy=8, nx=45, precision=W.FP32, T_left=0.8, T_right=1.2, ax=-0.1, Kn=0.2),
    "1d_fp32_line_32x16_tensor": W.make(Qx=16, Qy=16, nx=30, precision=W.FP32, T_left=1.0, T_right=1.3,
                                        Kn=0.3),
    "1d_fp64": W.make(Qx=4, Qy=4, nx=24, precision=W.FP64, advection=W.UPWIND2, T_left=1.0, T_right=1.0,
                      ax=-0.1, Kn=0.1),
    "2d_fp32_qz_8x4": W.make(Qx=4, Qy=4, Qz=4, nx=14, ny=4, Ly=0.2, precision=W.FP32, T_left=1.0,
                             T_right=2.0, Kn=0.5),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_force_field_matches_oracle(name):
    cfg = CASES[name]
    fields = _potential_field(cfg, seed=len(name))
    got, mom, s = _run(cfg, 6, fields)
    _check(cfg, got, mom, s)


def test_removed_field_restores_the_field_free_step():
    from paper_1708_03249_gb300 import hlb
    cfg = CASES["1d_fp32_line_16x8"]
    fields = _potential_field(cfg, seed=3)
    out = []
    for with_field in (False, True):
        with hlb.Handle(cfg, stream=_stream()) as h:
            h.init_equilibrium(1.0, 0.05, 0.0, 1.0)
            if with_field:
                h.set_force_field(0, *[a.reshape(-1) for a in fields])
                h.step(2)
                h.set_force_field(0)                    # removed: no field launch any more
                h.init_equilibrium(1.0, 0.05, 0.0, 1.0)
            h.step(5)
            out.append(h.get_state())
    np.testing.assert_array_equal(out[0], out[1])


def test_constant_field_equals_uniform_acceleration():
    from paper_1708_03249_gb300 import hlb
    cfg = W.make(Qx=8, Qy=8, nx=40, precision=W.FP32, T_left=1.0, T_right=1.4, Kn=0.3)
    a = (-0.35, 0.2)
    out = []
    for mode in ("uniform", "field"):
        with hlb.Handle(cfg, stream=_stream()) as h:
            h.init_equilibrium(1.0, 0.0, 0.0, 1.0)
            if mode == "uniform":
                h.set_force(a[0], a[1])
            else:
                h.set_force_field(0, np.full(cfg["nx"], a[0]), np.full(cfg["nx"], a[1]))
            h.step(20)
            out.append(h.get_state().astype(np.float64))
    assert np.abs(out[0] - out[1]).max() < 2e-6 * np.abs(out[0]).max()


def test_field_arguments_are_checked():
    from paper_1708_03249_gb300 import hlb
    cfg = CASES["1d_fp32_line_16x8"]
    with hlb.Handle(cfg, stream=_stream()) as h:
        with pytest.raises(ValueError):
            h.set_force_field(0, np.zeros(cfg["nx"] - 1))
        bad = np.zeros(cfg["nx"])
        bad[3] = np.nan
        with pytest.raises(hlb.HlbError) as e:
            h.set_force_field(0, bad)
        assert e.value.status == hlb.HLB_EINVAL
