"""FP32 parity with the FP64 oracle at the configurations' stated sizes and
lengths (the FP32 bar: moments within 1e-5 of the oracle).

The oracle's long runs are stored by ``tests/golden/make_long_runs.py`` (which
calls only the oracle): the final n, u, T, q per node after the stated number
of RK-3 steps, from the oracle's rest equilibrium times seeded factors, rounded
to FP32.  Here the CUDA path starts from exactly that FP32 state and runs the
same steps.  err(M) = max|M - M_ref| / max(max|M_ref|, s_M) with s_n = max n,
s_u = sqrt(max T), s_T = max T, s_q = max n T^{3/2}, per instance.

  stretched channel (512 cells, A = 0.9, Q = 8 x 8, T = 0.5 / 1.5, g = 0.5 at
      30 deg) at Kn = 0.01, 0.1, 1, 10: 3000 steps each;
  the 2D box's velocity set and physics (Q = 16 x 16, Kn = 0.05) on 24 x 24
      cells: 2000 steps;
  the large channel's velocity set and physics (16 x 8 x 8 velocities, Kn =
      0.5, its cell size and time step) on a 24 x 24 window: 500 steps;
  the first 64 seeded batched instances: 5000 steps (500 for the sixteen
      largest, whose oracle runs would exceed 5000 s of one core);
  the 2D box at its full size (256 x 256 x 512 velocities): one step, checked
      on sampled nodes against the oracle on 19 x 19 windows around them.
"""
import json
import math
import os
import sys

import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
LONG = os.path.join(GOLDEN, "long_runs")
if GOLDEN not in sys.path:
    sys.path.insert(0, GOLDEN)


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _load(name):
    path = os.path.join(LONG, name + ".npz")
    if not os.path.exists(path):
        pytest.skip(f"golden file {os.path.basename(path)} not written yet (tests/golden/make_long_runs.py)")
    d = np.load(path)
    return {k: d[k] for k in d.files}


def _errors(mom, ref, sl=slice(None)):
    n, u, T, q = (np.asarray(a, dtype=np.float64) for a in mom)
    rn, ru, rT, rq = ref["n"], ref["u"], ref["T"], ref["q"]
    n, u, T, q = n[sl], u.reshape(-1, 3)[sl], T[sl], q[sl]
    sT = np.abs(rT).max()
    return {"n": np.abs(n - rn).max() / np.abs(rn).max(),
            "u": np.abs(u - ru).max() / max(np.abs(ru).max(), math.sqrt(sT)),
            "T": np.abs(T - rT).max() / sT,
            "q": np.abs(q - rq).max() / max(np.abs(rq).max(), np.abs(rn).max() * sT ** 1.5)}


def _run(cfgs, states, steps, stochastic=False):
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(cfgs, stream=_stream()) as h:
        h.set_rounding(stochastic)
        h.set_state(np.concatenate([s.reshape(-1) for s in states]).astype(np.float32))
        h.step(steps)
        mom = h.moments()
        N, _ = h.diag()
    return mom, N


@pytest.mark.parametrize("stochastic", [False, True], ids=["nearest", "stochastic"])
@pytest.mark.parametrize("Kn", W.CHANNEL_1D_STRETCHED_KN)
def test_fp32_stretched_channel_at_length(Kn, stochastic):
    from make_long_runs import initial_state
    ref = _load(f"stretched_kn{Kn:g}")
    cfg = json.loads(str(ref["config"]))
    assert cfg == W.channel_1d_stretched(Kn)
    mom, N = _run([cfg], [initial_state(cfg, int(ref["seed"]))], int(ref["steps"]), stochastic)
    errs = _errors(mom, ref)
    assert max(errs.values()) < 1e-5, errs
    assert N[0] == pytest.approx(float(ref["N"]), rel=1e-5)


@pytest.mark.parametrize("stochastic", [False, True], ids=["nearest", "stochastic"])
def test_fp32_box_q16_at_length(stochastic):
    from make_long_runs import BOX_N, initial_state
    ref = _load(f"box{BOX_N}")
    cfg = json.loads(str(ref["config"]))
    assert cfg == W.scaled(W.BOX_2D, nx=BOX_N, ny=BOX_N)
    mom, N = _run([cfg], [initial_state(cfg, int(ref["seed"]))], int(ref["steps"]), stochastic)
    errs = _errors(mom, ref)
    assert max(errs.values()) < 1e-5, errs
    assert N[0] == pytest.approx(float(ref["N"]), rel=1e-5)


@pytest.mark.parametrize("stochastic", [False, True], ids=["nearest", "stochastic"])
def test_fp32_large_channel_window_at_length(stochastic):
    from make_long_runs import LARGE_N, initial_state, large_window
    ref = _load(f"large{LARGE_N}")
    cfg = json.loads(str(ref["config"]))
    assert cfg == large_window()
    mom, N = _run([cfg], [initial_state(cfg, int(ref["seed"]))], int(ref["steps"]), stochastic)
    errs = _errors(mom, ref)
    assert max(errs.values()) < 1e-5, errs
    assert N[0] == pytest.approx(float(ref["N"]), rel=1e-5)


def _batched_at_length(stochastic):
    # one handle per run length, all its instances advanced together;
    # per instance: the largest err(M) and the relative error of N
    from make_long_runs import BATCH_COUNT, initial_state
    from paper_1708_03249_gb300 import hlb
    insts = W.batched_instances(BATCH_COUNT)
    refs = {}
    for i in range(BATCH_COUNT):
        ref = _load(f"batched_{i:02d}")
        assert json.loads(str(ref["config"])) == insts[i]
        refs[i] = ref
    by_len = {}
    for i, ref in refs.items():
        by_len.setdefault(int(ref["steps"]), []).append(i)
    assert set(by_len) <= {W.BATCH_STEPS, 500}
    out = {}
    for steps, ids in by_len.items():
        with hlb.Handle([insts[i] for i in ids], stream=_stream()) as h:
            h.set_rounding(stochastic)
            h.set_state(np.concatenate([initial_state(insts[i], int(refs[i]["seed"])).reshape(-1) for i in ids])
                        .astype(np.float32))
            h.step(steps)
            mom = h.moments()
            N, _ = h.diag()
        off = 0
        for k, i in enumerate(ids):
            nodes = insts[i]["nx"] * insts[i]["ny"]
            errs = _errors(mom, refs[i], slice(off, off + nodes))
            out[i] = (max(errs.values()), abs(N[k] / float(refs[i]["N"]) - 1.0), errs)
            off += nodes
    assert len(out) == BATCH_COUNT
    return out, refs


def test_fp32_batched_instances_at_length_stochastic_rounding():
    # every one of the 64 instances at its stated length within the bar, with
    # the stage outputs rounded stochastically (hlb_set_rounding)
    out, _ = _batched_at_length(True)
    for i, (worst, dN, errs) in out.items():
        assert worst < 1e-5, (i, errs)
        assert dN < 1e-5, (i, dN)


def test_fp32_batched_instances_at_length_nearest():
    # Round to nearest drops a stage's increment dt L once it is below half
    # an ulp: a value stops changing when the residual max|f^{n+1} - f^n| /
    # (dt max f) falls below about 2^-24 / dt, short of the steady state.
    # Instances whose oracle run ends above that threshold must meet the bar;
    # those that end below it (steady to the last digits FP32 can resolve per
    # step) must stay within ten times it, and stochastic rounding must bring
    # each of them within it.
    out, refs = _batched_at_length(False)
    stuck = [i for i in out if float(refs[i]["residual"]) < 2.0 ** -24 / float(refs[i]["dt"])]
    for i, (worst, dN, errs) in out.items():
        if i not in stuck:
            assert worst < 1e-5, (i, errs)
            assert dN < 1e-5, (i, dN)
        else:
            assert worst < 1e-4, (i, errs)
    assert stuck
    sr, _ = _batched_at_length(True)
    for i in stuck:
        assert sr[i][0] < 1e-5, (i, sr[i])


def test_every_long_run_case_has_its_golden_file():
    # the stored runs cover every case tests/golden/make_long_runs.py defines
    from make_long_runs import cases
    missing = [name for name, *_ in cases() if not os.path.exists(os.path.join(LONG, name + ".npz"))]
    assert not missing, missing


def test_fp32_box_full_size_sampled_nodes():
    # The 2D box at its stated size (256 x 256 cells, 512 velocities), one RK-3
    # step from a perturbed equilibrium; the oracle steps a 19 x 19 window
    # around each sampled node (the RK-3 stencil reaches 9 cells), whose centre
    # is then exact.
    from oracle.solver import Solver, config_from
    from paper_1708_03249_gb300 import hlb
    cfg = W.BOX_2D
    nx, ny = cfg["nx"], cfg["ny"]
    with hlb.Handle(cfg, stream=_stream()) as h:
        V = h.values // h.nodes
        h.init_equilibrium(1.0, 0.05, -0.02, 1.1)
        f = h.get_state().reshape(ny, nx, V).astype(np.float64)
        f *= W.perturbation(f.shape, seed=31, amplitude=0.02)
        f = f.astype(np.float32)
        h.set_state(f)
        N0 = h.diag()[0][0]
        h.step(1)
        got = h.get_state().reshape(ny, nx, V)
        N1 = h.diag()[0][0]
        dt = h.dt()
    assert N1 == pytest.approx(N0, rel=1e-5)
    rng = np.random.default_rng(6)
    samples = [(0, 7), (nx - 1, 200), (3, 255), (nx - 5, 0)] + \
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
