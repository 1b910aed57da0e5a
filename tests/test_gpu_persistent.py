"""The persistent batched kernel (one launch per RK-3 step for a group of 1D
FP32 channels; work items of (stage, x-segment) from a queue, per-instance
progress counters, the node pass and the wall balance inside each item).

Parity with the FP64 oracle at the FP32 bar (err(M) <= 1e-5, per velocity
<= 2e-5), agreement with the per-stage launches to FP32 rounding (the moment
sums are formed in another order there), independence of the segmentation
(bit for bit: every cell's update is formed the same way whatever segment
holds it), and the launch shapes it is used for.
"""
import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _mixed(n=12, cap=70):
    # the seeded batched draws (all three velocity sets), shortened
    return [W.scaled(c, nx=min(c["nx"], cap)) for c in W.batched_instances(n)]


def test_persistent_kernel_is_used_where_eligible():
    from paper_1708_03249_gb300 import hlb
    # a 2D instance (its own group: another scheme) takes the pair kernel
    cfgs = _mixed(6) + [W.make(Qx=4, Qy=4, nx=20, ny=6, Ly=0.3, advection=W.UPWIND2, precision=W.FP32)]
    with hlb.Handle(cfgs, stream=_stream()) as h:
        forms = [h.step_form(i) for i in range(len(cfgs))]
    assert all(f["persistent"] for f in forms[:6]), forms
    assert not forms[6]["persistent"], forms
    assert all(f["segment_cells"] > 0 for f in forms[:6])
    # FP64, and a force-term form it has no instantiation of: per-stage launches
    for cfg in (W.make(Qx=4, Qy=4, nx=20, precision=W.FP64), W.make(Qx=8, Qy=8, nx=20, precision=W.FP32_TF32X3)):
        with hlb.Handle(cfg, stream=_stream()) as h:
            assert not h.step_form(0)["persistent"]
    # switched off
    with hlb.Handle(cfgs[:6], stream=_stream()) as h:
        h.set_persistent(False)
        assert not any(h.step_form(i)["persistent"] for i in range(6))


def test_persistent_matches_oracle():
    from test_gpu_parity import _check_fp32, run_pair
    got, mom, N, refs = run_pair(_mixed(12), 8)
    _check_fp32(got, mom, refs)


@pytest.mark.parametrize("adv", [W.WENO5, W.UPWIND2])
def test_persistent_ragged_segments_and_short_instances(adv):
    # instances of one work item (nx below the segment length, down to the
    # minimum of 6 cells), of several with a ragged last one, a stretched grid
    from test_gpu_parity import _check_fp32, run_pair
    cfgs = [W.make(Qx=4, Qy=4, nx=nx, advection=adv, precision=W.FP32, T_left=0.8, T_right=1.3, Kn=0.2,
                   stretch_A=A, **W.gravity(0.5, 25.0))
            for nx, A in ((6, 0.0), (7, 0.0), (23, 0.5), (131, 0.0), (250, 0.7))]
    got, mom, N, refs = run_pair(cfgs, 10)
    _check_fp32(got, mom, refs)


@pytest.mark.parametrize("Qx,Qy", [(4, 4), (8, 8), (16, 16), (16, 0)])
def test_persistent_equals_per_stage_to_rounding(Qx, Qy):
    from paper_1708_03249_gb300 import hlb
    cfgs = [W.make(Qx=Qx, Qy=Qy, nx=nx, precision=W.FP32, T_left=0.9, T_right=1.5, Kn=Kn,
                   **(W.gravity(0.6, 40.0) if Qy else {"ax": -0.6}))
            for nx, Kn in ((37, 0.05), (160, 1.0))]
    outs = []
    for persistent in (True, False):
        with hlb.Handle(cfgs, stream=_stream()) as h:
            h.set_persistent(persistent)
            assert h.step_form(0)["persistent"] == persistent
            h.init_equilibrium(1.0, 0.05, 0.02, 1.1)
            f = h.get_state().astype(np.float64) * W.perturbation(h.values, seed=41)
            h.set_state(f)
            h.step(40)
            outs.append(h.get_state().astype(np.float64))
    scale = np.abs(outs[1]).max()
    assert np.abs(outs[0] - outs[1]).max() < 2e-6 * scale


def test_autotune_keeps_the_state_and_the_result():
    # hlb_autotune times whole persistent steps (segment lengths, grids) and
    # the per-stage launches, and keeps the faster per group; it keeps the
    # state, and the steps after it agree with an untuned handle to FP32
    # rounding (bit for bit where the persistent kernel stays in use)
    from paper_1708_03249_gb300 import hlb
    cfgs = _mixed(9, cap=300)
    outs, forms = [], []
    for tune in (False, True):
        with hlb.Handle(cfgs, stream=_stream()) as h:
            h.init_equilibrium(1.0, 0.0, 0.0, 1.0)
            f = h.get_state().astype(np.float64) * W.perturbation(h.values, seed=43)
            h.set_state(f)
            before = h.get_state()
            if tune:
                segs = h.autotune()
                assert all(s > 0 for s in segs)
                assert np.array_equal(h.get_state(), before)
            forms.append([h.step_form(i)["persistent"] for i in range(len(cfgs))])
            h.step(12)
            outs.append(h.get_state().astype(np.float64))
    scale = np.abs(outs[0]).max()
    assert np.abs(outs[0] - outs[1]).max() < 2e-6 * scale
    if all(forms[1]):
        assert np.array_equal(outs[0], outs[1])
