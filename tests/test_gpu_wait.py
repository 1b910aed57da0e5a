"""Bounded device waits and the launch counter, on the GPU.

The marching stage kernels wait on their bulk-copy pipeline with a time
limit.  The test hook of the C ABI withholds the copies of one pipeline step
in every marching CTA, so that those waits run out: no fault and no trap, the
waits give up, record HLB_ETIMEOUT in the device error word and the CTAs
leave at their next barrier.  In the persistent batched kernel the same hook
withholds one work item's count on its instance's progress counter, so that
the items of the next stage of that instance wait on it until their bound runs
out (a per-instance device barrier that never opens); the launch's abort flag
then ends every CTA.  The context must stay usable, and once the hook is
cleared the handle must step exactly as a fresh one does."""
import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    # 2D FP32: the pair kernel (two rows x two cells per iteration)
    "pair_fp32_2d": W.make(Qx=4, Qy=4, nx=40, ny=6, Ly=0.3, advection=W.WENO5, precision=W.FP32,
                           T_left=1.0, T_right=1.5, ax=-0.2, ay=0.1, Kn=0.3),
    # 1D FP64: the scalar marching kernel
    "scalar_fp64_1d": W.scaled(W.CHANNEL_1D_FP64, nx=40),
    # 1D FP32: the persistent batched kernel (two instances of one velocity
    # set, per-instance progress counters), and the per-stage line kernel
    "persistent_fp32_1d": [W.make(Qx=8, Qy=8, nx=60, advection=W.WENO5, precision=W.FP32, T_left=1.0,
                                  T_right=1.4, Kn=0.3, **W.gravity(0.3, 20.0)),
                           W.make(Qx=8, Qy=8, nx=150, advection=W.WENO5, precision=W.FP32, T_left=1.0,
                                  T_right=0.7, Kn=0.1, ax=-0.4)],
    "line_fp32_1d": W.make(Qx=8, Qy=8, nx=60, advection=W.WENO5, precision=W.FP32, T_left=1.0, T_right=1.4,
                           Kn=0.3, **W.gravity(0.3, 20.0)),
}
PER_STAGE = {"line_fp32_1d"}


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _run(cfg, steps, hook, graphs, persistent=True):
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.set_options(use_graphs=graphs)
        h.set_persistent(persistent)
        if hook:
            h.init_equilibrium()
            h.set_wait_test(True, 0.002)
            h.step(steps)
            with pytest.raises(hlb.HlbError) as e:
                h.moments()
            assert e.value.status == hlb.HLB_ETIMEOUT
            # the error word was read and cleared; the context still works
            h.set_wait_test(False)
        h.init_equilibrium(1.0, 0.05, 0.0, 1.1)
        f0 = h.get_state().astype(np.float64)
        h.set_state(f0 * W.perturbation(f0.shape, seed=4, amplitude=0.05))
        h.step(steps)
        out = h.get_state()
        n, u, T, q = h.moments()
    assert np.isfinite(out).all() and np.isfinite(T).all()
    return out


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("graphs,steps", [(False, 1), (True, 30)])
def test_wait_runs_out_and_handle_recovers(name, graphs, steps):
    cfg = CASES[name]
    persistent = name not in PER_STAGE
    got = _run(cfg, steps, hook=True, graphs=graphs, persistent=persistent)
    ref = _run(cfg, steps, hook=False, graphs=graphs, persistent=persistent)
    np.testing.assert_array_equal(got, ref)


def test_wait_limit_is_validated():
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(CASES["pair_fp32_2d"], stream=_stream()) as h:
        for bad in (-1.0, 61.0, float("nan")):
            with pytest.raises(hlb.HlbError) as e:
                h.set_wait_test(False, bad)
            assert e.value.status == hlb.HLB_EINVAL


@pytest.mark.parametrize("graphs", [False, True])
def test_launch_count(graphs):
    from paper_1708_03249_gb300 import hlb
    # marching path: per stage sums, factor lines, wall, stage kernel
    with hlb.Handle(CASES["pair_fp32_2d"], stream=_stream()) as h:
        h.set_options(use_graphs=graphs)
        h.init_equilibrium()
        h.launch_count(reset=True)
        h.step(30)
        assert h.launch_count() == 30 * 12
    # generic path (a force along p_z): per stage wall and stage kernel
    cfg = W.make(Qx=3, Qy=4, Qz=2, nx=10, ny=6, Ly=0.6, precision=W.FP64, az=0.2, Kn=0.2)
    with hlb.Handle(cfg, stream=_stream()) as h:
        h.set_options(use_graphs=graphs)
        h.init_equilibrium()
        h.launch_count(reset=True)
        h.step(30)
        assert h.launch_count() == 30 * 6
    # persistent batched kernel: one launch per step per group
    with hlb.Handle(CASES["persistent_fp32_1d"], stream=_stream()) as h:
        h.set_options(use_graphs=graphs)
        h.init_equilibrium()
        assert h.step_form(0)["persistent"]
        h.launch_count(reset=True)
        h.step(30)
        assert h.launch_count() == 30
