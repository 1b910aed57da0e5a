"""hlb_prefetch_state / hlb_commit_state: a staged upload of the next state.

A state staged from page-locked memory while steps run on the current one,
then committed, must be exactly the state that hlb_set_state would have set
(byte for byte), and the steps that follow must give the same bits as after
hlb_set_state.  Several instances of two velocity sets exercise the
per-instance copies out of the staging buffer; one velocity set the buffer
swap (twice, so the old state buffer serves as staging buffer once).  A
commit with nothing staged and a buffer of the wrong size are rejected.
"""
import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cfgs(kind="groups"):
    if kind == "one_group":
        # one velocity set: the commit swaps the staging and state buffers
        return [W.make(Qx=8, Qy=8, nx=30, ny=5, Ly=0.2, Kn=0.5, ax=-0.2, precision=W.FP32),
                W.make(Qx=8, Qy=8, nx=16, Kn=1.0, T_right=1.5, precision=W.FP32)]
    if kind == "unaligned":
        # instances whose slices are not multiples of 16 bytes (6 velocities,
        # odd cell counts): the commit copies instance by instance
        return [W.make(Qx=3, nx=25, Kn=0.3, ax=-0.2, advection=W.UPWIND2, precision=W.FP32),
                W.make(Qx=4, Qy=4, nx=16, Kn=1.0, T_right=1.5, precision=W.FP32),
                W.make(Qx=3, nx=31, Kn=0.1, advection=W.UPWIND2, precision=W.FP32)]
    # two velocity sets: the commit copies the staging buffer into the groups
    # (one launch per group)
    return [W.make(Qx=4, Qy=4, nx=24, Kn=0.3, ax=-0.2, precision=W.FP32),
            W.make(Qx=8, Qy=8, nx=16, Kn=1.0, T_right=1.5, precision=W.FP32),
            W.make(Qx=4, Qy=4, nx=40, Kn=0.1, precision=W.FP32)]


@pytest.mark.parametrize("kind", ["groups", "one_group", "unaligned"])
def test_committed_state_equals_set_state_and_steps_agree(kind):
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(_cfgs(kind)) as a, hlb.Handle(_cfgs(kind)) as b:
        a.init_equilibrium(1.0, 0.0, 0.0, 1.0)
        f1 = a.get_state().astype(np.float64) * W.perturbation(a.values, seed=11, amplitude=0.05)
        pinned = torch.empty(a.values, dtype=torch.float32, pin_memory=True)
        pinned.numpy()[:] = f1.astype(np.float32)
        a.step(3)                                   # running on the old state
        a.prefetch_state(pinned.data_ptr(), a.state_bytes)
        a.step(2)                                   # overlaps the staged copy
        a.commit_state()
        got = a.get_state()
        np.testing.assert_array_equal(got, pinned.numpy())
        b.set_state(pinned.numpy())
        a.step(4)                                   # a graph is captured again after a swap
        b.step(4)
        np.testing.assert_array_equal(a.get_state(), b.get_state())
        with pytest.raises(hlb.HlbError) as e:     # the staged state was consumed
            a.commit_state()
        assert e.value.status == hlb.HLB_EINVAL
        # a second round through the same buffers (the old state buffer is now staging)
        f2 = pinned.numpy() * np.float32(1.01)
        pinned2 = torch.from_numpy(f2).pin_memory()
        a.prefetch_state(pinned2.data_ptr(), a.state_bytes)
        a.step(1)
        a.commit_state()
        b.set_state(pinned2.numpy())
        a.step(3)
        b.step(3)
        np.testing.assert_array_equal(a.get_state(), b.get_state())


def test_second_prefetch_replaces_the_first_and_bad_size_is_rejected():
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(_cfgs()) as h:
        h.init_equilibrium(1.0, 0.0, 0.0, 1.0)
        base = h.get_state()
        first = torch.from_numpy(base * np.float32(0.5)).pin_memory()
        second = torch.from_numpy(base * np.float32(2.0)).pin_memory()
        h.prefetch_state(first.data_ptr(), h.state_bytes)
        h.prefetch_state(second.data_ptr(), h.state_bytes)
        h.commit_state()
        np.testing.assert_array_equal(h.get_state(), second.numpy())
        with pytest.raises(hlb.HlbError) as e:
            h.prefetch_state(first.data_ptr(), h.state_bytes - 4)
        assert e.value.status == hlb.HLB_EINVAL


def test_autotune_keeps_the_state_and_the_results():
    # hlb_autotune only changes the segment length of the marching kernels: the
    # state survives the tuning launches and the steps after it give the same
    # bits as an untuned handle's (each cell's update does not depend on where
    # the segments end).  Two velocity sets, 1D and 2D instances.
    from paper_1708_03249_gb300 import hlb
    cfgs = [W.make(Qx=8, Qy=8, nx=300, Kn=0.3, ax=-0.2, precision=W.FP32),
            W.make(Qx=4, Qy=4, nx=90, ny=7, Ly=0.3, Kn=0.5, precision=W.FP32)]
    with hlb.Handle(cfgs) as a, hlb.Handle(cfgs) as b:
        for h in (a, b):
            # the per-stage launches (the tuner may also move a group to the
            # persistent kernel, which rounds the moment sums in another order;
            # tests/test_gpu_persistent.py covers that)
            h.set_persistent(False)
            h.init_equilibrium(1.0, 0.05, 0.0, 1.0)
            h.step(2)
        before = a.get_state()
        seg = a.autotune()
        assert len(seg) == 2 and all(v >= 12 and v % 6 == 0 for v in seg)
        np.testing.assert_array_equal(a.get_state(), before)
        a.step(5)
        b.step(5)
        np.testing.assert_array_equal(a.get_state(), b.get_state())



def test_async_moments_match_and_overlap_the_next_steps():
    # hlb_moments_async of each step in a staged-upload loop (the end-to-end
    # pattern: commit, prefetch the next state, one step, moments) gives the
    # same moments and the same final state, bit for bit, as the synchronous
    # loop; a multi-step call after a request (which reuses the buffer the
    # moments read) is ordered behind it.
    from paper_1708_03249_gb300 import hlb
    cfgs = _cfgs("one_group")
    with hlb.Handle(cfgs) as a, hlb.Handle(cfgs) as b:
        for h in (a, b):
            h.init_equilibrium(1.0, 0.02, 0.0, 1.0)
        base = a.get_state().astype(np.float64)
        states = [torch.from_numpy((base * W.perturbation(a.values, seed=30 + k, amplitude=0.04))
                                   .astype(np.float32)).pin_memory() for k in range(4)]
        nodes = a.nodes
        outs = [[torch.empty(c * nodes, dtype=torch.float64).pin_memory() for c in (1, 3, 1, 1)] for _ in range(4)]
        a.prefetch_state(states[0].data_ptr(), a.state_bytes)
        for k in range(4):
            a.commit_state()
            if k + 1 < 4:
                a.prefetch_state(states[k + 1].data_ptr(), a.state_bytes)
            a.step(1)
            a.moments_async(*[t.numpy() for t in outs[k]])
        a.moments_wait()
        for k in range(4):
            b.set_state(states[k].numpy())
            b.step(1)
            ref = b.moments()
            for got, r in zip(outs[k], ref):
                np.testing.assert_array_equal(got.numpy(), np.asarray(r).reshape(-1))
        np.testing.assert_array_equal(a.get_state(), b.get_state())
        # a request, then three steps (the third writes the buffer it reads)
        a.moments_async(*[t.numpy() for t in outs[0]])
        a.step(3)
        b.step(3)
        a.moments_wait()
        np.testing.assert_array_equal(a.get_state(), b.get_state())
        np.testing.assert_array_equal(outs[0][0].numpy(), np.asarray(ref[0]).reshape(-1))


@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_checkpoint_resume_is_bit_exact(prec):
    # run(2n) == run(n), checkpoint (hlb_get_state), restore into a fresh
    # handle (hlb_set_state), run(n): the same bits.  Two velocity sets and a
    # 2D instance (group streams, pair and line kernels); n = 37 crosses the
    # captured graph's 30-step boundary.
    from paper_1708_03249_gb300 import hlb
    cfgs = [dict(c, precision=prec) for c in _cfgs("groups")] + \
           [W.make(Qx=8, Qy=8, nx=20, ny=6, Ly=0.3, Kn=0.4, ax=-0.3, ay=-0.1, precision=prec)]
    n = 37
    with hlb.Handle(cfgs) as a:
        a.init_equilibrium(1.0, 0.05, 0.0, 1.1)
        f0 = a.get_state().astype(np.float64) * W.perturbation(a.values, seed=17, amplitude=0.05)
        a.set_state(f0)
        a.step(2 * n)
        whole = a.get_state()
    with hlb.Handle(cfgs) as b:
        b.set_state(f0)
        b.step(n)
        ckpt = b.get_state().copy()
    with hlb.Handle(cfgs) as c:
        c.set_state(ckpt)
        c.step(n)
        resumed = c.get_state()
    assert resumed.dtype == whole.dtype
    assert np.array_equal(resumed.view(np.uint8), whole.view(np.uint8))


@pytest.mark.parametrize("kind", ["groups", "unaligned"])
def test_device_state_io_matches_host_state_io(kind):
    # hlb_set_state_dev / hlb_get_state_dev between a device buffer in the
    # caller's layout and the groups' buffers: the same bytes as the host forms
    # (one launch per group when every slice is a multiple of 16 bytes, one
    # copy per instance otherwise)
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(_cfgs(kind), stream=torch.cuda.current_stream().cuda_stream) as h:
        h.init_equilibrium(1.0, 0.0, 0.0, 1.0)
        f = (h.get_state().astype(np.float64) * W.perturbation(h.values, seed=17, amplitude=0.05)).astype(np.float32)
        d_in = torch.from_numpy(f).cuda()
        torch.cuda.synchronize()
        h.set_state_dev(d_in.data_ptr(), h.state_bytes)
        np.testing.assert_array_equal(h.get_state(), f)
        h.step(2)
        d_out = torch.full((h.values,), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        h.get_state_dev(d_out.data_ptr(), h.state_bytes)
        torch.cuda.current_stream().synchronize()
        np.testing.assert_array_equal(d_out.cpu().numpy(), h.get_state())


@pytest.mark.parametrize("kind", ["groups", "one_group"])
def test_device_moments_match_host_moments(kind):
    # hlb_moments_dev (several instances: each group's moments kernel writes
    # its nodes straight into the caller's arrays) against hlb_moments
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(_cfgs(kind), stream=torch.cuda.current_stream().cuda_stream) as h:
        h.init_equilibrium(1.0, 0.02, 0.0, 1.1)
        h.step(3)
        ref = h.moments()
        N = h.nodes
        outs = [torch.full((k * N,), float("nan"), dtype=torch.float64, device="cuda") for k in (1, 3, 1, 1)]
        torch.cuda.synchronize()
        h.moments_dev(*(o.data_ptr() for o in outs))
        torch.cuda.current_stream().synchronize()
        for got, want in zip(outs, ref):
            np.testing.assert_array_equal(got.cpu().numpy(), np.asarray(want).reshape(-1))
