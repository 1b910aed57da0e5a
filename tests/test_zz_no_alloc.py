"""hlb_moments_noalloc: the moments for callers that cannot allocate.

The entry point runs the same moments kernel as hlb_moments_dev with its
scratch in a static device array, so on the same state both must give the
same numbers; the comparison below uses the FP64 moments tolerance of the
parity tests (1e-12 relative) and is repeated on two calls in a row, since
the shared scratch keeps the previous call's contents.  This file is named
to run last: pytest collects test files in name order.
"""
import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev_moments(h, fn):
    # NaN-filled outputs on torch's current stream, which is also the
    # handle's stream (see below), so the fill is ordered before the copies
    # and an output that the call failed to write would show as NaN
    n = torch.full((h.nodes,), float("nan"), dtype=torch.float64, device="cuda")
    u = torch.full((3 * h.nodes,), float("nan"), dtype=torch.float64, device="cuda")
    T = torch.full((h.nodes,), float("nan"), dtype=torch.float64, device="cuda")
    q = torch.full((h.nodes,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.current_stream().synchronize()
    fn(n.data_ptr(), u.data_ptr(), T.data_ptr(), q.data_ptr())
    torch.cuda.synchronize()
    return [a.cpu().numpy() for a in (n, u, T, q)]


def test_moments_noalloc_matches_moments_dev_twice():
    from paper_1708_03249_gb300 import hlb
    # two velocity-set groups, so the per-instance copies are exercised
    cfgs = [W.make(Qx=4, Qy=4, nx=24, Kn=0.3, ax=-0.2, precision=W.FP32),
            W.make(Qx=8, Qy=8, nx=16, Kn=1.0, T_right=1.5, precision=W.FP32),
            W.make(Qx=4, Qy=4, nx=40, Kn=0.1, precision=W.FP32)]
    with hlb.Handle(cfgs, stream=torch.cuda.current_stream().cuda_stream) as h:
        h.init_equilibrium(1.0, 0.1, 0.0, 1.1)
        f = h.get_state().astype(np.float64) * W.perturbation(h.values, seed=4)
        h.set_state(f)
        h.step(5)
        for _ in range(2):
            ref = _dev_moments(h, h.moments_dev)
            got = _dev_moments(h, h.moments_noalloc)
            for a, b in zip(got, ref):
                assert np.all(np.isfinite(a)) and np.all(np.isfinite(b))
                np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)
            h.step(1)


def test_moments_noalloc_rejects_oversized_groups():
    from paper_1708_03249_gb300 import hlb
    cfg = W.make(Qx=2, nx=(1 << 18) + 1, advection=W.UPWIND2, precision=W.FP32)
    with hlb.Handle(cfg) as h:
        n = torch.zeros(h.nodes, dtype=torch.float64, device="cuda")
        with pytest.raises(hlb.HlbError) as e:
            h.moments_noalloc(n.data_ptr(), None, None, None)
        assert e.value.status == hlb.HLB_EINVAL
        assert "262144" in str(e.value)
