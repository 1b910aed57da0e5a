"""Out-of-memory paths, exercised without exhausting the GPU.

hlb_set_alloc_fail_test makes the n-th library allocation fail as if memory
were exhausted.  For every n up to the number of allocations hlb_create makes
for a two-group handle (tables, state buffers, scratch, work lists of both
velocity sets), the creation must answer HLB_ENOMEM and leave nothing
behind: device memory returns to its level before the loop.  The first n
beyond that count gives a working handle.
"""
import numpy as np
import pytest

from paper_1708_03249_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cfgs():
    return [W.make(Qx=4, Qy=4, nx=24, Kn=0.3, ax=-0.1, precision=W.FP32),
            W.make(Qx=8, Qy=8, nx=16, Kn=1.0, T_right=1.4, precision=W.FP32)]


def test_every_allocation_of_create_fails_cleanly():
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(_cfgs()) as h:                 # load the kernels first
        h.init_equilibrium()
        h.step(2)
        h.moments()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for k in range(1, 1000):
            hlb.set_alloc_fail_test(k)
            try:
                h = hlb.Handle(_cfgs())
            except hlb.HlbError as e:
                assert e.status == hlb.HLB_ENOMEM, (k, str(e))
                failures += 1
                continue
            hlb.set_alloc_fail_test(0)
            with h:
                h.init_equilibrium()
                h.step(3)
                n, u, T, q = h.moments()
                assert np.isfinite(n).all() and np.isfinite(T).all()
            break
        else:
            pytest.fail("hlb_create never succeeded")
    finally:
        hlb.set_alloc_fail_test(0)
    assert failures >= 20, failures
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (64 << 20), (free0, free1)


def test_injected_failure_in_a_later_allocation():
    # the staging buffer of hlb_prefetch_state is allocated on first use
    from paper_1708_03249_gb300 import hlb
    with hlb.Handle(_cfgs()) as h:
        h.init_equilibrium()
        state = torch.from_numpy(h.get_state()).pin_memory()
        hlb.set_alloc_fail_test(1)
        try:
            with pytest.raises(hlb.HlbError) as e:
                h.prefetch_state(state.data_ptr(), h.state_bytes)
            assert e.value.status == hlb.HLB_ENOMEM
        finally:
            hlb.set_alloc_fail_test(0)
        h.prefetch_state(state.data_ptr(), h.state_bytes)    # works once memory is there
        h.commit_state()
        np.testing.assert_array_equal(h.get_state(), state.numpy())
