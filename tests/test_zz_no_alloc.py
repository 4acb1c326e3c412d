"""rsc_norm2_noalloc, the allocation-free norm, against the context-based rsc_norm2.

Callers that cannot allocate device memory (their framework's pool allocator
owns it all, or allocation is forbidden after start-up) use the variant whose
scratch is a fixed device array.  It is checked through the C ABI on two
calls in a row, with the tolerance of the other reductions (1e-12 relative).
This file is collected last so that a stop at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return _t


def test_norm2_noalloc_matches_context_norm_on_two_calls(torch):
    from paper_2508_16635_gb300 import RotatingShell, load_library
    from paper_2508_16635_gb300.rsc import NORM2_NOALLOC_MAX_N
    lib = load_library()
    gpu = RotatingShell(15, 4, 16, 1e-3, 100.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(77)
    # a ragged length spanning several blocks, then a second, shorter call that
    # must not see the first call's partial sums
    vs = [torch.tensor(rng.standard_normal(n), device="cuda") for n in (3_000_001, 70_000)]
    refs = [gpu.norm2(v) for v in vs]
    # warm-up call: the first call on a device looks up the scratch array's address
    assert lib.rsc_norm2_noalloc(ctypes.c_void_p(vs[1].data_ptr()), vs[1].numel(),
                                 ctypes.c_void_p(out.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for v, ref in zip(vs, refs):
        st = lib.rsc_norm2_noalloc(ctypes.c_void_p(v.data_ptr()), v.numel(),
                                   ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0
        torch.cuda.synchronize()
        assert abs(out.item() - ref) <= 1e-12 * ref
    # the calls allocated no device memory (the CUDA driver's free bytes and torch's allocator)
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    v = vs[0]
    # sizes beyond the fixed scratch are rejected before any launch
    st = lib.rsc_norm2_noalloc(ctypes.c_void_p(v.data_ptr()), NORM2_NOALLOC_MAX_N + 1,
                               ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 1
    gpu.close()
