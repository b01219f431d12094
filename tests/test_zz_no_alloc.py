"""The allocation-free white-noise entry point (wm_noise_loads_noalloc).

Some callers cannot allocate device memory -- code running while a CUDA graph
is captured, or a framework whose own allocator owns the device -- so the
library offers one entry point whose scratch is a fixed device array.  It must
give the same loads as the allocating wm_noise_loads, call after call (the
shared array keeps the previous call's contents), and refuse sizes beyond the
array with a clear error.  This file is collected last on purpose.
"""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu

SCRATCH_DOUBLES = 1 << 22


@pytest.fixture(scope="module")
def wm():
    from paper_2605_24882_gb300 import build as b
    b.build()
    import paper_2605_24882_gb300 as wm
    return wm


def call_noalloc(wm, hier, seed, ns, out):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = wm.lib().wm_noise_loads_noalloc(hier._h, seed, ns, C.c_void_p(out.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc


def test_noalloc_noise_matches_allocating_entry_point(wm):
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 2)
    N = hier.num_dofs(0)
    # two calls in a row: the second reuses the scratch left by the first
    for seed, ns in [(3, 35), (11, 7)]:
        ref = hier.noise_loads(seed, ns)
        out = torch.full((ns, N), float("nan"), dtype=torch.float64, device="cuda")
        assert call_noalloc(wm, hier, seed, ns, out) == 0
        torch.testing.assert_close(out, ref, rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_sizes_beyond_the_scratch(wm):
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 2)
    per_sample = 6 * 8 * 8 * 9  # elements x (p+1)^2
    ns = SCRATCH_DOUBLES // per_sample + 1
    out = torch.zeros((1, hier.num_dofs(0)), dtype=torch.float64, device="cuda")
    assert call_noalloc(wm, hier, 0, ns, out) == wm._capi.WM_ERR_INVALID_ARG
    assert b"scratch" in wm.lib().wm_last_error()
