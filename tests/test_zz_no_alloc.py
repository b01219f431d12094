"""The allocation-free white-noise entry point (wm_noise_loads_noalloc).

Some callers cannot allocate device memory: a host framework whose caching
allocator owns the device, or code that may not call cudaMalloc because it can
synchronise the device.  The library offers them one entry point whose scratch
is a fixed device array.  It must give the same loads as the allocating
wm_noise_loads and as the CPU oracle, call after call (the shared array keeps
the previous call's contents), and refuse sizes beyond the array and host
output buffers with a clear error.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
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


def test_noalloc_noise_matches_allocating_entry_point_and_oracle(wm):
    from oracle import geometry as geo
    from oracle.noise import noise_loads
    from oracle.space import GluedSpace
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 2)
    N = hier.num_dofs(0)
    sp_ = GluedSpace(geo.Surface("sphere", 2, 8))
    # two calls in a row: the second reuses the scratch left by the first
    for seed, ns in [(3, 35), (11, 7)]:
        ref = hier.noise_loads(seed, ns)
        out = torch.full((ns, N), float("nan"), dtype=torch.float64, device="cuda")
        assert call_noalloc(wm, hier, seed, ns, out) == 0
        torch.testing.assert_close(out, ref, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(out.cpu().numpy(), noise_loads(sp_, seed, ns), rtol=1e-11, atol=1e-14)


def test_noalloc_rejects_sizes_beyond_the_scratch(wm):
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 2)
    per_sample = 6 * 8 * 8 * 9  # elements x (p+1)^2
    ns = SCRATCH_DOUBLES // per_sample + 1
    out = torch.zeros((1, hier.num_dofs(0)), dtype=torch.float64, device="cuda")
    assert call_noalloc(wm, hier, 0, ns, out) == wm._capi.WM_ERR_INVALID_ARG
    assert b"scratch" in wm.lib().wm_last_error()


def test_noalloc_rejects_a_host_output_buffer(wm):
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 2)
    out = torch.zeros((2, hier.num_dofs(0)), dtype=torch.float64)  # host memory
    assert call_noalloc(wm, hier, 0, 2, out) == wm._capi.WM_ERR_INVALID_ARG
    assert b"device memory" in wm.lib().wm_last_error()
    assert (out == 0).all()
