"""ce_unconditional_static, the entry point for callers that cannot allocate
device memory at call time (an application whose GPU memory budget belongs to
its own pool, or a latency-critical loop that must not hit the implicit device
synchronisation of cudaMalloc/cudaFree).  It must reproduce ce_unconditional
bit for bit through the C ABI on consecutive calls, leave the device's free
memory unchanged (cudaMemGetInfo before and after each call), and reject grids
whose FFT intermediate does not fit its fixed buffer.

This file is collected last on purpose, and passes both alone in a fresh
process and after the other tests.
"""
import ctypes

import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def ce():
    from paper_2109_11044_gb300.build import build
    build()
    import paper_2109_11044_gb300 as mod
    mod.load_library()
    return mod


def test_static_matches_allocating_entry_point_on_two_calls(ce):
    lib = ce.load_library()
    wl = workloads.workload("shakemap512")
    ctx = ce.Context.from_workload(wl)
    R = 30   # 15 pairs of 4 MiB each: several chunks of the 16 MiB buffer
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty((R, wl.m, wl.m), dtype=torch.float32, device="cuda")
    for seed, r_offset in ((wl.sim_seed, 0), (wl.sim_seed + 1, 40)):
        ref = ctx.unconditional(R, seed, r_offset)   # allocating path
        before = ctx.info()["device_bytes"]
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]   # cudaMemGetInfo: every allocation on the device counts
        st = lib.ce_unconditional_static(ctx._ctx, R, seed, r_offset, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream))
        assert st == ce.CE_OK, lib.ce_last_error(ctx._ctx)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        assert ctx.info()["device_bytes"] == before
        assert torch.equal(out, ref)


def test_static_rejects_grids_beyond_the_buffer(ce):
    lib = ce.load_library()
    wl = workloads.workload("plain64").scaled(m=1100)   # P = 4096: 8 * 4096 * 1100 bytes per pair > 16 MiB
    ctx = ce.Context.from_workload(wl)
    out = torch.empty((2, wl.m, wl.m), dtype=torch.float32, device="cuda")
    st = lib.ce_unconditional_static(ctx._ctx, 2, 1, 0, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == ce.CE_ERR_ARG
    assert b"scratch" in lib.ce_last_error(ctx._ctx)
