"""aqmp_correlate_noalloc: the correlation for callers that may not allocate
device memory (memory owned by another allocator or a fixed budget, loops
that reserve everything at start-up).  It keeps its scratch in static device
arrays, so its result must equal the allocating entry point's run of the
same kernel (aqmp_correlate with gemm 3, the dense exact tensor-core
kernel) bit for bit, call after call, although every call reuses (and
overwrites) the same arrays.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    assert torch.cuda.is_available()
    return aqmp


def _noalloc(aqmp, b, dict_id, blocks):
    L = blocks.shape[0]
    M = aqmp.aqmp_num_atoms(b, dict_id)
    out = torch.full((L, M, 2), float("nan"), dtype=torch.float32, device="cuda")
    rc = aqmp.load_library().aqmp_correlate_noalloc(b, dict_id, ctypes.c_void_p(blocks.data_ptr()), L,
                                                   ctypes.c_void_p(out.data_ptr()),
                                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


def test_noalloc_equals_allocating_entry_point_on_consecutive_calls(lib):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    cases = [(8, 0, 300), (16, 2, 1000), (8, 0, 77), (4, 1, 4097)]
    for b, dict_id, L in cases:
        blocks = torch.randint(0, 256, (L, b, b), dtype=torch.uint8, device="cuda", generator=gen)
        blocks[0] = 255
        rc, got = _noalloc(lib, b, dict_id, blocks)
        assert rc == 0, lib.load_library().aqmp_last_error()
        ref = lib.aqmp_correlate(b, dict_id, blocks, gemm=3)
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), (b, dict_id, L)


def test_noalloc_calls_allocate_no_device_memory(lib):
    """What the entry point exists for: once every kernel it uses has been
    loaded (a warm-up call of each case), further calls over several sides
    and dictionaries leave the device's free memory, the default
    stream-ordered pool and PyTorch's reservation where they were."""
    raw = lib.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(4, 0, 5000), (8, 1, 777), (16, 2, 300), (16, 0, 1024), (8, 0, 64)]
    bufs = []
    for b, dict_id, L in cases:
        blocks = torch.randint(0, 256, (L, b, b), dtype=torch.uint8, device="cuda")
        out = torch.empty((L, lib.aqmp_num_atoms(b, dict_id), 2), dtype=torch.float32, device="cuda")
        bufs.append((b, dict_id, L, blocks, out))

    def run_all():
        for b, dict_id, L, blocks, out in bufs:
            rc = raw.aqmp_correlate_noalloc(b, dict_id, ctypes.c_void_p(blocks.data_ptr()), L,
                                            ctypes.c_void_p(out.data_ptr()), stream)
            assert rc == 0, raw.aqmp_last_error()
        torch.cuda.synchronize()

    run_all()                                  # loads every kernel and builds every table once
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    pool0 = _default_pool_used()
    for _ in range(3):
        run_all()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == reserved0
    assert _default_pool_used() == pool0
    assert abs(free1 - free0) <= 2 << 20, (free0, free1)


def _default_pool_used():
    """Bytes in use in the current device's default stream-ordered pool
    (cudaMemPoolAttrUsedMemCurrent), or None when the CUDA Python bindings
    are not installed."""
    try:
        from cuda.bindings import runtime as rt
    except ImportError:
        return None
    err, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    if err != rt.cudaError_t.cudaSuccess:
        return None
    err, used = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
    return int(used) if err == rt.cudaError_t.cudaSuccess else None


def test_noalloc_refuses_a_capturing_stream(lib):
    """A call cannot be captured into a graph (it waits for its stream):
    on a capturing stream it returns AQMP_E_UNSUPPORTED and queues nothing,
    and the capture still ends cleanly."""
    raw = lib.load_library()
    blocks = torch.zeros((8, 8, 8), dtype=torch.uint8, device="cuda")
    out = torch.zeros((8, 128, 2), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        out.mul_(1.0)                          # the capture holds one node of its own
        rc = raw.aqmp_correlate_noalloc(8, 0, ctypes.c_void_p(blocks.data_ptr()), 8,
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert rc == -8 and b"captured" in raw.aqmp_last_error()


def test_noalloc_rejects_requests_beyond_its_static_limits(lib):
    raw = lib.load_library()
    blocks = torch.zeros((16385, 16, 16), dtype=torch.uint8, device="cuda")
    out = torch.zeros((16385, 512, 2), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = raw.aqmp_correlate_noalloc(16, 0, ctypes.c_void_p(blocks.data_ptr()), 16385,
                                    ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == -1 and b"static scratch" in raw.aqmp_last_error()
    rc = raw.aqmp_correlate_noalloc(32, 0, ctypes.c_void_p(blocks.data_ptr()), 4,
                                    ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == -1 and b"4, 8 or 16" in raw.aqmp_last_error()
    # the largest accepted request still succeeds
    rc = raw.aqmp_correlate_noalloc(16, 0, ctypes.c_void_p(blocks.data_ptr()), 16384,
                                    ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert np.isfinite(out[:16384].cpu().numpy()).all()
