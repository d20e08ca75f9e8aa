"""aqmp_correlate_noalloc: the correlation for callers that may not allocate
device memory (memory owned by another allocator or a fixed budget, loops
that reserve everything at start-up).  It keeps its scratch in static device
arrays, so its result must equal the allocating entry point's bit for bit,
call after call, although every call reuses (and overwrites) the same
arrays.  This file is collected last on purpose."""
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
        ref = lib.aqmp_correlate(b, dict_id, blocks, gemm=0)
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), (b, dict_id, L)


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
