"""a2 on the GPU: the tcgen05 exact-limb correlation against the integer
SIMT kernel (bit for bit) and against the FP64 oracle's D^T y."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    aqmp.load_library()
    assert torch.cuda.is_available()
    return aqmp


def _blocks(L, b, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 256, size=(L, b, b), dtype=np.uint8)
    if L > 3:
        x[0] = 0
        x[1] = 255
        x[2] = np.where(np.arange(b)[None, :] < b // 2, 255, 0)
    return x


@pytest.mark.parametrize("b,dict_id,L", [(4, 0, 1), (4, 0, 200), (8, 0, 65), (8, 1, 64), (16, 0, 130),
                                         (16, 2, 7), (32, 0, 70), (64, 0, 66), (64, 1, 3), (128, 0, 5),
                                         (128, 2, 2)])
def test_tensor_core_matches_simt_and_fp64(lib, b, dict_id, L):
    host = _blocks(L, b, seed=b * 100 + L + dict_id)
    dev = torch.from_numpy(host).cuda()
    tc = lib.aqmp_correlate(b, dict_id, dev, gemm=0)
    simt = lib.aqmp_correlate(b, dict_id, dev, gemm=1)
    torch.cuda.synchronize()
    tc_h, simt_h = tc.cpu().numpy(), simt.cpu().numpy()
    # both kernels round the same exact integer once: identical bits
    assert np.array_equal(tc_h.view(np.uint32), simt_h.view(np.uint32))
    D = oracle.dictionary(b, dict_id)
    Dabs = np.abs(D)
    for l in range(L):
        y = oracle.unravel(host[l])
        ref = D @ y
        got = tc_h[l, :, 0].astype(np.float64) + tc_h[l, :, 1].astype(np.float64)
        # fixed-point dictionary: |err| <= 2^-49 sum|y| + rounding of the
        # result; plus the FP64 reference's own summation error, at most
        # n 2^-53 sum_v |phi_j[v] y[v]| (side 128: K = 16 384 in four chunks)
        bound = (2.0 ** -47 * np.sum(np.abs(y)) + 2.0 ** -46 * np.abs(ref) + 1e-12
                 + y.size * 2.0 ** -53 * (Dabs @ np.abs(y)))
        assert np.all(np.abs(got - ref) <= bound), (l, np.max(np.abs(got - ref) - bound))


@pytest.mark.parametrize("b,dict_id,L", [(8, 0, 65), (32, 0, 70), (64, 2, 5), (128, 0, 3)])
def test_bf16_form_is_within_its_rounding_bound(lib, b, dict_id, L):
    """The reduced-precision form: one BF16 pass of bf16(D) with FP32
    accumulation.  Against the FP64 D^T y: bf16 rounding of each entry
    (2^-9 relative), FP32 accumulation over n terms of the centred pixels,
    and the FP32 centring term."""
    host = _blocks(L, b, seed=b * 7 + L + dict_id)
    dev = torch.from_numpy(host).cuda()
    got = lib.aqmp_correlate(b, dict_id, dev, gemm=2).cpu().numpy()
    assert np.all(got[:, :, 1] == 0.0)
    D = oracle.dictionary(b, dict_id)
    Dabs = np.abs(D)
    worst = 0.0
    for l in range(L):
        y = oracle.unravel(host[l])
        ref = D @ y
        bound = (2.0 ** -8 * (Dabs @ np.abs(y)) + y.size * 2.0 ** -23 * (Dabs @ np.abs(y - 128.0))
                 + 2.0 ** -20 * (np.abs(ref) + 128.0 * Dabs.sum(axis=1)) + 1e-6)
        err = np.abs(got[l, :, 0].astype(np.float64) - ref)
        assert np.all(err <= bound), (l, float(np.max(err - bound)))
        worst = max(worst, float(np.max(err)))
    # an approximation, not the exact form (a constant block can come out exact)
    assert worst > 0.0
