"""a2 on the GPU.  The exact correlation with the separable fixed-point
dictionary (each 1-D basis row rounded to 2^-48, atoms their outer
products): the tensor-core, integer SIMT and mixed (DCT-II family on the
tensor cores, Haar family on the SIMT pipes) kernels against each other (bit
for bit) and against the FP64 oracle's D^T y within the bound of that
fixed-point dictionary.  The dense exact kernels (round(D 2^48) entries)
likewise, and the reduced-precision BF16 form within its rounding bound."""
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


CASES = [(4, 0, 1), (4, 0, 200), (8, 0, 65), (8, 1, 64), (16, 0, 130), (16, 2, 7), (32, 0, 70), (64, 0, 66),
         (64, 0, 1), (64, 0, 153), (64, 1, 3), (64, 2, 5), (128, 0, 5), (128, 2, 2)]


def _families(b, dict_id):
    return {0: [oracle.dct_1d(b), oracle.haar_1d(b)], 1: [oracle.dct_1d(b)], 2: [oracle.haar_1d(b)]}[dict_id]


def _separable_bound(b, dict_id, y_block, ref):
    """|c - D^T y| for the separable fixed-point dictionary: each entry
    B[p][i] B[q][m] errs by at most 2^-49 (|B[p][i]| + |B[q][m]|) + 2^-97, the
    result is rounded once into a double-float (2^-47 |c| with margin), and
    the FP64 reference itself errs by at most n 2^-53 sum_v |phi_j[v] y[v]|."""
    Y = np.abs(y_block.astype(np.float64))              # Y[i][m]
    out = []
    for B in _families(b, dict_id):
        A = np.abs(B)
        a = (A @ Y).sum(axis=1)                          # a[p] = sum_{i,m} |B[p][i]| |y[i][m]|
        c = (Y @ A.T).sum(axis=0)                        # c[q] = sum_{i,m} |y[i][m]| |B[q][m]|
        out.append((a[None, :] + c[:, None]).reshape(-1))   # atom index q b + p
    e = 2.0 ** -49 * np.concatenate(out) + 2.0 ** -97 * Y.sum()
    return e + 2.0 ** -47 * np.abs(ref) + 1e-12


@pytest.mark.parametrize("b,dict_id,L", CASES)
def test_separable_kernels_agree_and_match_fp64(lib, b, dict_id, L):
    host = _blocks(L, b, seed=b * 100 + L + dict_id)
    dev = torch.from_numpy(host).cuda()
    best = lib.aqmp_correlate(b, dict_id, dev, gemm=0)
    simt = lib.aqmp_correlate(b, dict_id, dev, gemm=1)
    torch.cuda.synchronize()
    best_h, simt_h = best.cpu().numpy(), simt.cpu().numpy()
    # both kernels round the same exact integer once: identical bits
    assert np.array_equal(best_h.view(np.uint32), simt_h.view(np.uint32))
    if b == 64:
        # at side 64 the default runs the DCT-II family on the tensor cores and
        # the Haar family on the SIMT pipes; the tensor-core kernel's own Haar
        # path (mode 6) agrees too
        tc_h = lib.aqmp_correlate(b, dict_id, dev, gemm=6).cpu().numpy()
        assert np.array_equal(tc_h.view(np.uint32), simt_h.view(np.uint32))
    D = oracle.dictionary(b, dict_id)
    Dabs = np.abs(D)
    for l in range(L):
        y = oracle.unravel(host[l])
        ref = D @ y
        got = best_h[l, :, 0].astype(np.float64) + best_h[l, :, 1].astype(np.float64)
        bound = _separable_bound(b, dict_id, host[l], ref) + y.size * 2.0 ** -53 * (Dabs @ np.abs(y))
        assert np.all(np.abs(got - ref) <= bound), (l, np.max(np.abs(got - ref) - bound))


@pytest.mark.parametrize("b,dict_id,L", [(4, 0, 200), (8, 1, 64), (16, 0, 130), (64, 0, 9), (128, 2, 2)])
def test_dense_kernels_agree_and_match_fp64(lib, b, dict_id, L):
    """The dense exact form (entries round(D 2^48), 8 digit planes on the
    tensor cores; the allocation-free entry point's kernel) against its
    integer SIMT twin and the FP64 D^T y."""
    host = _blocks(L, b, seed=b * 31 + L + dict_id)
    dev = torch.from_numpy(host).cuda()
    tc = lib.aqmp_correlate(b, dict_id, dev, gemm=3)
    simt = lib.aqmp_correlate(b, dict_id, dev, gemm=4)
    torch.cuda.synchronize()
    tc_h, simt_h = tc.cpu().numpy(), simt.cpu().numpy()
    assert np.array_equal(tc_h.view(np.uint32), simt_h.view(np.uint32))
    D = oracle.dictionary(b, dict_id)
    Dabs = np.abs(D)
    for l in range(L):
        y = oracle.unravel(host[l])
        ref = D @ y
        got = tc_h[l, :, 0].astype(np.float64) + tc_h[l, :, 1].astype(np.float64)
        # fixed-point dictionary: |err| <= 2^-49 sum|y| + rounding of the
        # result; plus the FP64 reference's own summation error
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


@pytest.mark.parametrize("b,dict_id,L", [(4, 0, 200), (8, 1, 64), (16, 0, 130), (32, 2, 9), (64, 0, 66), (128, 0, 3)])
def test_fp8_form_is_within_its_rounding_bound(lib, b, dict_id, L):
    """The FP8 form: e4m3(D s_j) against e4m3(y~ s_l) with power-of-two scales
    per atom and per block, FP32 accumulation.  An E4M3 value carries 3
    fraction bits (rounding error at most 2^-4 relative for normal values,
    2^-10 absolute below 2^-6), so against the FP64 D^T y the error is at
    most 2^-4 sum|D||y~| (pixels) + (2^-4 + 2^-8) sum|D|(|y~| + 128) (atoms)
    + the subnormal floor + FP32 accumulation."""
    host = _blocks(L, b, seed=b * 13 + L + dict_id)
    dev = torch.from_numpy(host).cuda()
    got = lib.aqmp_correlate(b, dict_id, dev, gemm=5).cpu().numpy()
    assert np.all(got[:, :, 1] == 0.0)
    D = oracle.dictionary(b, dict_id)
    Dabs = np.abs(D)
    dmax = Dabs.max(axis=1)                                  # per atom
    worst = 0.0
    for l in range(L):
        y = oracle.unravel(host[l])
        yc = np.abs(y - 128.0)
        ref = D @ y
        bound = (2.0 ** -4 * (Dabs @ yc) + (2.0 ** -4 + 2.0 ** -8) * (Dabs @ (yc + 128.0))
                 + 2.0 ** -10 * (2.0 * dmax / 448.0) * np.sum(yc + 128.0)
                 + y.size * 2.0 ** -22 * (Dabs @ (yc + 128.0)) + 1e-4)
        err = np.abs(got[l, :, 0].astype(np.float64) - ref)
        assert np.all(err <= bound), (l, float(np.max(err - bound)))
        worst = max(worst, float(np.max(err)))
    assert worst > 0.0


def _scene_blocks(L, seed):
    from paper_2605_09190_gb300 import synthetic
    img = synthetic.gradient_scene(512, 512, seed=seed)
    pw = synthetic.piecewise_scene(512, 512, seed=seed)
    out = []
    for l in range(L):
        src = img if l % 2 == 0 else pw
        r, c = (l // 2) % 8, (l // 16) % 8
        out.append(src[64 * r:64 * r + 64, 64 * c:64 * c + 64])
    return np.ascontiguousarray(np.stack(out))


@pytest.mark.parametrize("dict_id,L,kind", [(0, 66, "random"), (0, 160, "scenes"), (1, 5, "random"),
                                             (2, 7, "scenes"), (0, 1, "random")])
def test_bf16x2_correlation_is_within_its_bound(lib, dict_id, L, kind):
    """The BF16 form's correlation (split BF16 products, FP32 accumulation)
    against the exact form's, atom by atom, within the bound the kernel
    returns; and that bound against its definition, 25 2^-19 times the
    atom's mass sum |B[p][i]| |y[i][m] - mu| |B[q][m]| (mu the block's
    integer mean) plus the centring term's 2^-40 and the 2^-30 by which the
    exact form's fixed-point rows may differ from the real correlation."""
    host = _blocks(L, 64, seed=L + dict_id) if kind == "random" else _scene_blocks(L, seed=dict_id)
    dev = torch.from_numpy(host).cuda()
    c, e = lib.aqmp_correlate_bf16x2(64, dict_id, dev)
    ex = lib.aqmp_correlate(64, dict_id, dev, gemm=0)
    torch.cuda.synchronize()
    c, e, ex = c.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64), ex.cpu().numpy().astype(np.float64)
    got, ref = c[:, :, 0] + c[:, :, 1], ex[:, :, 0] + ex[:, :, 1]
    err = np.abs(got - ref)
    assert np.all(err <= e), float(np.max(err - e))
    fams = _families(64, dict_id)
    worst = 0.0
    for l in range(L):
        y = host[l].astype(np.float64)                     # y[i][m]: row i, column m
        mu = np.floor(y.mean() + 0.5)
        Yt = np.abs(y - mu)
        mass = np.concatenate([(np.abs(B) @ Yt @ np.abs(B).T).T.reshape(-1) for B in fams])   # index q b + p
        R = np.concatenate([np.outer(B.sum(axis=1), B.sum(axis=1)).T.reshape(-1) for B in fams])
        lo = 25 * 2.0 ** -19 * mass
        hi = 25 * 2.0 ** -19 * mass * (1 + 2.0 ** -5) + 2.0 ** -39 * mu * np.abs(R) + 2.0 ** -29   # three BF16 round-ups
        assert np.all(e[l] >= lo * (1 - 2.0 ** -12)) and np.all(e[l] <= hi)
        worst = max(worst, float(np.max(err[l] / np.maximum(e[l], 1e-300))))
    print(f"largest error / bound: {worst:.3f}")
