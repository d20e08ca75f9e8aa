"""Side-128 roots on the GPU (the 4096 x 4096 workload's quadtree runs from
128 x 128 blocks down to 4 x 4): the cluster pursuit and the K-chunked
tensor-core correlation against the FP64 oracle, the decoder at side 128,
and, at the full 4096 x 4096 RGB size, the subtrees of split side-128 roots
against the same quadrants encoded as side-64 roots -- a split block's
children restart from the original pixels (Algorithm 2), so the two encodes
must agree bit for bit there."""
import numpy as np
import pytest

import oracle
import parity
from paper_2605_09190_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    aqmp.load_library()
    assert torch.cuda.is_available()
    return aqmp


def smooth_scene(h, w):
    """A ramp plus two low-frequency waves: side-128 blocks converge in a
    handful of atoms at tolerance 2."""
    yy, xx = np.mgrid[0:h, 0:w]
    img = 60 + 0.35 * xx + 25 * np.cos(2 * np.pi * yy / 256.0) + 10 * np.sin(2 * np.pi * xx / 128.0)
    return np.clip(img, 0, 255).round().astype(np.uint8)


def run_both(lib, planes, tols, roots=None, **kw):
    code = lib.aqmp_encode_planes([torch.from_numpy(p).cuda() for p in planes], tols, **kw)
    leaves, atoms, lo = code.copy()
    okw = {k: v for k, v in kw.items() if k in ("cap_num", "cap_den", "min_block", "max_block", "dict_id")}
    enc = oracle.encode(planes, tols, roots=roots, threads=4, **okw)
    return code, leaves, atoms, lo, enc


def test_side128_roots_converge(lib):
    img = smooth_scene(256, 384)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [2.0], max_block=128, min_block=16)
    parity.compare(enc, leaves, atoms, lo, [img])
    assert np.all(leaves["b"] == 128) and np.all(leaves["converged"] == 1)
    st = code.stats()
    assert st["attempts_per_level"][0] == 6 and st["near_tie_leaves"] == 0
    # step 0 of every root is the DCT DC atom, tied with the identical Haar
    # scaling atom held by another CTA of the cluster: decided in full precision
    assert st["window_steps_per_level"][0] >= 6
    assert np.all(atoms["j"][leaves["atom_off"]] == 0)
    # the decoder at side 128 against the oracle's
    out = torch.empty(img.shape, dtype=torch.float32, device="cuda")
    code.decode(0, out)
    rec = out.cpu().numpy().astype(np.float64)
    ref = oracle.decode(enc, 0, *img.shape)
    assert np.max(np.abs(rec - ref)) <= 1e-5 * 255
    assert abs(oracle.psnr(rec, img) - oracle.psnr(ref, img)) <= 1e-4
    assert abs(oracle.ssim(rec, img) - oracle.ssim(ref, img)) <= 1e-4


@pytest.mark.parametrize("dict_id", [0, 1, 2])
def test_side128_splits_with_a_small_budget(lib, dict_id):
    # k(b) = max(1, b^2 / 1024): 16 atoms at side 128, 4 at 64, then 1 --
    # the side-128 pursuits run out of budget and split
    img = synthetic.piecewise_scene(256, 256, seed=11)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [2.0], max_block=128, min_block=8, cap_num=1,
                                            cap_den=1024, dict_id=dict_id)
    parity.compare(enc, leaves, atoms, lo, [img])
    st = code.stats()
    assert st["atom_iterations"] == enc.steps and st["attempts"] == enc.attempts
    assert st["attempts_per_level"][0] == 4 and np.any(leaves["b"] < 128)


def test_side128_long_pursuit_one_root(lib):
    # a budget of 96 atoms on a textured root: a long pursuit across the
    # four CTAs, then its children
    img = synthetic.piecewise_scene(256, 256, seed=4)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [3.0], roots=[[3]], max_block=128, min_block=16,
                                            cap_num=3, cap_den=512)
    gl, ga, glo = parity.restrict_to_roots(leaves, atoms, lo, 0, [3], 128, 256)
    gl["atom_off"] = np.concatenate([[0], np.cumsum(gl["n_atoms"].astype(np.int64))[:-1]]).astype(np.uint32)
    parity.compare(enc, gl, ga, glo, [img])


def test_side128_fp32_form_runs_and_tiles(lib):
    img = synthetic.piecewise_scene(256, 256, seed=2)
    code = lib.aqmp_encode_planes([torch.from_numpy(img).cuda()], 2.0, max_block=128, precision=lib.AQMP_PREC_FP32)
    leaves, atoms, lo = code.copy()
    assert int(np.sum(leaves["b"].astype(np.int64) ** 2)) == img.size
    exact = lib.aqmp_encode_planes([torch.from_numpy(img).cuda()], 2.0, max_block=128)
    el, ea, _ = exact.copy()
    # the uncertified FP32 form mostly reproduces the exact tree
    same = len(set(map(tuple, leaves[["y", "x", "b"]].tolist())) & set(map(tuple, el[["y", "x", "b"]].tolist())))
    assert same >= 0.9 * len(el)


def _by_position(leaves, atoms, lo):
    """Leaves sorted by (plane, y, x) with their atom runs in that order."""
    order = np.lexsort((leaves["x"], leaves["y"], leaves["plane"]))
    L = leaves[order]
    n = L["n_atoms"].astype(np.int64)
    starts = L["atom_off"].astype(np.int64)
    idx = np.repeat(starts - np.concatenate([[0], np.cumsum(n)[:-1]]), n) + np.arange(int(n.sum()))
    return L, atoms[idx], lo[idx]


def test_4096_rgb_split_roots_match_side64_roots(lib):
    """4096 x 4096 RGB at tolerance 2: every side-128 root that split has the
    same four subtrees, bit for bit, as the side-64 encode of its quadrants;
    converged side-128 leaves of few atoms match the oracle."""
    planes = [synthetic.piecewise_scene(4096, 4096, seed=7 + c) for c in range(3)]
    dev = [torch.from_numpy(p).cuda() for p in planes]
    c128 = lib.aqmp_encode_planes(dev, 2.0, max_block=128)
    l128, a128, lo128 = c128.copy()
    s128 = c128.stats()
    c128.free()
    c64 = lib.aqmp_encode_planes(dev, 2.0, max_block=64)
    l64, a64, lo64 = c64.copy()
    c64.free()
    for p in range(3):
        assert int(np.sum(l128[l128["plane"] == p]["b"].astype(np.int64) ** 2)) == 4096 * 4096
    assert s128["attempts_per_level"][0] == 3 * 32 * 32

    big = l128[l128["b"] == 128]
    root_id = lambda L: (L["plane"].astype(np.int64) * 1024 + (L["y"].astype(np.int64) // 128) * 32  # noqa: E731
                         + L["x"].astype(np.int64) // 128)
    keep64 = ~np.isin(root_id(l64), root_id(big))
    small = l128["b"] < 128
    A, Aa, Alo = _by_position(l128[small], a128, lo128)
    B, Ba, Blo = _by_position(l64[keep64], a64, lo64)
    assert len(A) == len(B)
    for f in ("plane", "y", "x", "b", "n_atoms", "converged"):
        np.testing.assert_array_equal(A[f], B[f], err_msg=f)
    # a leaf's own near-tie flag (bit 0) is the same; bit 1 marks a flagged ancestor
    np.testing.assert_array_equal(A["flags"] & 1, B["flags"] & 1)
    np.testing.assert_array_equal(Aa["j"], Ba["j"])
    np.testing.assert_array_equal(Aa["alpha"].view(np.uint32), Ba["alpha"].view(np.uint32))
    np.testing.assert_array_equal(Alo.view(np.uint32), Blo.view(np.uint32))

    # converged side-128 leaves with a short pursuit: the oracle on their roots
    short = big[(big["converged"] == 1) & (big["n_atoms"] <= 48)]
    picks = short[np.linspace(0, len(short) - 1, min(2, len(short))).astype(int)] if len(short) else short
    for L in picks:
        p, r = int(L["plane"]), int(L["y"]) // 128 * 32 + int(L["x"]) // 128
        enc = oracle.encode([planes[p]], [2.0], max_block=128, roots=[[r]])
        gl, ga, glo = parity.restrict_to_roots(l128, a128, lo128, p, [r], 128, 4096)
        gl["atom_off"] = 0
        gl["plane"] = 0
        parity.compare(enc, gl, ga, glo, [planes[p]])
