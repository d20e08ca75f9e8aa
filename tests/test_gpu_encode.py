"""The encoder hot path on the GPU against the FP64 oracle: atom indices,
split decisions and quadtree shape identical; coefficients within 1e-5
relative; reconstructions and PSNR / SSIM within the stated bounds."""
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


def run_both(lib, planes, tols, simt=False, **kw):
    dev = [torch.from_numpy(p).cuda() for p in planes]
    code = lib.aqmp_encode_planes(dev, tols, simt_gemm=simt, **kw)
    leaves, atoms, lo = code.copy()
    okw = {k: v for k, v in kw.items() if k in ("cap_num", "cap_den", "min_block", "max_block", "dict_id")}
    enc = oracle.encode(planes, tols, **okw)
    return code, leaves, atoms, lo, enc


# the 64x64 gradient scene at tol 2 is the parity configuration; the other
# tolerances exercise splits down to 4x4 leaves
@pytest.mark.parametrize("tol", [2.0, 1.0, 1.5, 3.0])
def test_gradient_scene_64(lib, tol):
    img = synthetic.gradient_scene(64, 64, seed=0)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [tol])
    rep = parity.compare(enc, leaves, atoms, lo, [img])
    st = code.stats()
    assert st["atom_iterations"] == enc.steps and st["attempts"] == enc.attempts
    assert st["near_tie_leaves"] == 0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_several_roots_and_levels(lib, seed):
    img = synthetic.gradient_scene(128, 192, seed=seed)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [1.25], max_block=32, min_block=4)
    parity.compare(enc, leaves, atoms, lo, [img])


def test_batch_of_planes_with_own_tolerances(lib):
    imgs = [synthetic.gradient_scene(64, 128, seed=s) for s in (5, 6, 7)]
    tols = [0.8, 1.7, 4.0]
    code, leaves, atoms, lo, enc = run_both(lib, imgs, tols, max_block=32)
    parity.compare(enc, leaves, atoms, lo, imgs)


def test_simt_and_tensor_core_paths_agree(lib):
    img = synthetic.piecewise_scene(128, 128, seed=3)
    a = run_both(lib, [img], [1.0], max_block=64)
    b = run_both(lib, [img], [1.0], max_block=64, simt=True)
    for x, y in zip(a[1:4], b[1:4]):
        assert np.array_equal(x, y)
    parity.compare(a[4], a[1], a[2], a[3], [img])


@pytest.mark.parametrize("dict_id", [1, 2])
def test_single_family_dictionaries(lib, dict_id):
    img = synthetic.gradient_scene(64, 64, seed=11)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [1.2], max_block=16, dict_id=dict_id)
    parity.compare(enc, leaves, atoms, lo, [img])


def test_fixed_block_size_and_full_budget(lib):
    img = synthetic.gradient_scene(64, 64, seed=12)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [0.5], min_block=8, max_block=8, cap_num=1, cap_den=2)
    parity.compare(enc, leaves, atoms, lo, [img])


def test_degenerate_planes(lib):
    planes = [synthetic.uniform_plane(64, 64, v) for v in (0, 128, 255)]
    planes.append(synthetic.noise_plane(64, 64, seed=4, sigma=70.0))
    code, leaves, atoms, lo, enc = run_both(lib, planes, [2.0, 2.0, 2.0, 1.0], max_block=32)
    parity.compare(enc, leaves, atoms, lo, planes)
    # a uniform plane: one DC atom per root (none for the zero plane)
    for p, v in ((0, 0), (1, 128), (2, 255)):
        sel = leaves[leaves["plane"] == p]
        assert np.all(sel["b"] == 32) and np.all(sel["n_atoms"] == (0 if v == 0 else 1))


def test_huge_tolerance_and_empty_pursuits(lib):
    img = synthetic.gradient_scene(64, 64, seed=13)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [1e6])
    assert len(atoms) == 0 and len(leaves) == 1
    parity.compare(enc, leaves, atoms, lo, [img])


def test_host_and_device_inputs_agree(lib):
    img = synthetic.gradient_scene(64, 64, seed=14)
    c1 = lib.aqmp_encode_planes([torch.from_numpy(img).cuda()], [1.3])
    c2 = lib.aqmp_encode_planes([img], [1.3])
    for x, y in zip(c1.copy(), c2.copy()):
        assert np.array_equal(x, y)


def test_decode_matches_oracle_reconstruction(lib):
    img = synthetic.piecewise_scene(128, 128, seed=9)
    code, leaves, atoms, lo, enc = run_both(lib, [img], [1.5])
    out = torch.empty((128, 128), dtype=torch.float32, device="cuda")
    code.decode(0, out)
    rec = out.cpu().numpy().astype(np.float64)
    ref = oracle.decode(enc, 0, 128, 128)
    # FP32 synthesis of FP32 coefficients: within 1e-5 of the 0-255 range
    assert np.max(np.abs(rec - ref)) <= 1e-5 * 255
    assert abs(oracle.psnr(rec, img) - oracle.psnr(ref, img)) <= 1e-4
    assert abs(oracle.ssim(rec, img) - oracle.ssim(ref, img)) <= 1e-4
    host = np.zeros((128, 128), np.float32)
    code.decode(0, host)
    assert np.array_equal(host, out.cpu().numpy())


def test_converged_leaves_meet_the_tolerance_on_the_gpu_reconstruction(lib):
    img = synthetic.piecewise_scene(256, 256, seed=21)
    tol = 2.0
    code = lib.aqmp_encode_planes([torch.from_numpy(img).cuda()], [tol])
    leaves, atoms, lo = code.copy()
    out = torch.empty((256, 256), dtype=torch.float32, device="cuda")
    code.decode(0, out)
    rec = out.cpu().numpy().astype(np.float64)
    cover = np.zeros(img.shape, int)
    for L in leaves:
        b, y, x = int(L["b"]), int(L["y"]), int(L["x"])
        cover[y:y + b, x:x + b] += 1
        if L["converged"]:
            rmse = np.sqrt(np.mean((rec[y:y + b, x:x + b] - img[y:y + b, x:x + b]) ** 2))
            assert rmse < tol * (1 + 1e-5)
        else:
            assert b == 4 and L["n_atoms"] == 4
    assert np.all(cover == 1)


# the 512x512 piecewise scene at tol {1, 2, 4, 8}, encoded in one batched
# call exactly as the benchmark runs it; the oracle checks sampled roots
def test_piecewise_512_tolerance_sweep_sampled_roots(lib):
    img = synthetic.piecewise_scene(512, 512, seed=1)
    tols = [1.0, 2.0, 4.0, 8.0]
    planes = [img] * 4
    code = lib.aqmp_encode_planes([torch.from_numpy(img).cuda()] * 4, tols)
    leaves, atoms, lo = code.copy()
    st = code.stats()
    # every root holding a leaf whose decisions were not certified is checked
    # too (it must still agree exactly), on top of a fixed spread of roots
    base = [0, 9, 27, 36, 54, 63]
    flagged = leaves[leaves["flags"] != 0]
    samples = []
    for p in range(4):
        extra = {int(L["y"]) // 64 * 8 + int(L["x"]) // 64 for L in flagged if L["plane"] == p}
        samples.append(sorted(set(base) | extra))
    enc = oracle.encode(planes, tols, roots=samples)
    parts = [parity.restrict_to_roots(leaves, atoms, lo, p, samples[p], 64, 512) for p in range(4)]
    gl = np.concatenate([p[0] for p in parts])
    ga = np.concatenate([p[1] for p in parts])
    glo = np.concatenate([p[2] for p in parts])
    gl["atom_off"] = np.concatenate([[0], np.cumsum(gl["n_atoms"].astype(np.int64))[:-1]]).astype(np.uint32)
    parity.compare(enc, gl, ga, glo, planes, allow_flagged=True)
    assert st["near_tie_leaves"] == len(flagged) <= 2
    # whole-image invariants
    for p in range(4):
        sel = leaves[leaves["plane"] == p]
        assert int(np.sum(sel["b"].astype(np.int64) ** 2)) == 512 * 512


def test_uneven_rgb_batch_in_one_call(lib):
    """Leaves of many images and sizes go through one batched encode; every
    plane's sampled roots match the oracle."""
    batch = synthetic.uneven_rgb_batch(4, seed=5, wmin=128, wmax=320, hmin=128, hmax=256)
    planes = [p for (_, _, chans) in batch for p in chans]
    code = lib.aqmp_encode_planes([torch.from_numpy(p).cuda() for p in planes], 1.5)
    leaves, atoms, lo = code.copy()
    samples = []
    for i, p in enumerate(planes):               # one root per plane: first, middle or last
        nroots = (p.shape[0] // 64) * (p.shape[1] // 64)
        samples.append([(0, nroots // 2, nroots - 1)[i % 3]])
    enc = oracle.encode(planes, [1.5] * len(planes), roots=samples)
    parts = [parity.restrict_to_roots(leaves, atoms, lo, i, samples[i], 64, planes[i].shape[1])
             for i in range(len(planes))]
    gl = np.concatenate([q[0] for q in parts])
    ga = np.concatenate([q[1] for q in parts])
    glo = np.concatenate([q[2] for q in parts])
    gl["atom_off"] = np.concatenate([[0], np.cumsum(gl["n_atoms"].astype(np.int64))[:-1]]).astype(np.uint32)
    parity.compare(enc, gl, ga, glo, planes, allow_flagged=True)
    for i, p in enumerate(planes):
        sel = leaves[leaves["plane"] == i]
        assert int(np.sum(sel["b"].astype(np.int64) ** 2)) == p.size


def _dfs_keys(leaves, shapes, max_block, min_block):
    """(plane, root in raster order, Z-order cell inside the root) of every
    leaf: strictly increasing along the canonical depth-first order."""
    levels = int(np.log2(max_block // min_block))
    keys = []
    for L in leaves:
        p, y, x = int(L["plane"]), int(L["y"]), int(L["x"])
        root = (y // max_block) * (shapes[p][1] // max_block) + x // max_block
        cy, cx = (y % max_block) // min_block, (x % max_block) // min_block
        z = 0
        for bit in range(levels - 1, -1, -1):
            z = (z << 2) | (((cy >> bit) & 1) << 1) | ((cx >> bit) & 1)
        keys.append((p, root, z))
    return keys


@pytest.mark.parametrize("min_block,max_block", [(4, 64), (8, 32), (16, 16), (4, 8)])
def test_device_arrays_are_in_canonical_order(lib, min_block, max_block):
    """The encode writes its leaf and atom arrays in the canonical order on the
    device: the device views equal the host copy, leaf keys increase
    depth-first, atom offsets are the running sum of the step counts and the
    leaves tile every plane."""
    batch = synthetic.uneven_rgb_batch(3, seed=11, wmin=64, wmax=192, hmin=64, hmax=128)
    planes = [p for (_, _, chans) in batch for p in chans] + [synthetic.uniform_plane(64, 128, 77)]
    tols = [0.5 + 0.5 * (i % 4) for i in range(len(planes))]
    code = lib.aqmp_encode_planes([torch.from_numpy(p).cuda() for p in planes], tols,
                                  min_block=min_block, max_block=max_block)
    leaves, atoms, lo = code.copy()
    dl = lib.aqmp_device_leaves(code)
    dj, da = lib.aqmp_device_atoms(code)
    np.testing.assert_array_equal(dl.view(np.uint8), leaves.view(np.uint8))
    np.testing.assert_array_equal(dj.cpu().numpy(), atoms["j"].astype(np.int64))
    np.testing.assert_array_equal(da.cpu().numpy().view(np.uint32), atoms["alpha"].view(np.uint32))
    keys = _dfs_keys(leaves, [p.shape for p in planes], max_block, min_block)
    assert all(a < b for a, b in zip(keys, keys[1:]))
    offs = np.concatenate([[0], np.cumsum(leaves["n_atoms"].astype(np.int64))[:-1]])
    np.testing.assert_array_equal(leaves["atom_off"].astype(np.int64), offs)
    assert int(leaves["n_atoms"].astype(np.int64).sum()) == len(atoms)
    for i, p in enumerate(planes):
        sel = leaves[leaves["plane"] == i]
        assert int(np.sum(sel["b"].astype(np.int64) ** 2)) == p.size
    code.free()


def test_one_large_plane_sampled_roots(lib):
    """One 16384 x 8192 plane (134 M px, 32 768 roots): sampled roots at the
    corners and in the middle match the oracle, the leaves tile the plane and
    the leaf order is depth-first (the 64-bit index arithmetic at size)."""
    h, w = 16384, 8192
    img = synthetic.gradient_scene(h, w, seed=13)
    code = lib.aqmp_encode_planes([torch.from_numpy(img).cuda()], 3.0)
    leaves, atoms, lo = code.copy()
    code.free()
    assert int(np.sum(leaves["b"].astype(np.int64) ** 2)) == h * w
    keys = _dfs_keys(leaves, [img.shape], 64, 4)
    assert all(a < b for a, b in zip(keys, keys[1:]))
    nroots = (h // 64) * (w // 64)
    roots = sorted({0, w // 64 - 1, nroots // 2 + 17, nroots - w // 64, nroots - 1})
    enc = oracle.encode([img], [3.0], roots=[roots])
    gl, ga, glo = parity.restrict_to_roots(leaves, atoms, lo, 0, roots, 64, w)
    gl["atom_off"] = np.concatenate([[0], np.cumsum(gl["n_atoms"].astype(np.int64))[:-1]]).astype(np.uint32)
    parity.compare(enc, gl, ga, glo, [img])


def test_batch_entry_point_equals_the_plane_list(lib):
    """aqmp_encode_batch (images of several sizes and channel counts) gives the
    plane-list encode's result bit for bit."""
    imgs = [np.stack([synthetic.gradient_scene(128, 192, seed=30 + c) for c in range(3)]),
            synthetic.piecewise_scene(64, 128, seed=33)[None]]
    dev = [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]
    a = lib.aqmp_encode_batch(dev, rmse_tol=2.0)
    planes = [p for im in dev for p in im]
    b = lib.aqmp_encode_planes(planes, 2.0)
    for x, y in zip(a.copy(), b.copy()):
        np.testing.assert_array_equal(x.view(np.uint8), y.view(np.uint8))
    assert a.stats()["n_leaves"] == b.stats()["n_leaves"] > 0
