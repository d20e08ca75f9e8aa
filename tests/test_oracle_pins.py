"""Pins for the FP64 oracle: each check ties the oracle to something other
than itself -- a library transform, a closed form, an invariant of the
mathematics, or brute force on tiny inputs -- so that a dropped term, a wrong
sign or index, or a transposed operand anywhere in it fails one of them."""
import numpy as np
import pytest
import scipy.fft
import scipy.ndimage

import oracle
from paper_2605_09190_gb300 import synthetic

SIDES = [4, 8, 16, 32]


def fast_haar_1d(x: np.ndarray) -> np.ndarray:
    """Pyramid (filter-bank) Haar analysis of a length-2^J vector, written
    independently of the oracle's support-interval construction: repeated
    pairwise sums and differences scaled by 1/sqrt(2); output = [scaling,
    coarsest detail, ..., finest details]."""
    a = np.asarray(x, np.float64)
    details = []
    while a.shape[0] > 1:
        s = (a[0::2] + a[1::2]) / np.sqrt(2.0)
        d = (a[0::2] - a[1::2]) / np.sqrt(2.0)
        details.insert(0, d)
        a = s
    return np.concatenate([a] + details)


def fast_haar_2d(Y: np.ndarray) -> np.ndarray:
    Z = np.apply_along_axis(fast_haar_1d, 0, Y)
    return np.apply_along_axis(fast_haar_1d, 1, Z)


# --------------------------------------------------------------- tables

@pytest.mark.parametrize("b", SIDES + [64, 128])
def test_dct_rows_match_scipy(b):
    ref = scipy.fft.dct(np.eye(b), type=2, norm="ortho", axis=0)
    # the argument pi/N (m + 1/2) k reaches ~1e4 at b = 64, so cos carries ~1e-13 of
    # argument rounding; a wrong term or index would be off by O(0.1)
    np.testing.assert_allclose(oracle.dct_1d(b), ref, atol=2e-13, rtol=0)


@pytest.mark.parametrize("b", SIDES + [64, 128])
def test_haar_rows_match_filter_bank(b):
    ref = np.stack([fast_haar_1d(e) for e in np.eye(b)], axis=1)   # column m = transform of e_m
    np.testing.assert_allclose(oracle.haar_1d(b), ref, atol=2e-15, rtol=0)


@pytest.mark.parametrize("b", SIDES + [64, 128])
def test_dct_rows_are_even_or_odd_about_the_centre(b):
    # cos(pi k (2 (b - 1 - m) + 1) / 2b) = (-1)^k cos(pi k (2m + 1) / 2b): the
    # symmetry the exact separable kernels use to halve the DCT-II contractions
    C = scipy.fft.dct(np.eye(b), type=2, norm="ortho", axis=0)
    sign = (-1.0) ** np.arange(b)[:, None]
    np.testing.assert_allclose(C[:, ::-1], sign * C, atol=2e-13, rtol=0)
    np.testing.assert_allclose(oracle.dct_1d(b)[:, ::-1], sign * oracle.dct_1d(b), atol=2e-13, rtol=0)


@pytest.mark.parametrize("b", SIDES + [64, 128])
def test_haar_rows_are_two_constant_halves_of_one_magnitude_per_scale(b):
    # each Haar row is v > 0 on the first half of a dyadic interval and -v on
    # the second (row 0: v on the whole block), with v fixed by the interval's
    # length: the structure behind the summed-area form of the Haar correlations
    H = np.stack([fast_haar_1d(e) for e in np.eye(b)], axis=1)
    by_len = {}
    for r in range(b):
        nz = np.nonzero(np.abs(H[r]) > 1e-12)[0]
        s, e = int(nz[0]), int(nz[-1]) + 1
        L = e - s
        assert len(nz) == L and L & (L - 1) == 0 and s % L == 0
        v = H[r, s]
        assert v > 0
        want = np.full(L, v) if r == 0 else np.concatenate([np.full(L // 2, v), np.full(L // 2, -v)])
        np.testing.assert_allclose(H[r, s:e], want, atol=1e-15, rtol=0)
        key = (L, r == 0)
        by_len.setdefault(key, v)
        assert abs(by_len[key] - v) < 1e-15
        np.testing.assert_allclose(oracle.haar_1d(b)[r], H[r], atol=2e-15, rtol=0)


@pytest.mark.parametrize("b", SIDES)
def test_dictionary_families_orthonormal(b):
    n = b * b
    D = oracle.dictionary(b, 0)
    assert D.shape == (2 * n, n)
    G = D @ D.T
    np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-14)
    np.testing.assert_allclose(G[:n, :n], np.eye(n), atol=1e-14)
    np.testing.assert_allclose(G[n:, n:], np.eye(n), atol=1e-14)
    # the DCT DC atom and the Haar scaling atom are the same vector, bit for bit
    assert np.array_equal(D[0], D[n])
    # no other pair of atoms coincides
    off = np.abs(G - np.eye(2 * n))
    off[0, n] = off[n, 0] = 0.0
    assert off.max() < 1.0 - 1e-6


@pytest.mark.parametrize("b", SIDES)
def test_dct_family_correlations_are_dctn(b):
    """Column-major unravel + atom index q*b+p: D_dct^T y = dctn(Y)[p, q]."""
    rng = np.random.default_rng(b)
    Y = rng.integers(0, 256, size=(b, b)).astype(np.float64)
    c = oracle.dictionary(b, 1) @ oracle.unravel(Y)
    ref = scipy.fft.dctn(Y, type=2, norm="ortho")
    np.testing.assert_allclose(c.reshape(b, b).T, ref, atol=1e-10)


@pytest.mark.parametrize("b", SIDES)
def test_haar_family_correlations_are_separable_fast_haar(b):
    rng = np.random.default_rng(100 + b)
    Y = rng.integers(0, 256, size=(b, b)).astype(np.float64)
    c = oracle.dictionary(b, 2) @ oracle.unravel(Y)
    ref = fast_haar_2d(Y)
    np.testing.assert_allclose(c.reshape(b, b).T, ref, atol=1e-10)
    # the union dictionary is the two families stacked, DCT first
    c0 = oracle.dictionary(b, 0) @ oracle.unravel(Y)
    np.testing.assert_array_equal(c0[b * b:], c)


def test_unravel_is_column_concatenation():
    A = np.arange(12, dtype=np.float64).reshape(3, 4)
    assert list(oracle.unravel(A)) == [0, 4, 8, 1, 5, 9, 2, 6, 10, 3, 7, 11]


# -------------------------------------------------------------- pursuit

def _sorted_coeffs(coef_matrix):
    """Coefficients in |.|-descending order, ties to the lowest atom index
    (atom index q*b + p for coefficient [p, q])."""
    flat = coef_matrix.T.reshape(-1)
    order = sorted(range(flat.size), key=lambda j: (-abs(flat[j]), j))
    return np.array(order), flat[order]


@pytest.mark.parametrize("b", [4, 8, 16])
def test_mp_on_dct_basis_is_sorted_dctn(b):
    """An orthonormal dictionary: MP picks the transform coefficients in
    magnitude order and reconstructs exactly in b^2 steps."""
    rng = np.random.default_rng(7 + b)
    Y = rng.normal(100.0, 30.0, size=(b, b))
    n = b * b
    res = oracle.mp(oracle.dictionary(b, 1), oracle.unravel(Y), 0.0, n)
    j_ref, a_ref = _sorted_coeffs(scipy.fft.dctn(Y, norm="ortho"))
    assert res["steps"] == n
    np.testing.assert_array_equal(res["j"], j_ref)
    np.testing.assert_allclose(res["alpha"], a_ref, rtol=1e-12, atol=1e-10)
    assert res["energy"][-1] < 1e-18 * res["energy"][0]


@pytest.mark.parametrize("b", [4, 8, 16])
def test_mp_on_haar_basis_is_sorted_fast_haar(b):
    rng = np.random.default_rng(17 + b)
    Y = rng.normal(100.0, 30.0, size=(b, b))
    n = b * b
    res = oracle.mp(oracle.dictionary(b, 2), oracle.unravel(Y), 0.0, n)
    j_ref, a_ref = _sorted_coeffs(fast_haar_2d(Y))
    np.testing.assert_array_equal(res["j"], j_ref)
    np.testing.assert_allclose(res["alpha"], a_ref, rtol=1e-12, atol=1e-10)
    assert res["energy"][-1] < 1e-18 * res["energy"][0]


def test_side128_correlations_and_first_steps():
    """Side 128, the largest root: D^T y is dctn and the separable fast Haar
    of the block (the atom index and unravel conventions at that size), and
    the first MP steps take the largest |correlation| and drop the energy by
    alpha^2 each."""
    b, n = 128, 128 * 128
    rng = np.random.default_rng(128)
    Y = rng.integers(0, 256, size=(b, b)).astype(np.float64)
    D = oracle.dictionary(b, 0)
    y = oracle.unravel(Y)
    c = D @ y
    np.testing.assert_allclose(c[:n].reshape(b, b).T, scipy.fft.dctn(Y, type=2, norm="ortho"), atol=1e-9)
    np.testing.assert_allclose(c[n:].reshape(b, b).T, fast_haar_2d(Y), atol=1e-9)
    res = oracle.mp(D, y, 0.0, 3)
    assert res["j"][0] == int(np.argmax(np.abs(c))) == 0     # DC, before the identical Haar scaling atom
    E = res["energy"]
    np.testing.assert_allclose(E[:-1] - E[1:], res["alpha"] ** 2, rtol=0, atol=1e-12 * E[0])
    r1 = y - res["alpha"][0] * D[0]
    c1 = D @ r1
    c1[[0, n]] = 0.0                                          # the chosen atom and its twin
    assert res["j"][1] == int(np.argmax(np.abs(c1)))


@pytest.mark.parametrize("b,seed", [(8, 1), (16, 2), (32, 3)])
def test_mp_energy_drops_by_alpha_squared(b, seed):
    """Unit-norm atoms: ||r_{t+1}||^2 = ||r_t||^2 - alpha_t^2 (Pythagoras),
    with the energy recomputed from the residual at every step."""
    rng = np.random.default_rng(seed)
    Y = rng.integers(0, 256, size=(b, b)).astype(np.float64)
    res = oracle.mp(oracle.dictionary(b, 0), oracle.unravel(Y), 0.0, b * b // 4)
    E = res["energy"]
    np.testing.assert_allclose(E[:-1] - E[1:], res["alpha"] ** 2, rtol=0, atol=1e-12 * E[0])
    assert np.all(np.diff(E) <= 0)


@pytest.mark.parametrize("seed", range(6))
def test_mp_steps_are_brute_force_best_fits_4x4(seed):
    """Each step's atom and coefficient equal the best one-atom least-squares
    fit of the current residual (numpy lstsq over all 32 atoms), with the
    residual rebuilt independently as y - sum alpha_s phi_s."""
    b = 4
    rng = np.random.default_rng(seed)
    Y = rng.integers(0, 256, size=(b, b)).astype(np.float64)
    if seed == 5:
        Y[:, :2] = 255.0                       # a saturated half-block
    D = oracle.dictionary(b, 0)
    y = oracle.unravel(Y)
    res = oracle.mp(D, y, 0.0, 12)
    r = y.copy()
    for t in range(res["steps"]):
        errs, coefs = [], []
        for j in range(D.shape[0]):
            coef, *_ = np.linalg.lstsq(D[j][:, None], r, rcond=None)
            coefs.append(coef[0])
            errs.append(np.sum((r - coef[0] * D[j]) ** 2))
        errs = np.array(errs)
        best = int(np.argmin(errs))
        # ties between numerically equal fits go to the lower index
        near = np.nonzero(errs <= errs[best] + 1e-9 * max(1.0, errs[best]))[0]
        assert res["j"][t] == near.min()
        assert abs(res["alpha"][t] - coefs[near.min()]) <= 1e-9 * max(1.0, abs(coefs[near.min()]))
        r = r - res["alpha"][t] * D[res["j"][t]]


def test_mp_stop_rule_is_strict_and_checked_before_each_step():
    b = 4
    D = oracle.dictionary(b, 0)
    y = oracle.unravel(synthetic.noise_plane(b, b, seed=3))
    full = oracle.mp(D, y, 0.0, 4)
    E = full["energy"]
    band = 2.0 ** -32 * E[0]            # energies this close to eps^2 count as equal to it
    # a threshold exactly equal to E_2 does not stop at step 2 (strict '<')
    r = oracle.mp(D, y, E[2], 4)
    assert r["steps"] == 3 and r["converged"]
    # nor does one inside the equality band
    r = oracle.mp(D, y, E[2] + 0.5 * band, 4)
    assert r["steps"] == 3 and r["converged"]
    # a threshold clearly above E_2 stops after two steps
    r = oracle.mp(D, y, E[2] + 2.0 * band, 4)
    assert r["steps"] == 2 and r["converged"]
    # the test after the last budgeted step still counts: meeting the
    # tolerance exactly at step k is convergence, not a split
    r = oracle.mp(D, y, E[2] + 2.0 * band, 2)
    assert r["steps"] == 2 and r["converged"]
    # a threshold above E_0 takes no step at all
    r = oracle.mp(D, y, E[0] + 2.0 * band, 4)
    assert r["steps"] == 0 and r["converged"]
    # the budget ends an unconverged pursuit after exactly k steps
    r = oracle.mp(D, y, 0.0, 3)
    assert r["steps"] == 3 and not r["converged"]


@pytest.mark.parametrize("b", [4, 8])
def test_exact_ties_go_to_the_lowest_index(b):
    """Symmetric blocks (Y = Y^T) have dctn(Y)[p, q] = dctn(Y)[q, p] exactly:
    atoms q b + p and p b + q tie, and the lower index must be taken first
    however the two correlations happen to round."""
    rng = np.random.default_rng(40 + b)
    lower_first = 0
    for trial in range(40):
        A = rng.integers(0, 128, size=(b, b)).astype(np.float64)
        Y = A + A.T
        res = oracle.mp(oracle.dictionary(b, 1), oracle.unravel(Y), 0.0, b * b)
        coef = scipy.fft.dctn(Y, norm="ortho")
        seen = set()
        for j in res["j"]:
            p, q = int(j) % b, int(j) // b
            if p != q and abs(abs(coef[p, q]) - abs(coef[q, p])) <= 1e-9 * np.abs(coef).max():
                partner = p * b + q
                # the partner (same magnitude) must not have been taken first
                # if its index is lower
                if partner < j:
                    assert partner in seen, (trial, int(j), partner)
                lower_first += 1
            seen.add(int(j))
    assert lower_first > 100


# ------------------------------------------------------------ quadtree

def _leaf_recon_rmse(enc, i, img, dict_id=0):
    L = enc.leaves[i]
    b = int(L["b"])
    j, a = enc.leaf_atoms(i)
    D = oracle.dictionary(b, dict_id)
    v = a @ D[j] if len(j) else np.zeros(b * b)
    blk = img[L["y"]:L["y"] + b, L["x"]:L["x"] + b].astype(np.float64)
    return np.sqrt(np.mean((v.reshape(b, b).T - blk) ** 2))


def test_constant_image_gives_one_dc_atom_per_root():
    img = synthetic.uniform_plane(64, 128, 200)
    enc = oracle.encode([img], 2.0, min_block=4, max_block=32)
    assert len(enc.leaves) == 8
    assert np.all(enc.leaves["n_atoms"] == 1) and np.all(enc.leaves["converged"] == 1)
    assert np.all(enc.atom_j == 0)
    np.testing.assert_allclose(enc.atom_alpha, 200.0 * 32, rtol=1e-14)


def test_zero_image_takes_no_step():
    enc = oracle.encode([synthetic.uniform_plane(32, 32, 0)], 0.5, max_block=16)
    assert len(enc.leaves) == 4 and enc.steps == 0
    assert np.all(enc.leaves["converged"] == 1)


def test_huge_tolerance_keeps_roots_without_atoms():
    img = synthetic.gradient_scene(64, 64, seed=4)
    enc = oracle.encode([img], 1e6, max_block=16)
    assert len(enc.leaves) == 16 and len(enc.atom_j) == 0
    assert np.all(enc.leaves["b"] == 16) and np.all(enc.leaves["converged"] == 1)


def test_strong_noise_descends_to_min_blocks_with_full_budget():
    img = synthetic.noise_plane(32, 32, seed=5, sigma=60.0)
    enc = oracle.encode([img], 1.0, min_block=4, max_block=16)
    assert np.all(enc.leaves["b"] == 4) and len(enc.leaves) == 64
    assert np.all(enc.leaves["n_atoms"] == 4) and np.all(enc.leaves["converged"] == 0)


@pytest.mark.parametrize("seed,tol", [(0, 1.0), (1, 1.5), (2, 2.0)])
def test_quadtree_tiles_and_respects_tolerance(seed, tol):
    img = synthetic.gradient_scene(64, 64, seed=seed)
    enc = oracle.encode([img], tol, min_block=4, max_block=32)
    cover = np.zeros(img.shape, int)
    for L in enc.leaves:
        cover[L["y"]:L["y"] + L["b"], L["x"]:L["x"] + L["b"]] += 1
    assert np.all(cover == 1)
    for i, L in enumerate(enc.leaves):
        k = oracle.sparsity_cap(int(L["b"]))
        assert L["n_atoms"] <= k
        if L["converged"]:
            assert _leaf_recon_rmse(enc, i, img) < np.float32(tol)
        else:
            assert L["b"] == 4 and L["n_atoms"] == k
    # every parent of a leaf failed: rerun MP on each parent block
    parents = {(int(L["y"]) // (2 * L["b"]) * (2 * L["b"]), int(L["x"]) // (2 * L["b"]) * (2 * L["b"]),
                2 * int(L["b"])) for L in enc.leaves if L["b"] < 32}
    for (py, px, pb) in parents:
        blk = img[py:py + pb, px:px + pb]
        r = oracle.mp(oracle.dictionary(pb, 0), oracle.unravel(blk),
                      oracle.eps2_of(tol, pb), oracle.sparsity_cap(pb))
        assert not r["converged"]


def test_depth_first_leaf_order():
    img = synthetic.noise_plane(16, 32, seed=9, sigma=60.0)
    enc = oracle.encode([img], 1.0, min_block=4, max_block=16)
    # root 0 then root 1; inside a root TL, TR, BL, BR recursively (Z order)
    def z(y, x):
        key = 0
        for bit in range(2, -1, -1):
            key = key * 4 + (((y >> bit) & 1) << 1 | ((x >> bit) & 1))
        return key
    keys = [(int(L["x"]) // 16, z(int(L["y"]) % 16 // 4, int(L["x"]) % 16 // 4)) for L in enc.leaves]
    assert keys == sorted(keys)


def test_decoder_reconstructs_exactly_with_full_orthonormal_budget():
    img = synthetic.gradient_scene(32, 32, seed=6)
    enc = oracle.encode([img], 0.0, cap_num=1, cap_den=1, min_block=8, max_block=8, dict_id=1)
    rec = oracle.decode(enc, 0, 32, 32, dict_id=1)
    np.testing.assert_allclose(rec, img, atol=1e-9)


def test_decoder_places_each_leaf_as_d_times_x():
    img = synthetic.gradient_scene(64, 64, seed=2)
    enc = oracle.encode([img], 1.5, max_block=32)
    rec = oracle.decode(enc, 0, 64, 64)
    for i, L in enumerate(enc.leaves):
        b = int(L["b"])
        j, a = enc.leaf_atoms(i)
        v = a @ oracle.dictionary(b, 0)[j] if len(j) else np.zeros(b * b)
        np.testing.assert_allclose(rec[L["y"]:L["y"] + b, L["x"]:L["x"] + b], v.reshape(b, b).T,
                                   atol=1e-9)


# ------------------------------------------------------------- metrics

def test_psnr_closed_form():
    ref = synthetic.gradient_scene(32, 32, seed=1).astype(np.float64)
    assert oracle.psnr(ref + 1.0, ref) == pytest.approx(20 * np.log10(255.0), abs=1e-9) or \
        np.any(ref == 255)
    x = np.full((8, 8), 100.0)
    assert oracle.psnr(x + 2.0, x) == pytest.approx(10 * np.log10(255.0 ** 2 / 4.0), abs=1e-12)


def test_ssim_identity_and_uniform_closed_form():
    img = synthetic.gradient_scene(48, 48, seed=3)
    assert oracle.ssim(img, img) == pytest.approx(1.0, abs=1e-12)
    a, c = 100.0, 130.0
    x = np.full((20, 20), a)
    y = np.full((20, 20), c)
    C1 = (0.01 * 255) ** 2
    assert oracle.ssim(y, x) == pytest.approx((2 * a * c + C1) / (a * a + c * c + C1), rel=1e-12)


def test_ssim_matches_scipy_gaussian_filtering():
    """Same statistic computed through scipy's separable Gaussian filter
    (radius 5 = an 11x11 window), cropped to the valid region."""
    x = synthetic.gradient_scene(64, 64, seed=8).astype(np.float64)
    y = np.clip(x + np.random.default_rng(0).normal(0, 6, x.shape), 0, 255)
    f = lambda im: scipy.ndimage.gaussian_filter(im, 1.5, truncate=5 / 1.5, mode="constant")[5:-5, 5:-5]
    mx, my = f(x), f(y)
    vx, vy, cxy = f(x * x) - mx ** 2, f(y * y) - my ** 2, f(x * y) - mx * my
    C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    ref = np.mean(((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx ** 2 + my ** 2 + C1) * (vx + vy + C2)))
    assert oracle.ssim(y, x) == pytest.approx(ref, abs=1e-10)
