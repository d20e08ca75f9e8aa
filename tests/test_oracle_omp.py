"""Pins of the oracle's Orthogonal Matching Pursuit (the solver the paper's
authors ran, Section 2.2): scikit-learn's OrthogonalMatchingPursuit, the
reduction to MP on an orthonormal dictionary, and the least-squares
optimality of every re-fit."""
import numpy as np
import pytest

import oracle
from paper_2605_09190_gb300 import synthetic


def _blocks():
    yield oracle.unravel(synthetic.gradient_scene(8, 8, seed=1)).astype(float)
    yield oracle.unravel(synthetic.noise_plane(8, 8, seed=2)).astype(float)
    yield oracle.unravel(synthetic.piecewise_scene(16, 16, seed=3)).astype(float)


@pytest.mark.parametrize("steps", [1, 4, 12])
def test_matches_scikit_learn(steps):
    sk = pytest.importorskip("sklearn.linear_model")
    for y in _blocks():
        b = int(np.sqrt(y.size))
        D = oracle.dictionary(b, 0)
        r = oracle.mp(D, y, 0.0, steps, "omp")
        assert r["steps"] == steps
        ref = sk.OrthogonalMatchingPursuit(n_nonzero_coefs=steps, fit_intercept=False).fit(D.T, y)
        support = np.flatnonzero(ref.coef_)
        assert sorted(r["j"].tolist()) == support.tolist()
        np.testing.assert_allclose(r["alpha"], ref.coef_[r["j"]], rtol=1e-9, atol=1e-9 * np.linalg.norm(y))


def test_reduces_to_mp_on_an_orthonormal_dictionary():
    for y in _blocks():
        b = int(np.sqrt(y.size))
        D = oracle.dictionary(b, 1)                     # DCT only
        k = y.size // 4
        o = oracle.mp(D, y, 0.0, k, "omp")
        m = oracle.mp(D, y, 0.0, k, "mp")
        np.testing.assert_array_equal(o["j"], m["j"])
        np.testing.assert_allclose(o["alpha"], m["alpha"], rtol=1e-12, atol=1e-12 * np.linalg.norm(y))


def test_each_refit_is_the_least_squares_solution():
    for y in _blocks():
        b = int(np.sqrt(y.size))
        D = oracle.dictionary(b, 0)
        r = oracle.mp(D, y, 0.0, y.size // 4, "omp")
        for t in range(1, r["steps"] + 1):
            rt = oracle.mp(D, y, 0.0, t, "omp")
            np.testing.assert_array_equal(rt["j"], r["j"][:t])
            x, *_ = np.linalg.lstsq(D[rt["j"]].T, y, rcond=None)
            np.testing.assert_allclose(rt["alpha"], x, rtol=1e-9, atol=1e-9 * np.linalg.norm(y))
            res = y - D[rt["j"]].T @ rt["alpha"]
            assert np.abs(D[rt["j"]] @ res).max() <= 1e-9 * np.linalg.norm(y)
            assert abs(res @ res - rt["energy"][-1]) <= 1e-9 * (y @ y)
        # the energy never rises and the stop rule holds
        assert np.all(np.diff(r["energy"]) <= 1e-9 * (y @ y))


def test_stop_rule_and_quadtree():
    img = synthetic.gradient_scene(32, 32, seed=5)
    enc = oracle.encode([img], [2.0], min_block=4, max_block=16, algorithm="omp")
    assert int(np.sum(enc.leaves["b"].astype(np.int64) ** 2)) == img.size
    rec = oracle.decode(enc, 0, 32, 32)
    for L in enc.leaves:
        b, y0, x0 = int(L["b"]), int(L["y"]), int(L["x"])
        err = rec[y0:y0 + b, x0:x0 + b] - img[y0:y0 + b, x0:x0 + b]
        if L["converged"]:
            assert float(np.sum(err * err)) < 4.0 * b * b
        else:
            assert b == 4
