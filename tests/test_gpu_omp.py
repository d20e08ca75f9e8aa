"""Orthogonal Matching Pursuit on the GPU against the FP64 oracle's OMP:
support (atom indices in selection order), quadtree shape and converged
flags identical; coefficients within 1e-5 relative (stored FP32) and
hi + lo within 2^-30 ||y|| (two FP64 evaluations of the same re-fit).
Sides 4..16 run a warp per leaf, sides 32 and 64 a CTA per leaf with the
Cholesky factor in global memory and, past a support size, the separable
W X W^T form of the cross-family Gram terms; the cases below reach both."""
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


def _both(lib, planes, tols, **kw):
    code = lib.aqmp_encode_planes([torch.from_numpy(p).cuda() for p in planes], tols, omp=True, **kw)
    leaves, atoms, lo = code.copy()
    code.free()
    okw = {k: v for k, v in kw.items() if k in ("cap_num", "cap_den", "min_block", "max_block", "dict_id")}
    enc = oracle.encode(planes, tols, algorithm="omp", **okw)
    return leaves, atoms, lo, enc


@pytest.mark.parametrize("tol", [1.0, 2.0, 4.0])
def test_gradient_scene(lib, tol):
    planes = [synthetic.gradient_scene(64, 64, seed=1)]
    leaves, atoms, lo, enc = _both(lib, planes, [tol], max_block=16)
    st = parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    assert st["leaves"] >= 16 and (tol > 2.0 or st["leaves"] > 16)


def test_several_planes_and_sides(lib):
    planes = [synthetic.piecewise_scene(64, 128, seed=2), synthetic.noise_plane(32, 64, seed=3),
              synthetic.uniform_plane(32, 32, 90)]
    leaves, atoms, lo, enc = _both(lib, planes, [1.5, 6.0, 0.5], max_block=16, min_block=4)
    parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    assert set(np.unique(leaves["b"])) >= {4, 16}            # split to the smallest side and kept whole


@pytest.mark.parametrize("dict_id", [1, 2])
def test_single_family_reduces_to_mp(lib, dict_id):
    """On an orthonormal dictionary OMP selects like MP and its re-fit
    returns the MP coefficients."""
    planes = [synthetic.gradient_scene(32, 32, seed=4)]
    leaves, atoms, lo, enc = _both(lib, planes, [1.0], max_block=16, dict_id=dict_id)
    parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    mp = oracle.encode(planes, [1.0], max_block=16, dict_id=dict_id)
    np.testing.assert_array_equal(enc.atom_j, mp.atom_j)


def test_zero_tolerance_runs_the_budget(lib):
    planes = [synthetic.noise_plane(16, 16, seed=5)]
    leaves, atoms, lo, enc = _both(lib, planes, [0.0], max_block=8, min_block=8)
    parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    assert np.all(leaves["n_atoms"] == 16)


def test_fewer_atoms_than_mp_for_the_same_tolerance(lib):
    """The re-fit removes more energy per atom: at the same tolerance OMP
    never needs more atoms than MP on a leaf both keep."""
    planes = [synthetic.piecewise_scene(64, 64, seed=6)]
    o = lib.aqmp_encode_planes([torch.from_numpy(planes[0]).cuda()], 2.0, omp=True, max_block=16)
    m = lib.aqmp_encode_planes([torch.from_numpy(planes[0]).cuda()], 2.0, max_block=16)
    assert o.stats()["n_atoms"] <= m.stats()["n_atoms"]


def test_side64_gradient_root(lib):
    """One 64x64 root that converges at side 64 (direct cross terms)."""
    planes = [synthetic.gradient_scene(64, 64, seed=1)]
    leaves, atoms, lo, enc = _both(lib, planes, [4.0], max_block=64)
    parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    assert 64 in set(np.unique(leaves["b"]))


def test_side64_budget_splits_down_the_tree(lib):
    """A capped budget (32 atoms at side 64, 8 at 32, ...) makes the roots
    split through every level of the 64 -> 4 tree."""
    planes = [synthetic.piecewise_scene(64, 64, seed=2)]
    leaves, atoms, lo, enc = _both(lib, planes, [1.0], max_block=64, cap_num=1, cap_den=128)
    parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    assert len(leaves) > 4


def test_side32_past_the_separable_crossover(lib):
    """128 atoms on one noise block of side 32: each family's support passes
    the 51 atoms above which its cross terms go through W X W^T."""
    planes = [synthetic.noise_plane(32, 32, seed=3)]
    leaves, atoms, lo, enc = _both(lib, planes, [0.0], max_block=32, min_block=32, cap_num=1, cap_den=8)
    parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    j = atoms["j"]
    assert min(int(np.sum(j < 1024)), int(np.sum(j >= 1024))) > 51


def test_side64_past_the_separable_crossover(lib):
    """256 atoms on one noise block of side 64 (the oracle needs ~30 s):
    both families' supports pass the 120 atoms of the side-64 crossover."""
    planes = [synthetic.noise_plane(64, 64, seed=3)]
    leaves, atoms, lo, enc = _both(lib, planes, [0.0], max_block=64, min_block=64, cap_num=1, cap_den=16)
    parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    j = atoms["j"]
    assert min(int(np.sum(j < 4096)), int(np.sum(j >= 4096))) > 120


@pytest.mark.parametrize("dict_id", [1, 2])
def test_side64_single_family_reduces_to_mp(lib, dict_id):
    planes = [synthetic.gradient_scene(64, 64, seed=4)]
    leaves, atoms, lo, enc = _both(lib, planes, [4.0], max_block=64, dict_id=dict_id)
    parity.compare(enc, leaves, atoms, lo, planes, df_tol=2.0 ** -30)
    mp = oracle.encode(planes, [4.0], max_block=64, dict_id=dict_id)
    np.testing.assert_array_equal(enc.atom_j, mp.atom_j)


def test_unsupported_configurations_are_refused(lib):
    plane = torch.from_numpy(synthetic.gradient_scene(128, 128, seed=7)).cuda()
    for kw in ({"max_block": 128}, {"max_block": 64, "cap_num": 1, "cap_den": 2},
               {"max_block": 16, "cap_num": 1, "cap_den": 2},
               {"max_block": 16, "precision": lib.AQMP_PREC_FP32}):
        with pytest.raises(lib.AqmpError) as e:
            lib.aqmp_encode_planes([plane], 2.0, omp=True, **kw)
        assert e.value.code == -8                              # AQMP_E_UNSUPPORTED
