"""The BF16 form with rescore (AQMP_PREC_BF16_RESCORE) on the GPU.

At side 64 it starts each pursuit from the split-BF16 correlation and makes
exact, before every step, each atom whose bounded value could be the argmax;
a leaf needing more than 8 such atoms in one step is redone by the exact
form.  Its decisions are therefore those of the exact form: the same tree
and atom indices, coefficients equal to a few units in the last place of the
double-float state (the rescored atoms' running values differ from the exact
form's only by the rounding of the added difference), and, against the FP64
oracle, the parity of the exact form."""
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


def _run(lib, planes, tols, precision, **kw):
    dev = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in planes]
    code = lib.aqmp_encode_planes(dev, tols, precision=precision, **kw)
    out = code.copy(), code.stats()
    code.free()
    return out


def _same_decisions(a, b, rel=2.0 ** -30):
    (la, aa, loa), _ = a
    (lb, ab, lob), _ = b
    for f in ("plane", "y", "x", "b", "n_atoms", "converged", "atom_off"):
        np.testing.assert_array_equal(la[f], lb[f])
    np.testing.assert_array_equal(aa["j"], ab["j"])
    xa = aa["alpha"].astype(np.float64) + loa
    xb = ab["alpha"].astype(np.float64) + lob
    assert np.all(np.abs(xa - xb) <= rel * np.maximum(np.abs(xb), 1.0))


def test_uneven_gradient_batch_decides_as_the_exact_form(lib):
    batch = synthetic.uneven_rgb_batch(3, seed=0, scene=synthetic.gradient_scene, wmax=1024, hmax=768)
    planes = [c for (_, _, chans) in batch for c in chans]
    ex = _run(lib, planes, 2.0, lib.AQMP_PREC_EXACT)
    rs = _run(lib, planes, 2.0, lib.AQMP_PREC_BF16_RESCORE)
    _same_decisions(rs, ex)
    st = rs[1]
    assert st["rescored_atoms"] > 0
    print(f"\nrescored {st['rescored_atoms']} atoms in {st['rescore_rounds']} rounds over "
          f"{st['attempts_per_level'][0]} side-64 pursuits ({st['iterations_per_level'][0]} steps), "
          f"{st['fallback_leaves']} fallback leaves")


@pytest.mark.parametrize("tol", [1.0, 4.0])
def test_piecewise_planes_decide_as_the_exact_form(lib, tol):
    planes = [synthetic.piecewise_scene(512, 512, seed=1)[:256, :256]]
    _same_decisions(_run(lib, planes, tol, lib.AQMP_PREC_BF16_RESCORE), _run(lib, planes, tol, lib.AQMP_PREC_EXACT))


def test_parity_with_the_oracle(lib):
    planes = [synthetic.gradient_scene(64, 128, seed=3)]
    (leaves, atoms, lo), _ = _run(lib, planes, 2.0, lib.AQMP_PREC_BF16_RESCORE)
    enc = oracle.encode(planes, [2.0], max_block=64)
    parity.compare(enc, leaves, atoms, lo, planes)


def _tied_haar_block():
    """128 plus twelve finest-level 2-D Haar atoms of equal amplitude on
    disjoint 2x2 supports (pixels 128 +- 10): after the constant atom, twelve
    exactly tied correlations, more than a rescore takes."""
    H = oracle.haar_1d(64)
    fine = [r for r in range(64) if np.count_nonzero(np.abs(H[r]) > 1e-12) == 2]
    y = np.zeros((64, 64))
    for k in range(12):
        p, q = fine[2 * k], fine[2 * k + 1]
        y += 20.0 * np.outer(H[p], H[q])
    blk = np.rint(128.0 + y)
    assert np.allclose(blk, 128.0 + y)
    return blk.astype(np.uint8)


def test_more_candidates_than_the_rescore_takes_fall_back(lib):
    planes = [_tied_haar_block()]
    rs = _run(lib, planes, 0.5, lib.AQMP_PREC_BF16_RESCORE, max_block=64, min_block=64)
    ex = _run(lib, planes, 0.5, lib.AQMP_PREC_EXACT, max_block=64, min_block=64)
    assert rs[1]["fallback_leaves"] == 1
    _same_decisions(rs, ex)
    (leaves, atoms, lo), _ = rs
    parity.compare(oracle.encode(planes, [0.5], max_block=64, min_block=64), leaves, atoms, lo, planes)


@pytest.mark.parametrize("dict_id", [1, 2])
def test_single_family(lib, dict_id):
    planes = [synthetic.gradient_scene(128, 128, seed=5)]
    _same_decisions(_run(lib, planes, 2.0, lib.AQMP_PREC_BF16_RESCORE, dict_id=dict_id),
                    _run(lib, planes, 2.0, lib.AQMP_PREC_EXACT, dict_id=dict_id))
