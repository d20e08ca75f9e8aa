"""Comparison helpers: CUDA library output against the FP64 oracle.

Bar (from the arithmetic of the two sides):
  * atom indices, leaf positions / sizes / step counts, converged flags and
    the quadtree shape: identical;
  * alpha (the stored FP32 coefficient): |a_gpu - a_fp64| <= 1e-5 |a_fp64|
    (plus 1e-9 ||y|| for coefficients at rounding level);
  * alpha as computed (hi + lo double-float): |a - a_fp64| <= 2^-34 ||y||,
    which the certification band (2^-36 ||y||) sits below.
Leaves whose pursuit (or an ancestor's) reported a near tie are not
certified; callers decide whether any are allowed (the tests allow none)."""
import numpy as np

import oracle


def _key(L):
    return (int(L["plane"]), int(L["y"]), int(L["x"]), int(L["b"]))


def compare(enc, leaves, atoms, alpha_lo, planes, rel_tol=1e-5, df_tol=2.0 ** -34, allow_flagged=False):
    """Compare a whole encode; returns a dict of statistics, raises
    AssertionError on the first disagreement."""
    assert len(leaves) == len(enc.leaves), f"leaf count {len(leaves)} vs oracle {len(enc.leaves)}"
    worst_rel = 0.0
    worst_df = 0.0
    for i, (G, O) in enumerate(zip(leaves, enc.leaves)):
        assert _key(G) == _key(O), f"leaf {i}: {_key(G)} vs oracle {_key(O)}"
        assert int(G["n_atoms"]) == int(O["n_atoms"]), f"leaf {i} {_key(G)}: steps {G['n_atoms']} vs {O['n_atoms']}"
        assert int(G["converged"]) == int(O["converged"]), f"leaf {i} {_key(G)}: converged flag"
        assert allow_flagged or int(G["flags"]) == 0, f"leaf {i} {_key(G)}: near-tie flag {int(G['flags'])}"
        n = int(G["n_atoms"])
        gs = slice(int(G["atom_off"]), int(G["atom_off"]) + n)
        oj, oa = enc.leaf_atoms(i)
        np.testing.assert_array_equal(atoms["j"][gs].astype(np.int64), oj.astype(np.int64),
                                      err_msg=f"leaf {i} {_key(G)}: atom indices")
        if n:
            b = int(G["b"])
            blk = planes[int(G["plane"])][G["y"]:G["y"] + b, G["x"]:G["x"] + b].astype(np.float64)
            S = float(np.sqrt(np.sum(blk * blk)))
            a32 = atoms["alpha"][gs].astype(np.float64)
            rel = np.abs(a32 - oa) / np.maximum(np.abs(oa), 1e-9 * S / rel_tol)
            worst_rel = max(worst_rel, float(rel.max()))
            assert rel.max() <= rel_tol, f"leaf {i} {_key(G)}: alpha rel err {rel.max():.3g}"
            adf = a32 + alpha_lo[gs].astype(np.float64)
            e = float(np.abs(adf - oa).max()) / max(S, 1.0)
            worst_df = max(worst_df, e)
            assert e <= df_tol, f"leaf {i} {_key(G)}: double-float alpha err {e:.3g} of ||y||"
    return {"leaves": len(leaves), "atoms": int(len(atoms)), "worst_alpha_rel": worst_rel,
            "worst_alpha_df": worst_df}


def restrict_to_roots(leaves, atoms, alpha_lo, plane, roots, max_block, width):
    """GPU leaves (canonical order) of the given roots of one plane, with the
    atom arrays re-based, in root order as listed."""
    rx = width // max_block
    out_l, out_a, out_lo = [], [], []
    off = 0
    for r in roots:
        ry, rxx = divmod(r, rx)
        sel = np.nonzero((leaves["plane"] == plane) & (leaves["y"] // max_block == ry)
                         & (leaves["x"] // max_block == rxx))[0]
        for i in sel:
            L = leaves[i].copy()
            s = slice(int(L["atom_off"]), int(L["atom_off"]) + int(L["n_atoms"]))
            L["atom_off"] = off
            off += int(L["n_atoms"])
            out_l.append(L)
            out_a.append(atoms[s])
            out_lo.append(alpha_lo[s])
    cat = lambda xs, like: np.concatenate(xs) if xs else like[:0]
    return (np.array(out_l, dtype=leaves.dtype) if out_l else leaves[:0], cat(out_a, atoms),
            cat(out_lo, alpha_lo))
