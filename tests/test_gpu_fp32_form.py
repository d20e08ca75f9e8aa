"""The plain FP32 form (precision AQMP_PREC_FP32): FP32 pursuit state, not
certified.  It must still produce a valid quadtree code (tiling, budgets,
converged leaves meeting the tolerance on their own reconstruction), and its
agreement with the exact form is measured: the share of identical leaves and
the PSNR / SSIM differences."""
import json

import numpy as np
import pytest

import oracle
from paper_2605_09190_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    assert torch.cuda.is_available()
    return aqmp


def test_fp32_form_is_valid_and_close_to_the_exact_form(lib, tmp_path):
    img = synthetic.piecewise_scene(512, 512, seed=1)
    tols = [1.0, 2.0, 4.0, 8.0]
    dev = [torch.from_numpy(img).cuda()] * 4
    exact = lib.aqmp_encode_planes(dev, tols)
    fp32 = lib.aqmp_encode_planes(dev, tols, precision=lib.AQMP_PREC_FP32)
    le, ae, _ = exact.copy()
    lf, af, _ = fp32.copy()
    report = {}
    out = torch.empty((512, 512), dtype=torch.float32, device="cuda")
    for p, tol in enumerate(tols):
        sel = lf[lf["plane"] == p]
        cover = np.zeros(img.shape, int)
        for L in sel:
            cover[L["y"]:L["y"] + L["b"], L["x"]:L["x"] + L["b"]] += 1
            assert L["n_atoms"] <= oracle.sparsity_cap(int(L["b"]))
        assert np.all(cover == 1)
        fp32.decode(p, out)
        rf = out.cpu().numpy().astype(np.float64)
        exact.decode(p, out)
        re_ = out.cpu().numpy().astype(np.float64)
        for L in sel:
            if L["converged"]:
                b, y, x = int(L["b"]), int(L["y"]), int(L["x"])
                rmse = np.sqrt(np.mean((rf[y:y + b, x:x + b] - img[y:y + b, x:x + b]) ** 2))
                # FP32 energy bookkeeping: the reconstruction may miss the
                # tolerance by FP32 rounding of ||y||^2 - sum alpha^2
                assert rmse < tol * 1.01
        se = le[le["plane"] == p]
        keys_e = {(int(L["y"]), int(L["x"]), int(L["b"])) for L in se}
        keys_f = {(int(L["y"]), int(L["x"]), int(L["b"])) for L in sel}
        report[tol] = {"leaves_exact": len(se), "leaves_fp32": len(sel),
                       "same_leaf_positions": len(keys_e & keys_f) / max(1, len(keys_e | keys_f)),
                       "psnr_exact": oracle.psnr(re_, img), "psnr_fp32": oracle.psnr(rf, img),
                       "ssim_exact": oracle.ssim(re_, img), "ssim_fp32": oracle.ssim(rf, img)}
        assert abs(report[tol]["psnr_fp32"] - report[tol]["psnr_exact"]) < 0.5
        assert abs(report[tol]["ssim_fp32"] - report[tol]["ssim_exact"]) < 0.01
    print(json.dumps(report, indent=1))            # the comparison, shown with pytest -s


@pytest.mark.parametrize("max_block", [64, 128])
def test_bf16_form_tiles_and_stays_close_to_the_exact_form(lib, max_block):
    """The reduced-precision form (BF16 correlation, FP32 pursuit): a valid
    quadtree whose reconstruction is within a fraction of a dB of the exact
    (certified) form's."""
    img = synthetic.piecewise_scene(256, 256, seed=3)
    dev = torch.from_numpy(img).cuda()
    codes = {p: lib.aqmp_encode_planes([dev], 2.0, max_block=max_block, precision=p)
             for p in (lib.AQMP_PREC_EXACT, lib.AQMP_PREC_BF16)}
    psnr = {}
    for p, code in codes.items():
        leaves, atoms, lo = code.copy()
        assert int(np.sum(leaves["b"].astype(np.int64) ** 2)) == img.size
        out = torch.empty(img.shape, dtype=torch.float32, device="cuda")
        code.decode(0, out)
        psnr[p] = oracle.psnr(out.cpu().numpy().astype(np.float64), img)
    assert abs(psnr[lib.AQMP_PREC_BF16] - psnr[lib.AQMP_PREC_EXACT]) < 0.5
