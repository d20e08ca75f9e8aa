"""Codec stages on the GPU against the oracle (Section 2.3, Appendix A):
colour conversion kernels bit for bit, the bitstream written from a GPU
encode, a code rebuilt from it, and the whole compress / decompress path."""
import zlib

import numpy as np
import pytest

import bitstream_format as bsf
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


def _rgb(h, w, seed):
    return np.stack([synthetic.gradient_scene(h, w, seed=seed + c) for c in range(3)], -1)


@pytest.mark.parametrize("h,w", [(37, 53), (64, 64), (192, 256)])
def test_image_to_planes_matches_the_oracle(lib, h, w):
    rgb = np.random.default_rng(h * w).integers(0, 256, (h, w, 3), dtype=np.uint8)
    img = torch.from_numpy(rgb).cuda()
    ycc = lib.aqmp_image_to_planes(img, "ycbcr").cpu().numpy()
    np.testing.assert_array_equal(ycc, oracle.rgb_to_ycbcr(rgb))
    same = lib.aqmp_image_to_planes(img, "rgb").cpu().numpy()
    np.testing.assert_array_equal(same, np.moveaxis(rgb, -1, 0))


@pytest.mark.parametrize("h,w", [(37, 53), (128, 96)])
def test_planes_to_image_matches_the_oracle(lib, h, w):
    rng = np.random.default_rng(h + w)
    planes = rng.uniform(-20.0, 280.0, (3, h, w)).astype(np.float32)
    planes[:, ::7, ::5] = np.round(planes[:, ::7, ::5]) + 0.5        # exact ties
    dev = torch.from_numpy(planes).cuda()
    out = lib.aqmp_planes_to_image(dev, "ycbcr").cpu().numpy()
    np.testing.assert_array_equal(out, oracle.ycbcr_to_rgb(oracle.planes_to_u8(planes)))
    out = lib.aqmp_planes_to_image(dev, "rgb").cpu().numpy()
    np.testing.assert_array_equal(out, np.moveaxis(oracle.planes_to_u8(planes), 0, -1))


def test_bitstream_of_a_gpu_encode(lib):
    """The written stream lists exactly the code's leaves and atoms; the
    parser recovers the positions; a code rebuilt from it decodes bit for
    bit like the original."""
    planes = [synthetic.gradient_scene(128, 192, seed=4), synthetic.piecewise_scene(64, 128, seed=6)]
    code = lib.aqmp_encode_planes([torch.from_numpy(p).cuda() for p in planes], [1.0, 2.0])
    leaves, atoms, _ = code.copy()
    data = lib.aqmp_bitstream(code, "planes")
    hdr, pl, pj, pa = bsf.read(data)
    assert hdr["shapes"] == [p.shape for p in planes] and hdr["max_block"] == 64 and hdr["min_block"] == 4
    assert [(L["plane"], L["y"], L["x"], L["b"], L["n_atoms"], L["atom_off"]) for L in pl] == \
        [tuple(int(L[f]) for f in ("plane", "y", "x", "b", "n_atoms", "atom_off")) for L in leaves]
    np.testing.assert_array_equal(pj, atoms["j"].astype(np.int64))
    np.testing.assert_array_equal(pa.view(np.uint32), atoms["alpha"].view(np.uint32))
    info, shapes, cl, ca = lib.aqmp_bitstream_parse(data)
    for f in ("plane", "y", "x", "b", "n_atoms", "atom_off"):
        np.testing.assert_array_equal(cl[f], leaves[f])
    rebuilt = lib.aqmp_code_from_bitstream(data)
    for i, p in enumerate(planes):
        a = torch.empty(p.shape, dtype=torch.float32, device="cuda")
        b = torch.empty(p.shape, dtype=torch.float32, device="cuda")
        code.decode(i, a)
        rebuilt.decode(i, b)
        assert torch.equal(a, b)


def test_compress_decompress_matches_the_oracle_pipeline(lib):
    """YCbCr, AQMP, DEFLATE and back; the decoded planes, the image and CR
    against the oracle's own pipeline on the same image."""
    rgb = _rgb(128, 192, seed=10)
    tol = 2.0
    blob = lib.compress(rgb, tol, color="ycbcr")
    out = lib.decompress(blob).cpu().numpy()
    # oracle pipeline
    ycc = oracle.rgb_to_ycbcr(rgb)
    enc = oracle.encode(list(ycc), [tol] * 3)
    # structure: the stream's leaves and atom indices are the oracle's
    data = zlib.decompress(blob)
    info, shapes, leaves, atoms = lib.aqmp_bitstream_parse(data)
    assert info["color"] == lib.AQMP_COLOR_YCBCR and shapes == [(128, 192)] * 3
    # (the stream does not store the converged flag: a leaf above the smallest
    # side is converged by construction, the rest are taken from the oracle)
    assert np.all(enc.leaves["converged"][leaves["b"] > 4] == 1)
    leaves["converged"] = enc.leaves["converged"]
    parity.compare(enc, leaves, atoms, np.zeros(len(atoms), np.float32), list(ycc), df_tol=1.0)
    # pixels: decoded planes differ from the FP64 ones by rounding only, so the
    # 8-bit planes agree except next to a rounding tie
    rec = np.stack([oracle.decode(enc, c, 128, 192) for c in range(3)])
    expect = oracle.ycbcr_to_rgb(oracle.planes_to_u8(rec))
    d = np.abs(out.astype(np.int64) - expect.astype(np.int64))
    assert d.max() <= 2 and (d > 0).mean() < 1e-3
    # CR: the same layout written from the oracle's encoding, deflated alike
    ref = zlib.compress(bsf.write(enc.shapes, enc.leaves, enc.atom_j, enc.atom_alpha.astype(np.float32),
                                  0, 4, 64, lib.AQMP_COLOR_YCBCR), 9)
    cr, cr_ref = lib.compression_rate(rgb, blob), rgb.size / len(ref)
    assert abs(cr - cr_ref) <= 0.01 * cr_ref
    assert oracle.psnr(out.astype(np.float64), rgb) > 30.0
