"""Codec stages without a GPU (Section 2.3 steps (i) and (iii), Appendix A):
the oracle's YCbCr pinned to the ITU-T T.871 matrix, and the library's
host bitstream parser against an independent writer fed with oracle
encodings."""
import numpy as np
import pytest

import bitstream_format as bsf
import oracle
from paper_2605_09190_gb300 import synthetic

# T.871 (JFIF) full-range matrices, as published
T871 = np.array([[0.299, 0.587, 0.114],
                 [-0.168736, -0.331264, 0.5],
                 [0.5, -0.418688, -0.081312]])
T871_INV = np.array([[1.0, 0.0, 1.402],
                     [1.0, -0.344136, -0.714136],
                     [1.0, 1.772, 0.0]])
# 3 x 255 x 2^-17: the most a 16-bit rounding of the three coefficients can move a sum
COEF_ERR = 3 * 255 * 2.0 ** -17


def _colors(seed=0):
    g = np.arange(0, 256, 5)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    rnd = np.random.default_rng(seed).integers(0, 256, (100_000, 3))
    return np.concatenate([grid, rnd]).astype(np.uint8)


def _check_rounding(fixed, real):
    """fixed = round-half-up(real) clamped, except within COEF_ERR of a tie."""
    ref = np.clip(np.floor(real + 0.5), 0, 255)
    d = fixed.astype(np.int64) - ref.astype(np.int64)
    assert np.abs(d).max() <= 1
    far = np.abs(real - np.floor(real) - 0.5) > COEF_ERR
    assert np.all(d[far] == 0)


def test_ycbcr_textbook_primaries_and_greys():
    rgb = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255], [0, 0, 0], [128, 128, 128]]],
                   np.uint8)
    ycc = oracle.rgb_to_ycbcr(rgb)[:, 0, :].T
    # red: Y 76.245, Cb 84.97, Cr 255.5 -> clamp; green: 149.685, 43.528, 21.235;
    # blue: 29.07, 255.5 -> clamp, 107.265
    np.testing.assert_array_equal(ycc, [[76, 85, 255], [150, 44, 21], [29, 255, 107],
                                        [255, 128, 128], [0, 128, 128], [128, 128, 128]])
    v = np.arange(256, dtype=np.uint8)
    grey = np.stack([v, v, v], -1)[None]
    ycc = oracle.rgb_to_ycbcr(grey)
    np.testing.assert_array_equal(ycc[0, 0], v)
    assert np.all(ycc[1:] == 128)
    np.testing.assert_array_equal(oracle.ycbcr_to_rgb(ycc)[0], grey[0])


def test_ycbcr_forward_is_the_real_matrix_rounded():
    rgb = _colors()
    fixed = oracle.rgb_to_ycbcr(rgb[None])[:, 0, :].T
    real = rgb.astype(np.float64) @ T871.T + np.array([0.0, 128.0, 128.0])
    _check_rounding(fixed, real)


def test_ycbcr_inverse_is_the_real_matrix_rounded():
    ycc = _colors(1)
    fixed = oracle.ycbcr_to_rgb(ycc.T[:, None, :])[0]
    real = (ycc.astype(np.float64) - np.array([0.0, 128.0, 128.0])) @ T871_INV.T
    _check_rounding(fixed, real)


def test_ycbcr_round_trip_loses_at_most_one_level():
    rgb = _colors(2)
    back = oracle.ycbcr_to_rgb(oracle.rgb_to_ycbcr(rgb[None]))[0]
    assert np.abs(back.astype(np.int64) - rgb.astype(np.int64)).max() <= 1


def test_planes_to_u8_rounds_ties_to_even_and_clamps():
    x = np.array([0.5, 1.5, 2.5, 2.4999, -0.5, -3.0, 254.5, 255.5, 300.0, 127.50001])
    np.testing.assert_array_equal(oracle.planes_to_u8(x), [0, 2, 2, 2, 0, 0, 254, 255, 255, 128])


# ------------------------------------------------------------ bitstream

@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    aqmp.load_library()
    return aqmp


def _oracle_stream(color=0):
    planes = [synthetic.gradient_scene(64, 96, seed=3), synthetic.piecewise_scene(32, 64, seed=2)]
    enc = oracle.encode(planes, [1.0, 2.0], min_block=4, max_block=32)
    data = bsf.write(enc.shapes, enc.leaves, enc.atom_j, enc.atom_alpha.astype(np.float32), 0, 4, 32, color)
    return enc, data


def test_parser_reads_an_independently_written_oracle_encoding(lib):
    enc, data = _oracle_stream(color=2)
    info, shapes, leaves, atoms = lib.aqmp_bitstream_parse(data)
    assert (info["version"], info["color"], info["dict_id"], info["min_block"], info["max_block"]) == (1, 2, 0, 4, 32)
    assert shapes == [(64, 96), (32, 64)]
    assert len(leaves) == len(enc.leaves) and len(atoms) == len(enc.atom_j)
    for f in ("plane", "y", "x", "b", "n_atoms", "atom_off"):
        np.testing.assert_array_equal(leaves[f].astype(np.int64), enc.leaves[f].astype(np.int64), err_msg=f)
    np.testing.assert_array_equal(atoms["j"].astype(np.int64), enc.atom_j.astype(np.int64))
    np.testing.assert_array_equal(atoms["alpha"], enc.atom_alpha.astype(np.float32))
    assert len(set(zip(leaves["plane"], leaves["y"], leaves["x"]))) == len(leaves)
    # the Python reader agrees with its own writer
    hdr, pl, pj, pa = bsf.read(data)
    assert [(L["plane"], L["y"], L["x"], L["b"]) for L in pl] == \
        [(int(L["plane"]), int(L["y"]), int(L["x"]), int(L["b"])) for L in enc.leaves]


def test_parser_rejects_malformed_streams(lib):
    _, data = _oracle_stream()
    bad = [data[:3], b"XQMP" + data[4:], data[:-1], data + b"\0",
           data[:4] + bytes([2]) + data[5:]]                      # version 2
    # a leaf larger than its root: level byte of the first leaf set past the top
    nl0 = int.from_bytes(data[24:28], "little")
    first_level = 16 + 16 * 2
    bad.append(data[:first_level] + bytes([9]) + data[first_level + 1:])
    # the second leaf of a split root claims the whole root
    k = next(i for i in range(nl0 - 1) if data[first_level + i] > 0) + 1
    bad.append(data[:first_level + k] + bytes([0]) + data[first_level + k + 1:])
    for blob in bad:
        with pytest.raises(lib.AqmpError) as e:
            lib.aqmp_bitstream_parse(blob)
        assert e.value.code == -1                                 # AQMP_E_ARG
