"""Independent Python statement of the library's bitstream layout (the input
of the lossless stage, Section 2.3 step (iii)), used to check the library's
writer and parser against each other and against the oracle's encodings.

Little-endian: "AQMP", u8 version (1), u8 color, u8 dict_id, u8 0,
u16 min_block, u16 max_block, u32 n_planes; per plane u32 h, w, n_leaves,
n_atoms; then per plane: n_leaves u8 levels log2(max_block / b), n_leaves
LEB128 step counts, n_atoms u16 atom indices, n_atoms f32 coefficients.
Leaves are listed in canonical order (planes, roots in raster order,
depth-first TL, TR, BL, BR); positions are implied by that order."""
import struct

import numpy as np


def _varint(v):
    out = bytearray()
    while v >= 0x80:
        out.append((v & 0x7F) | 0x80)
        v >>= 7
    out.append(v)
    return bytes(out)


def write(shapes, leaves, atom_j, atom_alpha, dict_id, min_block, max_block, color=0):
    """shapes: [(h, w)]; leaves: records with plane, b, n_atoms, atom_off
    (canonical order); atom_j / atom_alpha: flat arrays indexed by atom_off."""
    top = int(np.log2(max_block))
    out = bytearray(b"AQMP")
    out += struct.pack("<BBBBHHI", 1, color, dict_id, 0, min_block, max_block, len(shapes))
    per = [[L for L in leaves if int(L["plane"]) == p] for p in range(len(shapes))]
    for (h, w), ls in zip(shapes, per):
        out += struct.pack("<IIII", h, w, len(ls), sum(int(L["n_atoms"]) for L in ls))
    for ls in per:
        out += bytes(top - int(np.log2(int(L["b"]))) for L in ls)
        for L in ls:
            out += _varint(int(L["n_atoms"]))
        for L in ls:
            o, n = int(L["atom_off"]), int(L["n_atoms"])
            out += np.asarray(atom_j[o:o + n], "<u2").tobytes()
        for L in ls:
            o, n = int(L["atom_off"]), int(L["n_atoms"])
            out += np.asarray(atom_alpha[o:o + n], "<f4").tobytes()
    return bytes(out)


def read(data):
    """-> dict(header), list of leaves (plane, y, x, b, n_atoms, atom_off),
    atom indices, coefficients (float32)."""
    assert data[:4] == b"AQMP"
    version, color, dict_id, _, nb, mb, np_ = struct.unpack_from("<BBBBHHI", data, 4)
    pos = 16
    heads = []
    for _ in range(np_):
        heads.append(struct.unpack_from("<IIII", data, pos))
        pos += 16
    leaves, js, alphas = [], [], []
    for p, (h, w, nl, na) in enumerate(heads):
        levels = list(data[pos:pos + nl])
        pos += nl
        counts = []
        for _ in range(nl):
            v, shift = 0, 0
            while True:
                byte = data[pos]
                pos += 1
                v |= (byte & 0x7F) << shift
                shift += 7
                if not byte & 0x80:
                    break
            counts.append(v)
        j = np.frombuffer(data, "<u2", na, pos).astype(np.int64)
        pos += 2 * na
        a = np.frombuffer(data, "<f4", na, pos).copy()
        pos += 4 * na
        # positions: depth-first walk of each root against the leaf sizes
        base = sum(len(x) for x in js)
        off = 0
        k = 0
        for ry in range(h // mb):
            for rx in range(w // mb):
                stack = [(ry * mb, rx * mb, mb)]
                while stack:
                    y, x, b = stack.pop()
                    lb = mb >> levels[k]
                    if lb < b:
                        c = b // 2
                        stack += [(y + c, x + c, c), (y + c, x, c), (y, x + c, c), (y, x, c)]
                        continue
                    assert lb == b, "leaf larger than its node"
                    leaves.append({"plane": p, "y": y, "x": x, "b": b, "n_atoms": counts[k],
                                   "atom_off": base + off})
                    off += counts[k]
                    k += 1
        assert k == nl, "leaves do not tile the plane"
        js.append(j)
        alphas.append(a)
    assert pos == len(data), "trailing bytes"
    header = {"version": version, "color": color, "dict_id": dict_id, "min_block": nb, "max_block": mb,
              "shapes": [(h, w) for (h, w, _, _) in heads]}
    return header, leaves, np.concatenate(js) if js else np.zeros(0, np.int64), \
        np.concatenate(alphas) if alphas else np.zeros(0, np.float32)

