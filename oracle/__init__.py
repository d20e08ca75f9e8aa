"""FP64 CPU oracle for the AQMP encoder hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library never
loads it and shares no code, table or constant generator with it.

The arithmetic lives in ``aqmp_oracle.c`` (plain C, double precision, sums in
ascending index order, built with ``-ffp-contract=off``); this module compiles
it on first use, marshals numpy arrays through ctypes and adds the image
metrics, which the paper defines in Section 3:

* PSNR = 10 log10(255^2 / MSE) on the reconstruction clipped to [0, 255]
  (the paper uses SSIM only; PSNR is the conventional companion metric);
* SSIM, Section 3 equation, with C1 = (K1 L)^2, C2 = (K2 L)^2, K1 = 0.01,
  K2 = 0.03, L = 255 (the values the paper calls common) and an 11x11
  Gaussian window of sigma 1.5 over the valid region (the paper names no
  window; this is the usual one).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aqmp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lib_lock = threading.Lock()

LEAF_DTYPE = np.dtype([("plane", np.int32), ("b", np.int32), ("y", np.int32),
                       ("x", np.int32), ("atom_off", np.int32), ("n_atoms", np.int32),
                       ("converged", np.int32), ("_pad", np.int32),
                       ("min_margin", np.float64)])


def build(force: bool = False) -> str:
    """Compile the oracle's C source into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    P = ctypes.c_void_p
    I, L, Dbl = ctypes.c_int, ctypes.c_long, ctypes.c_double
    lib.oracle_dct_1d.argtypes = [I, P]
    lib.oracle_haar_1d.argtypes = [I, P]
    lib.oracle_haar_1d.restype = I
    lib.oracle_dictionary.argtypes = [I, I, P]
    lib.oracle_dictionary.restype = I
    lib.oracle_mp.argtypes = [P, I, I, P, Dbl, I, P, P, P, P, P]
    lib.oracle_mp.restype = I
    lib.oracle_omp.argtypes = [P, I, I, P, Dbl, I, P, P, P, P, P]
    lib.oracle_omp.restype = I
    lib.oracle_encode_roots.argtypes = [P, L, I, I, I, Dbl, I, I, I, I, I, P, L, L,
                                        P, L, P, P, P, L, P, P, P, I]
    lib.oracle_encode_roots.restype = I
    lib.oracle_decode_leaf.argtypes = [P, I, I, I, P, P, I, P, L]
    return lib


def _load():
    global _lib
    with _lib_lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
        return _lib


class use_library:
    """Context manager that points this module at another build of the
    oracle's C source (used by the tests that plant mistakes in a copy of it
    to show that the pins catch them)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        with _lib_lock:
            self._saved = _lib
            _lib = _configure(ctypes.CDLL(self.path))
        with _dict_lock:
            self._saved_dicts = dict(_dict_cache)
            _dict_cache.clear()
        return self

    def __exit__(self, *exc):
        global _lib
        with _lib_lock:
            _lib = self._saved
        with _dict_lock:
            _dict_cache.clear()
            _dict_cache.update(self._saved_dicts)
        return False


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# ------------------------------------------------------------------ tables

def dct_1d(b: int) -> np.ndarray:
    """1-D DCT-II matrix C[k, m] (Section 2.1, Eq. (1)-(2))."""
    out = np.empty((b, b), np.float64)
    _load().oracle_dct_1d(b, _ptr(out))
    return out


def haar_1d(b: int) -> np.ndarray:
    """1-D orthonormal Haar matrix, rows ordered scaling, then scale by scale."""
    out = np.empty((b, b), np.float64)
    if _load().oracle_haar_1d(b, _ptr(out)) != 0:
        raise ValueError("Haar side must be a power of two")
    return out


def num_atoms(b: int, dict_id: int) -> int:
    return 2 * b * b if dict_id == 0 else b * b


_dict_cache: dict = {}
_dict_lock = threading.Lock()


def dictionary(b: int, dict_id: int = 0) -> np.ndarray:
    """D_N as an (M, n) array: row j is atom j over the unravelled block."""
    key = (b, dict_id)
    with _dict_lock:
        if key not in _dict_cache:
            D = np.empty((num_atoms(b, dict_id), b * b), np.float64)
            if _load().oracle_dictionary(b, dict_id, _ptr(D)) != 0:
                raise ValueError(f"bad dictionary side {b}")
            _dict_cache[key] = D
        return _dict_cache[key]


def sparsity_cap(b: int, cap_num: int = 1, cap_den: int = 4) -> int:
    """Per-size atom budget k = max(1, floor(b^2 cap_num / cap_den))."""
    return max(1, (b * b * cap_num) // cap_den)


def eps2_of(tol: float, b: int) -> float:
    """Squared l2 threshold for an RMSE tolerance on the 0-255 scale.

    ``tol`` is first rounded to float32, the precision the library's
    parameter block carries, so both sides compare against the same value."""
    t = float(np.float32(tol))
    return t * t * float(b * b)


# ---------------------------------------------------------------- pursuit

def unravel(block: np.ndarray) -> np.ndarray:
    """Concatenate the block's columns (Appendix A)."""
    return np.ascontiguousarray(np.asarray(block, np.float64).T).reshape(-1)


def mp(D: np.ndarray, y: np.ndarray, eps2: float, k: int, algorithm: str = "mp") -> dict:
    """Matching Pursuit on one vector (Section 2.2 with Eq. (3)); with
    algorithm="omp", Orthogonal Matching Pursuit (least-squares re-fit of the
    support after every selection; `alpha` holds the final coefficients)."""
    D = np.ascontiguousarray(D, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    M, n = D.shape
    j = np.zeros(max(k, 1), np.int32)
    al = np.zeros(max(k, 1), np.float64)
    mg = np.zeros(max(k, 1), np.float64)
    en = np.zeros(k + 1, np.float64)
    conv = ctypes.c_int(0)
    fn = _load().oracle_omp if algorithm == "omp" else _load().oracle_mp
    t = fn(_ptr(D), n, M, _ptr(y), float(eps2), int(k), _ptr(j), _ptr(al), _ptr(mg), _ptr(en),
           ctypes.byref(conv))
    if t < 0:
        raise MemoryError("oracle pursuit allocation failed")
    return {"j": j[:t].copy(), "alpha": al[:t].copy(), "margin": mg[:t].copy(),
            "energy": en[:t + 1].copy(), "converged": bool(conv.value), "steps": t}


class Encoding:
    """Leaves in depth-first order (per plane, roots row-major) and atoms."""

    def __init__(self, leaves, atom_j, atom_alpha, attempts, steps, shapes):
        self.leaves = leaves
        self.atom_j = atom_j
        self.atom_alpha = atom_alpha
        self.attempts = attempts
        self.steps = steps
        self.shapes = shapes

    def leaf_atoms(self, i):
        L = self.leaves[i]
        s = slice(int(L["atom_off"]), int(L["atom_off"]) + int(L["n_atoms"]))
        return self.atom_j[s], self.atom_alpha[s]


def _dict_ptrs(min_block, max_block, dict_id):
    nlev = int(np.log2(max_block)) + 1
    arrs = [None] * nlev
    ptrs = (ctypes.c_void_p * nlev)()
    b = min_block
    while b <= max_block:
        lv = int(np.log2(b))
        arrs[lv] = dictionary(b, dict_id)
        ptrs[lv] = arrs[lv].ctypes.data
        b *= 2
    return arrs, ptrs


def encode(planes, tols, cap_num=1, cap_den=4, min_block=4, max_block=64, dict_id=0,
           roots=None, threads=None, algorithm: str = "mp") -> Encoding:
    """Algorithms 1-2 over a list of 2-D uint8 planes, one tolerance per plane.

    ``roots`` optionally restricts plane p to the root indices ``roots[p]``
    (row-major root numbering); work is spread over ``threads`` host threads,
    one root per task (roots are independent subtrees)."""
    planes = [np.ascontiguousarray(p, np.uint8) for p in planes]
    if np.isscalar(tols):
        tols = [tols] * len(planes)
    tols = [float(np.float32(t)) for t in tols]
    _arrs, ptrs = _dict_ptrs(min_block, max_block, dict_id)
    lib = _load()
    tasks = []
    for p, pl in enumerate(planes):
        h, w = pl.shape
        if h % max_block or w % max_block:
            raise ValueError("plane size must be a multiple of max_block")
        nroots = (h // max_block) * (w // max_block)
        rs = range(nroots) if roots is None or roots[p] is None else roots[p]
        for r in rs:
            tasks.append((p, int(r)))

    def run(task):
        p, r = task
        pl = planes[p]
        h, w = pl.shape
        cap_leaves = (max_block // min_block) ** 2
        # every leaf holds at most max(1, b^2 cap) atoms, so a root's subtree
        # holds at most max_block^2 * ceil(cap) + (number of leaves)
        cap_atoms = max_block * max_block * max(1, -(-cap_num // cap_den)) + cap_leaves
        lv = np.zeros(cap_leaves, LEAF_DTYPE)
        aj = np.zeros(cap_atoms, np.int32)
        aa = np.zeros(cap_atoms, np.float64)
        nl, na, att, st = (ctypes.c_long(), ctypes.c_long(), ctypes.c_long(), ctypes.c_long())
        rc = lib.oracle_encode_roots(_ptr(pl), w, h, w, p, tols[p], cap_num, cap_den,
                                     min_block, max_block, dict_id, ptrs, r, r + 1,
                                     _ptr(lv), cap_leaves, ctypes.byref(nl), _ptr(aj), _ptr(aa),
                                     cap_atoms, ctypes.byref(na), ctypes.byref(att),
                                     ctypes.byref(st), 1 if algorithm == "omp" else 0)
        if rc != 0:
            raise RuntimeError(f"oracle_encode_roots failed with {rc}")
        return lv[:nl.value], aj[:na.value], aa[:na.value], att.value, st.value

    nthreads = threads or min(len(tasks), os.cpu_count() or 1) or 1
    if nthreads > 1 and len(tasks) > 1:
        with ThreadPoolExecutor(nthreads) as ex:
            parts = list(ex.map(run, tasks))
    else:
        parts = [run(t) for t in tasks]
    leaves, js, als = [], [], []
    off = 0
    attempts = steps = 0
    for lv, aj, aa, att, st in parts:
        lv = lv.copy()
        lv["atom_off"] += off
        off += len(aj)
        leaves.append(lv)
        js.append(aj)
        als.append(aa)
        attempts += att
        steps += st
    cat = (lambda xs, dt: np.concatenate(xs) if xs else np.zeros(0, dt))
    return Encoding(cat(leaves, LEAF_DTYPE), cat(js, np.int32), cat(als, np.float64),
                    attempts, steps, [p.shape for p in planes])


def decode(enc: Encoding, plane: int, h: int, w: int, dict_id: int = 0) -> np.ndarray:
    """Algorithm 3 for one plane: FP64 reconstruction (unclipped)."""
    out = np.zeros((h, w), np.float64)
    lib = _load()
    for i in np.nonzero(enc.leaves["plane"] == plane)[0]:
        L = enc.leaves[i]
        b = int(L["b"])
        D = dictionary(b, dict_id)
        aj, aa = enc.leaf_atoms(i)
        aj = np.ascontiguousarray(aj)
        aa = np.ascontiguousarray(aa)
        lib.oracle_decode_leaf(_ptr(D), b, int(L["y"]), int(L["x"]), _ptr(aj), _ptr(aa),
                               len(aj), _ptr(out), w)
    return out


# ----------------------------------------------------------------- metrics

def psnr(recon: np.ndarray, ref: np.ndarray) -> float:
    """PSNR in dB on the reconstruction clipped to [0, 255]."""
    x = np.clip(np.asarray(recon, np.float64), 0.0, 255.0)
    d = x - np.asarray(ref, np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(255.0 ** 2 / mse)


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(r * r) / (2.0 * sigma * sigma))
    w = np.outer(g, g)
    return w / w.sum()


def ssim(recon: np.ndarray, ref: np.ndarray, L: float = 255.0, K1: float = 0.01,
         K2: float = 0.03, size: int = 11, sigma: float = 1.5, clip: bool = True) -> float:
    """Mean SSIM (Section 3 equation) over the valid region of an 11x11
    Gaussian window; the reconstruction is clipped to [0, 255] first unless
    `clip` is False (the differentiable refinement's loss)."""
    x = np.asarray(ref, np.float64)
    y = np.asarray(recon, np.float64)
    if clip:
        y = np.clip(y, 0.0, 255.0)
    w = gaussian_window(size, sigma)
    H, W = x.shape
    oh, ow = H - size + 1, W - size + 1
    mx = np.zeros((oh, ow)); my = np.zeros((oh, ow))
    sxx = np.zeros((oh, ow)); syy = np.zeros((oh, ow)); sxy = np.zeros((oh, ow))
    for di in range(size):
        for dj in range(size):
            a = x[di:di + oh, dj:dj + ow]
            b = y[di:di + oh, dj:dj + ow]
            c = w[di, dj]
            mx += c * a; my += c * b
            sxx += c * a * a; syy += c * b * b; sxy += c * a * b
    vx = sxx - mx * mx
    vy = syy - my * my
    cxy = sxy - mx * my
    C1 = (K1 * L) ** 2
    C2 = (K2 * L) ** 2
    smap = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    return float(smap.mean())


# ---------------------------------------------------------------- codec stages
# Section 2.3 step (i) converts an image's channels to RGB or YCbCr and codes
# each channel on its own; the decoder's step (iii) converts back.  The
# paper fixes no YCbCr variant.  Reading: the full-range JFIF matrix (ITU-T
# T.871), Y = 0.299 R + 0.587 G + 0.114 B, Cb = 128 - 0.168736 R -
# 0.331264 G + 0.5 B, Cr = 128 + 0.5 R - 0.418688 G - 0.081312 B, with the
# inverse R = Y + 1.402 (Cr - 128), G = Y - 0.344136 (Cb - 128) -
# 0.714136 (Cr - 128), B = Y + 1.772 (Cb - 128); every coefficient taken in
# 16-bit fixed point (round(c 2^16); the two pairs that must cancel on greys
# are rounded to sum to 2^15), the sum rounded half up and clamped to
# [0, 255].  Integer arithmetic, so the definition is exact.  Decoded
# planes are real-valued and are first rounded to the nearest integer, ties
# to even, and clamped.

_YCC_FWD = np.array([[19595, 38470, 7471],
                     [-11058, -21710, 32768],
                     [32768, -27439, -5329]], np.int64)
_YCC_INV = np.array([[0, 91881],            # R: (Cb - 128, Cr - 128)
                     [-22553, -46802],      # G
                     [116130, 0]], np.int64)  # B


def rgb_to_ycbcr(img: np.ndarray) -> np.ndarray:
    """(h, w, 3) uint8 RGB -> (3, h, w) uint8 Y, Cb, Cr."""
    rgb = np.asarray(img).astype(np.int64)
    out = np.empty((3,) + rgb.shape[:2], np.int64)
    for c in range(3):
        acc = (_YCC_FWD[c, 0] * rgb[..., 0] + _YCC_FWD[c, 1] * rgb[..., 1]
               + _YCC_FWD[c, 2] * rgb[..., 2] + 32768)
        if c > 0:
            acc = acc + (128 << 16)
        out[c] = acc >> 16                      # floor: with + 2^15, half up
    return np.clip(out, 0, 255).astype(np.uint8)


def ycbcr_to_rgb(planes: np.ndarray) -> np.ndarray:
    """(3, h, w) uint8 Y, Cb, Cr -> (h, w, 3) uint8 RGB."""
    p = np.asarray(planes).astype(np.int64)
    y, db, dr = p[0], p[1] - 128, p[2] - 128
    out = np.empty(p.shape[1:] + (3,), np.int64)
    for c in range(3):
        out[..., c] = y + ((_YCC_INV[c, 0] * db + _YCC_INV[c, 1] * dr + 32768) >> 16)
    return np.clip(out, 0, 255).astype(np.uint8)


def planes_to_u8(planes: np.ndarray) -> np.ndarray:
    """Decoded real-valued planes -> uint8: nearest integer (ties to even),
    clamped to [0, 255]."""
    return np.clip(np.rint(np.asarray(planes, np.float64)), 0, 255).astype(np.uint8)
