"""Thin ctypes binding of libaqmp.so (include/aqmp.h): argument marshalling
only.  Every step of the encoder runs in the library's CUDA kernels; there is
no Python or CPU fallback, and a missing library raises immediately.

Names follow the C ABI: ``aqmp_encode_planes``, ``aqmp_encode``,
``aqmp_decode``, ``aqmp_code_copy``, ``aqmp_code_stats``, ``aqmp_correlate``,
``aqmp_num_atoms``.  Device memory and streams come from PyTorch tensors and
``torch.cuda.current_stream()``; numpy arrays are accepted as host memory.
"""
from __future__ import annotations

import ctypes
import os
import threading
import zlib

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libaqmp.so")

AQMP_OK = 0
ERRORS = {-1: "AQMP_E_ARG", -2: "AQMP_E_SHAPE", -3: "AQMP_E_DICT", -4: "AQMP_E_OOM", -5: "AQMP_E_CUDA",
          -6: "AQMP_E_QUEUE_OVERFLOW", -7: "AQMP_E_TIMEOUT", -8: "AQMP_E_UNSUPPORTED"}
AQMP_DICT_DCT_HAAR, AQMP_DICT_DCT, AQMP_DICT_HAAR = 0, 1, 2
AQMP_PREC_EXACT = 0
AQMP_PREC_FP32 = 1
AQMP_PREC_BF16 = 2
AQMP_PREC_FP8 = 3
AQMP_PREC_BF16_RESCORE = 4
AQMP_FLAG_INPUT_DEVICE = 1
AQMP_FLAG_SIMT_GEMM = 2
AQMP_FLAG_NO_AUTOTUNE = 4
AQMP_FLAG_ALT_THREADS = 8
AQMP_FLAG_OMP = 16
AQMP_LEAF_NEAR_TIE = 1
AQMP_LEAF_NEAR_TIE_PARENT = 2


class AqmpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class aqmp_params(ctypes.Structure):
    _fields_ = [("rmse_tol", ctypes.c_float), ("cap_num", ctypes.c_int32), ("cap_den", ctypes.c_int32),
                ("min_block", ctypes.c_int32), ("max_block", ctypes.c_int32), ("dict_id", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class aqmp_plane(ctypes.Structure):
    _fields_ = [("pixels", ctypes.c_void_p), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("pitch", ctypes.c_int64), ("rmse_tol", ctypes.c_float)]


class aqmp_stats(ctypes.Structure):
    _fields_ = [("n_leaves", ctypes.c_uint64), ("n_atoms", ctypes.c_uint64), ("attempts", ctypes.c_uint64),
                ("atom_iterations", ctypes.c_uint64), ("near_tie_leaves", ctypes.c_uint64),
                ("attempts_per_level", ctypes.c_uint64 * 8), ("iterations_per_level", ctypes.c_uint64 * 8),
                ("window_steps_per_level", ctypes.c_uint64 * 8), ("max_leaf_steps_per_level", ctypes.c_uint64 * 8),
                ("rescored_atoms", ctypes.c_uint64), ("fallback_leaves", ctypes.c_uint64),
                ("rescore_rounds", ctypes.c_uint64)]


LEAF_DTYPE = np.dtype([("plane", np.uint32), ("y", np.uint32), ("x", np.uint32), ("atom_off", np.uint32),
                       ("b", np.uint16), ("n_atoms", np.uint16), ("converged", np.uint8),
                       ("flags", np.uint8), ("reserved", np.uint16)])
ATOM_DTYPE = np.dtype([("j", np.uint32), ("alpha", np.float32)])

# symbols declared in include/aqmp.h
EXPORTS = ["aqmp_params_default", "aqmp_encode_planes", "aqmp_encode", "aqmp_code_stats", "aqmp_code_copy",
           "aqmp_decode", "aqmp_code_free", "aqmp_correlate", "aqmp_num_atoms", "aqmp_last_error",
           "aqmp_version", "aqmp_profile_enable", "aqmp_profile_reset", "aqmp_profile_read",
           "aqmp_correlate_noalloc", "aqmp_selftest_wait", "aqmp_code_device", "aqmp_synth_forward",
           "aqmp_synth_backward", "aqmp_ssim", "aqmp_image_to_planes", "aqmp_planes_to_image",
           "aqmp_bitstream_size", "aqmp_bitstream_write", "aqmp_bitstream_parse", "aqmp_code_from_bitstream",
           "aqmp_autotune_read", "aqmp_autotune_reset", "aqmp_profile_filter", "aqmp_encode_batch",
           "aqmp_correlate_bf16x2", "aqmp_last_device_ms", "aqmp_selftest_round"]


class aqmp_tune_entry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("side", ctypes.c_int), ("dict_id", ctypes.c_int),
                ("precision", ctypes.c_int), ("capacity_log2", ctypes.c_int), ("chosen", ctypes.c_int),
                ("samples", ctypes.c_int * 2), ("best_ms", ctypes.c_double * 2)]

AQMP_COLOR_PLANES, AQMP_COLOR_RGB, AQMP_COLOR_YCBCR = 0, 1, 2
_COLOR_NAMES = {"planes": AQMP_COLOR_PLANES, "gray": AQMP_COLOR_PLANES, "rgb": AQMP_COLOR_RGB,
                "ycbcr": AQMP_COLOR_YCBCR}


class aqmp_bitstream_info(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int), ("color", ctypes.c_int), ("dict_id", ctypes.c_int),
                ("n_planes", ctypes.c_int), ("min_block", ctypes.c_int), ("max_block", ctypes.c_int),
                ("n_leaves", ctypes.c_uint64), ("n_atoms", ctypes.c_uint64)]


class aqmp_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]

_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libaqmp.so (built by ``build_lib``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"libaqmp.so not built at {p}: run `python -m paper_2605_09190_gb300.build_lib`")
        lib = ctypes.CDLL(p)
        V, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.aqmp_params_default.argtypes = [ctypes.POINTER(aqmp_params)]
        lib.aqmp_params_default.restype = None
        lib.aqmp_encode_planes.argtypes = [ctypes.POINTER(aqmp_params), ctypes.POINTER(aqmp_plane), I, V,
                                           ctypes.POINTER(V)]
        lib.aqmp_encode.argtypes = [ctypes.POINTER(aqmp_params), V, I, I, I, ctypes.c_size_t, V, ctypes.POINTER(V)]
        lib.aqmp_encode_batch.argtypes = [ctypes.POINTER(aqmp_params), I, V, V, V, V, V, V, ctypes.POINTER(V)]
        lib.aqmp_code_stats.argtypes = [V, ctypes.POINTER(aqmp_stats)]
        lib.aqmp_code_copy.argtypes = [V, V, V, V]
        lib.aqmp_decode.argtypes = [V, I, V, I64, I, V]
        lib.aqmp_code_free.argtypes = [V]
        lib.aqmp_code_free.restype = None
        lib.aqmp_correlate.argtypes = [I, I, V, I64, V, I, V]
        lib.aqmp_correlate_noalloc.argtypes = [I, I, V, I64, V, V]
        lib.aqmp_correlate_bf16x2.argtypes = [I, I, V, I64, V, V, V]
        lib.aqmp_selftest_wait.argtypes = [I, V]
        U64P = ctypes.POINTER(ctypes.c_uint64)
        lib.aqmp_code_device.argtypes = [V, ctypes.POINTER(V), ctypes.POINTER(V), U64P, U64P]
        lib.aqmp_synth_forward.argtypes = [V, I, V, V, I64, V]
        lib.aqmp_synth_backward.argtypes = [V, I, V, I64, V, V]
        lib.aqmp_ssim.argtypes = [V, V, I, I, I64, V, V, ctypes.c_double, V]
        lib.aqmp_num_atoms.argtypes = [I, I]
        lib.aqmp_last_error.restype = ctypes.c_char_p
        lib.aqmp_last_device_ms.argtypes = [ctypes.POINTER(ctypes.c_double)]
        lib.aqmp_selftest_round.argtypes = [V, I64, V, V]
        lib.aqmp_version.restype = ctypes.c_char_p
        lib.aqmp_profile_enable.argtypes = [I]
        lib.aqmp_profile_reset.argtypes = []
        lib.aqmp_profile_reset.restype = None
        lib.aqmp_profile_read.argtypes = [V, I, ctypes.POINTER(I)]
        lib.aqmp_profile_filter.argtypes = [ctypes.c_char_p]
        lib.aqmp_autotune_read.argtypes = [V, I, ctypes.POINTER(I)]
        lib.aqmp_autotune_reset.argtypes = []
        lib.aqmp_autotune_reset.restype = None
        lib.aqmp_image_to_planes.argtypes = [V, I, I, I, I64, I, V, I64, V]
        lib.aqmp_planes_to_image.argtypes = [V, I, I, I, I64, I, V, I64, V]
        lib.aqmp_bitstream_size.argtypes = [V, U64P]
        lib.aqmp_bitstream_write.argtypes = [V, I, V, ctypes.c_uint64, U64P]
        lib.aqmp_bitstream_parse.argtypes = [V, ctypes.c_uint64, ctypes.POINTER(aqmp_bitstream_info), V, V, V]
        lib.aqmp_code_from_bitstream.argtypes = [V, ctypes.c_uint64, ctypes.POINTER(V)]
        if path is None:
            _lib = lib
        return lib


def _check(rc):
    if rc != AQMP_OK:
        msg = load_library().aqmp_last_error().decode(errors="replace")
        raise AqmpError(rc, msg)


def _stream_handle(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_params(**kw) -> aqmp_params:
    p = aqmp_params()
    load_library().aqmp_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Code:
    """An encode result (library-owned, device resident)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().aqmp_code_free(self._h)
            self._h = ctypes.c_void_p(0)

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        return aqmp_code_stats(self)

    def copy(self):
        return aqmp_code_copy(self)

    def decode(self, plane: int = 0, out=None, stream=None):
        return aqmp_decode(self, plane, out, stream)


def _as_plane(x, tol, device_input):
    if hasattr(x, "data_ptr"):             # torch tensor
        if x.dtype.itemsize != 1 or x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("planes must be 2-D uint8 tensors with unit column stride")
        h, w = x.shape
        ptr, pitch = x.data_ptr(), x.stride(0)
        on_dev = x.is_cuda
    else:
        x = np.ascontiguousarray(x, np.uint8)
        h, w = x.shape
        ptr, pitch, on_dev = x.ctypes.data, x.strides[0], False
    if on_dev != device_input:
        raise ValueError("all planes must be either device (CUDA) tensors or host arrays")
    return aqmp_plane(ptr, h, w, pitch, -1.0 if tol is None else float(tol)), x


def aqmp_encode_planes(planes, tols=None, params: aqmp_params | None = None, stream=None, simt_gemm=False,
                       autotune=True, alt_threads=False, omp=False, **param_kw) -> Code:
    """Encode a list of 2-D uint8 planes (torch CUDA tensors, or host numpy
    arrays / CPU tensors), one optional tolerance per plane."""
    if params is None:
        params = default_params(**param_kw)
    first = planes[0]
    device_input = bool(getattr(first, "is_cuda", False))
    if tols is None or np.isscalar(tols):
        tols = [tols] * len(planes)
    arr = (aqmp_plane * len(planes))()
    keep = []
    for i, (pl, t) in enumerate(zip(planes, tols)):
        arr[i], ref = _as_plane(pl, t, device_input)
        keep.append(ref)
    p = aqmp_params.from_buffer_copy(params)
    p.flags = (p.flags | (AQMP_FLAG_INPUT_DEVICE if device_input else 0)
               | (AQMP_FLAG_SIMT_GEMM if simt_gemm else 0) | (0 if autotune else AQMP_FLAG_NO_AUTOTUNE)
               | (AQMP_FLAG_ALT_THREADS if alt_threads else 0) | (AQMP_FLAG_OMP if omp else 0))
    out = ctypes.c_void_p()
    _check(load_library().aqmp_encode_planes(ctypes.byref(p), arr, len(planes), _stream_handle(stream),
                                             ctypes.byref(out)))
    return Code(out.value)


def aqmp_encode(pixels, params: aqmp_params | None = None, stream=None, **param_kw) -> Code:
    """Encode a (channels, h, w) uint8 stack with the parameters' tolerance."""
    return aqmp_encode_planes([pixels[c] for c in range(pixels.shape[0])], None, params, stream, **param_kw)


def aqmp_encode_batch(images, params: aqmp_params | None = None, stream=None, **param_kw) -> Code:
    """Encode several images at once (Algorithm 1 over a batch): each image a
    (channels, h, w) uint8 CUDA tensor, contiguous; planes are numbered image
    by image and all use the parameters' tolerance."""
    if params is None:
        params = default_params(**param_kw)
    n = len(images)
    ptrs = (ctypes.c_void_p * n)(*[im.data_ptr() for im in images])
    ch = (ctypes.c_int * n)(*[int(im.shape[0]) for im in images])
    hh = (ctypes.c_int * n)(*[int(im.shape[1]) for im in images])
    ww = (ctypes.c_int * n)(*[int(im.shape[2]) for im in images])
    pp = (ctypes.c_size_t * n)(*[int(im.stride(1)) for im in images])
    for im in images:
        if (im.dtype.itemsize != 1 or not im.is_cuda or im.stride(2) != 1
                or (im.shape[0] > 1 and im.stride(0) != im.shape[1] * im.stride(1))):
            raise ValueError("images must be (channels, h, w) uint8 CUDA tensors with stacked rows")
    p = aqmp_params.from_buffer_copy(params)
    p.flags = p.flags | AQMP_FLAG_INPUT_DEVICE
    out = ctypes.c_void_p()
    _check(load_library().aqmp_encode_batch(ctypes.byref(p), n, ptrs, ch, hh, ww, pp, _stream_handle(stream),
                                            ctypes.byref(out)))
    return Code(out.value)


def aqmp_code_stats(code: Code) -> dict:
    s = aqmp_stats()
    _check(load_library().aqmp_code_stats(code.handle, ctypes.byref(s)))
    return {"n_leaves": s.n_leaves, "n_atoms": s.n_atoms, "attempts": s.attempts,
            "atom_iterations": s.atom_iterations, "near_tie_leaves": s.near_tie_leaves,
            "attempts_per_level": list(s.attempts_per_level),
            "iterations_per_level": list(s.iterations_per_level),
            "window_steps_per_level": list(s.window_steps_per_level),
            "max_leaf_steps_per_level": list(s.max_leaf_steps_per_level),
            "rescored_atoms": s.rescored_atoms, "fallback_leaves": s.fallback_leaves,
            "rescore_rounds": s.rescore_rounds}


def _pinned(n: int, dtype) -> np.ndarray:
    """Host array of n elements in page-locked memory from torch's caching
    host allocator (blocks are reused, so a copy into them is plain DMA with
    no page faults); the array keeps its block alive."""
    dt = np.dtype(dtype)
    if n == 0:
        return np.zeros(0, dt)
    try:
        import torch
        buf = torch.empty(n * dt.itemsize, dtype=torch.uint8, pin_memory=True)
    except (ImportError, RuntimeError):          # no driver to pin with: ordinary memory
        return np.empty(n, dt)
    return buf.numpy().view(dt)


def aqmp_code_copy(code: Code):
    """Host copies (leaves, atoms, alpha_lo) in canonical depth-first order,
    in page-locked memory."""
    st = aqmp_code_stats(code)
    leaves = _pinned(st["n_leaves"], LEAF_DTYPE)
    atoms = _pinned(st["n_atoms"], ATOM_DTYPE)
    lo = _pinned(st["n_atoms"], np.float32)
    _check(load_library().aqmp_code_copy(code.handle, leaves.ctypes.data, atoms.ctypes.data, lo.ctypes.data))
    return leaves, atoms, lo


def aqmp_decode(code: Code, plane: int = 0, out=None, stream=None):
    """Decode one plane into `out` (a CUDA float32 tensor, or a new host
    numpy array when `out` is None)."""
    lib = load_library()
    if out is None:
        st = aqmp_code_stats(code)          # noqa: F841 (validates the handle)
        raise ValueError("pass an output buffer (torch CUDA tensor or numpy float32 array)")
    if hasattr(out, "data_ptr"):
        _check(lib.aqmp_decode(code.handle, plane, ctypes.c_void_p(out.data_ptr()), out.stride(0),
                               1 if out.is_cuda else 0, _stream_handle(stream)))
    else:
        if out.dtype != np.float32 or not out.flags.c_contiguous:
            raise ValueError("host output must be a C-contiguous float32 array")
        _check(lib.aqmp_decode(code.handle, plane, ctypes.c_void_p(out.ctypes.data), out.shape[1], 0,
                               _stream_handle(stream)))
    return out


def aqmp_correlate(b: int, dict_id: int, blocks, gemm: int = 0, stream=None):
    """Initial correlations of L contiguous b x b uint8 blocks (a CUDA tensor
    of shape (L, b, b)); returns a CUDA float32 tensor (L, M, 2) of
    double-float pairs."""
    import torch
    L = blocks.shape[0]
    M = aqmp_num_atoms(b, dict_id)
    out = torch.empty((L, M, 2), dtype=torch.float32, device=blocks.device)
    _check(load_library().aqmp_correlate(b, dict_id, ctypes.c_void_p(blocks.data_ptr()), L,
                                         ctypes.c_void_p(out.data_ptr()), gemm, _stream_handle(stream)))
    return out


def aqmp_correlate_bf16x2(b: int, dict_id: int, blocks, stream=None):
    """The BF16 form's initial correlation of L contiguous b x b uint8
    blocks (a CUDA tensor (L, b, b)) and its per-atom error bound: a CUDA
    float32 tensor (L, M, 2) of double-float pairs and one (L, M)."""
    import torch
    L = blocks.shape[0]
    M = aqmp_num_atoms(b, dict_id)
    out = torch.empty((L, M, 2), dtype=torch.float32, device=blocks.device)
    bound = torch.empty((L, M), dtype=torch.float32, device=blocks.device)
    _check(load_library().aqmp_correlate_bf16x2(b, dict_id, ctypes.c_void_p(blocks.data_ptr()), L,
                                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(bound.data_ptr()),
                                                _stream_handle(stream)))
    return out, bound


def aqmp_selftest_round(words, stream=None):
    """int128 -> double-float rounding on the device: `words` is a CUDA int64
    tensor of shape (n, 2), (low, high) words of each integer T; returns a
    CUDA float32 tensor (n, 2) of (RN(T), RN(T - RN(T))) 2^-96."""
    import torch
    words = words.contiguous()
    out = torch.empty((words.shape[0], 2), dtype=torch.float32, device=words.device)
    _check(load_library().aqmp_selftest_round(ctypes.c_void_p(words.data_ptr()), words.shape[0],
                                              ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def aqmp_last_device_ms() -> float:
    """Device time (ms) of the last encode on the current device, from CUDA
    events around its kernels on the stream that ran them (-1: none yet)."""
    ms = ctypes.c_double()
    _check(load_library().aqmp_last_device_ms(ctypes.byref(ms)))
    return ms.value


def aqmp_num_atoms(b: int, dict_id: int) -> int:
    m = load_library().aqmp_num_atoms(b, dict_id)
    if m < 0:
        raise AqmpError(m, "bad side or dictionary")
    return m


def aqmp_version() -> str:
    return load_library().aqmp_version().decode()


def aqmp_profile_enable(on: bool = True) -> bool:
    return bool(load_library().aqmp_profile_enable(1 if on else 0))


def aqmp_profile_reset() -> None:
    load_library().aqmp_profile_reset()


def aqmp_profile_read() -> dict:
    """{kernel name: (launches, total milliseconds)} accumulated so far."""
    arr = (aqmp_kernel_time * 64)()
    n = ctypes.c_int(0)
    _check(load_library().aqmp_profile_read(arr, 64, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


def aqmp_profile_filter(prefix: str | None = None) -> None:
    """Time only kernels whose name starts with `prefix` (None: all)."""
    _check(load_library().aqmp_profile_filter(prefix.encode() if prefix else None))


def aqmp_autotune_read() -> list:
    """The autotuner's choice points on the current device: dicts with kind
    ("corr": 0 tcgen05 / 1 SIMT, "mp": 0 default / 1 alternate launch
    shape), side, dict_id, precision, capacity_log2, chosen (-1 while
    measuring), samples and best_ms per candidate."""
    arr = (aqmp_tune_entry * 64)()
    n = ctypes.c_int(0)
    _check(load_library().aqmp_autotune_read(arr, 64, ctypes.byref(n)))
    return [{"kind": ("corr", "mp")[e.kind], "side": e.side, "dict_id": e.dict_id, "precision": e.precision,
             "capacity_log2": e.capacity_log2, "chosen": e.chosen, "samples": list(e.samples),
             "best_ms": list(e.best_ms)} for e in arr[:min(n.value, 64)]]


def aqmp_autotune_reset() -> None:
    load_library().aqmp_autotune_reset()


def aqmp_selftest_wait(limit_ms: int = 50, stream=None) -> int:
    """Run the bounded-wait check; returns the library's status code
    (AQMP_E_TIMEOUT, -7, is the expected outcome)."""
    return load_library().aqmp_selftest_wait(int(limit_ms), _stream_handle(stream))


def aqmp_code_device(code: Code):
    """(leaf ptr, atom ptr, n_leaves, n_atoms): device arrays in canonical order (as aqmp_code_copy)."""
    lv, at = ctypes.c_void_p(), ctypes.c_void_p()
    nl, na = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load_library().aqmp_code_device(code.handle, ctypes.byref(lv), ctypes.byref(at), ctypes.byref(nl),
                                           ctypes.byref(na)))
    return lv.value, at.value, nl.value, na.value


class _DeviceArray:
    """Zero-copy view of library device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def aqmp_device_atoms(code: Code):
    """The code's atoms in canonical order as new CUDA tensors
    (j: int64, alpha: float32)."""
    import torch
    _, at, _, na = aqmp_code_device(code)
    if na == 0:
        return (torch.zeros(0, dtype=torch.int64, device="cuda"), torch.zeros(0, dtype=torch.float32, device="cuda"))
    raw = torch.as_tensor(_DeviceArray(at, (na, 2), "<i4"), device="cuda").clone()
    return raw[:, 0].to(torch.int64), raw[:, 1].contiguous().view(torch.float32).clone()


def aqmp_device_leaves(code: Code):
    """The code's leaves in canonical order as a host structured array."""
    import torch
    lv, _, nl, _ = aqmp_code_device(code)
    if nl == 0:
        return np.zeros(0, LEAF_DTYPE)
    raw = torch.as_tensor(_DeviceArray(lv, (nl, LEAF_DTYPE.itemsize), "|u1"), device="cuda").cpu().numpy()
    return raw.view(LEAF_DTYPE).reshape(-1)


def aqmp_synth_forward(code: Code, plane: int, alpha, out, stream=None):
    _check(load_library().aqmp_synth_forward(code.handle, plane, ctypes.c_void_p(alpha.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream_handle(stream)))
    return out


def aqmp_synth_backward(code: Code, plane: int, grad_out, grad_alpha, stream=None):
    _check(load_library().aqmp_synth_backward(code.handle, plane, ctypes.c_void_p(grad_out.data_ptr()),
                                              grad_out.stride(0), ctypes.c_void_p(grad_alpha.data_ptr()),
                                              _stream_handle(stream)))
    return grad_alpha


def aqmp_ssim(x, y, ssim_out, grad_y=None, grad_scale: float = 1.0, stream=None):
    """Mean SSIM of y against x (CUDA float32 images) into ssim_out (a CUDA
    float64 scalar tensor); with grad_y, also grad_scale * dSSIM/dy."""
    h, w = x.shape
    _check(load_library().aqmp_ssim(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), h, w, x.stride(0),
                                    ctypes.c_void_p(ssim_out.data_ptr()),
                                    ctypes.c_void_p(grad_y.data_ptr()) if grad_y is not None else None,
                                    float(grad_scale), _stream_handle(stream)))
    return ssim_out


# ---------------------------------------------------------------- codec stages
# Section 2.3: (i) colour conversion, (ii) the encoder above, (iii) DEFLATE of
# the bitstream; the decoder reverses them.

def _color_id(color) -> int:
    return _COLOR_NAMES[color] if isinstance(color, str) else int(color)


def aqmp_image_to_planes(img, color="ycbcr", stream=None):
    """(h, w, C) or (h, w) uint8 CUDA tensor -> (C, h, w) uint8 CUDA planes."""
    import torch
    if img.dim() == 2:
        img = img.unsqueeze(-1)
    if img.dtype != torch.uint8 or not img.is_cuda or not img.is_contiguous():
        raise ValueError("image must be a contiguous uint8 CUDA tensor (h, w[, C])")
    h, w, ch = img.shape
    planes = torch.empty((ch, h, w), dtype=torch.uint8, device=img.device)
    _check(load_library().aqmp_image_to_planes(ctypes.c_void_p(img.data_ptr()), h, w, ch, img.stride(0),
                                               _color_id(color), ctypes.c_void_p(planes.data_ptr()), w,
                                               _stream_handle(stream)))
    return planes


def aqmp_planes_to_image(planes, color="ycbcr", stream=None):
    """(C, h, w) float32 CUDA planes (decoder output) -> (h, w, C) uint8."""
    import torch
    if planes.dtype != torch.float32 or not planes.is_cuda or not planes.is_contiguous() or planes.dim() != 3:
        raise ValueError("planes must be a contiguous (C, h, w) float32 CUDA tensor")
    ch, h, w = planes.shape
    img = torch.empty((h, w, ch), dtype=torch.uint8, device=planes.device)
    _check(load_library().aqmp_planes_to_image(ctypes.c_void_p(planes.data_ptr()), h, w, ch, w, _color_id(color),
                                               ctypes.c_void_p(img.data_ptr()), w * ch, _stream_handle(stream)))
    return img


def aqmp_bitstream(code: Code, color="planes") -> bytes:
    """The serialised MP output (the lossless stage's input)."""
    lib = load_library()
    n = ctypes.c_uint64()
    _check(lib.aqmp_bitstream_size(code.handle, ctypes.byref(n)))
    buf = (ctypes.c_uint8 * max(1, n.value))()
    ln = ctypes.c_uint64()
    _check(lib.aqmp_bitstream_write(code.handle, _color_id(color), buf, n.value, ctypes.byref(ln)))
    return bytes(buf)[:ln.value]


def aqmp_bitstream_parse(data: bytes):
    """Host parse: (info dict, shapes [(h, w)], leaves, atoms), leaves in
    canonical order with positions recovered from the traversal."""
    lib = load_library()
    info = aqmp_bitstream_info()
    _check(lib.aqmp_bitstream_parse(data, len(data), ctypes.byref(info), None, None, None))
    shapes = np.zeros(2 * max(1, info.n_planes), np.int32)
    leaves = np.zeros(info.n_leaves, LEAF_DTYPE)
    atoms = np.zeros(info.n_atoms, ATOM_DTYPE)
    _check(lib.aqmp_bitstream_parse(data, len(data), ctypes.byref(info), shapes.ctypes.data,
                                    leaves.ctypes.data if len(leaves) else None,
                                    atoms.ctypes.data if len(atoms) else None))
    d = {k: getattr(info, k) for k, _ in aqmp_bitstream_info._fields_}
    return d, [(int(shapes[2 * i]), int(shapes[2 * i + 1])) for i in range(info.n_planes)], leaves, atoms


def aqmp_code_from_bitstream(data: bytes) -> Code:
    out = ctypes.c_void_p()
    _check(load_library().aqmp_code_from_bitstream(data, len(data), ctypes.byref(out)))
    return Code(out.value)


def compress(image, tol: float, color="ycbcr", level: int = 9, stream=None, **param_kw) -> bytes:
    """The whole encoder of Section 2.3 / Appendix A: colour conversion,
    AQMP, DEFLATE (zlib container).  `image` is an (h, w, 3) or (h, w)
    uint8 array or CUDA tensor; h and w must be multiples of max_block."""
    import torch
    img = image if hasattr(image, "data_ptr") else torch.from_numpy(np.ascontiguousarray(image))
    img = img.cuda() if not img.is_cuda else img
    if img.dim() == 2:
        color = "planes"
    planes = aqmp_image_to_planes(img.contiguous(), color, stream)
    code = aqmp_encode_planes([planes[c] for c in range(planes.shape[0])], tol, stream=stream, **param_kw)
    try:
        return zlib.compress(aqmp_bitstream(code, color), level)
    finally:
        code.free()


def decompress(blob: bytes, stream=None):
    """Inverse of `compress`: inflate, rebuild the code, decode every plane
    (Algorithm 3), convert back to RGB when the stream says YCbCr.  Returns
    an (h, w, C) uint8 CUDA tensor."""
    import torch
    data = zlib.decompress(blob)
    info, shapes, _, _ = aqmp_bitstream_parse(data)
    if len(set(shapes)) != 1:
        raise ValueError("planes of different sizes do not form one image")
    h, w = shapes[0]
    code = aqmp_code_from_bitstream(data)
    try:
        planes = torch.empty((info["n_planes"], h, w), dtype=torch.float32, device="cuda")
        for c in range(info["n_planes"]):
            aqmp_decode(code, c, planes[c], stream)
        return aqmp_planes_to_image(planes, info["color"], stream)
    finally:
        code.free()


def compression_rate(image, blob: bytes) -> float:
    """CR of Section 3: original size over compressed size, in bytes; the
    original is taken as the raw 8-bit pixels (h w C bytes)."""
    n = int(np.prod(image.shape))
    return n / len(blob)
