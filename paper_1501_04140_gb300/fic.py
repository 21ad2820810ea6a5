"""Thin ctypes binding of libfic.so (include/fic.h), same names as the C ABI.

Argument marshalling only: every step of the encoder runs in the library's
CUDA kernels.  Images may be torch CUDA tensors (device pointers) or host
arrays (numpy / CPU tensors, copied by the library on the call's stream).
There is no fallback: without the built library or a usable sm_103 device the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfic.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fic.h")

FIC_OK = 0
FIC_EINVAL = -1
FIC_ENOMEM = -2
FIC_ECUDA = -3
FIC_ETIMEOUT = -4
FIC_EUNSUPPORTED = -5
FIC_ERANGE = -6

FIC_S_PREDEFINED = 0
FIC_S_GRID = 1
FIC_S_EXACT = 2
FIC_PREC_TENSOR = 0
FIC_PREC_FP32 = 1

FIC_POOL_KEYS = 0
FIC_POOL_KEPT = 1
FIC_POOL_SUMS = 2
FIC_POOL_SQSUMS = 3

# faults of the fic_debug_inject test hook
FIC_FAULT_NONE = 0
FIC_FAULT_DROP_TILE_COPY = 1

# limits of fic_decode_static's fixed workspace
FIC_DECODE_STATIC_MAX_PIXELS = 1024 * 1024
FIC_DECODE_STATIC_MAX_ITERS = 1024


class fic_params(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("range_size0", C.c_int), ("domain_step", C.c_int),
                ("rms_threshold", C.c_double), ("single_level", C.c_int), ("s_mode", C.c_int),
                ("grid_samples", C.c_int), ("entropy_percentile", C.c_double),
                ("precision", C.c_int), ("autotune", C.c_int), ("pool_size", C.c_int)]


class fic_image(C.Structure):
    _fields_ = [("pixels", C.c_void_p), ("width", C.c_int), ("height", C.c_int),
                ("pitch", C.c_int), ("host", C.c_int)]


class fic_transform(C.Structure):
    _fields_ = [("level", C.c_int32), ("x", C.c_int32), ("y", C.c_int32), ("size", C.c_int32),
                ("dom_index", C.c_int32), ("dom_x", C.c_int32), ("dom_y", C.c_int32),
                ("iso", C.c_int32), ("s_idx", C.c_int32), ("p", C.c_int32), ("q", C.c_int32),
                ("reserved", C.c_int32), ("e_num", C.c_int64), ("o_num", C.c_int64),
                ("e", C.c_double), ("s", C.c_double), ("o", C.c_double)]


class fic_level_stats(C.Structure):
    _fields_ = [("size", C.c_int32), ("pool_size", C.c_int32), ("n_kept", C.c_int32),
                ("fallback", C.c_int32), ("thr_key", C.c_int64), ("n_active", C.c_int32),
                ("n_accepted", C.c_int32), ("matches", C.c_double)]


class fic_pool_info_t(C.Structure):
    _fields_ = [("size", C.c_int32), ("step", C.c_int32), ("px", C.c_int32), ("py", C.c_int32),
                ("pool_size", C.c_int32), ("n_kept", C.c_int32), ("fallback", C.c_int32),
                ("reserved", C.c_int32), ("thr_key", C.c_int64)]


TRANSFORM_DTYPE = np.dtype([(n, "<i4") for n in ("level", "x", "y", "size", "dom_index", "dom_x",
                                                  "dom_y", "iso", "s_idx", "p", "q", "reserved")]
                           + [("e_num", "<i8"), ("o_num", "<i8"), ("e", "<f8"), ("s", "<f8"),
                              ("o", "<f8")])
assert TRANSFORM_DTYPE.itemsize == C.sizeof(fic_transform)

_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)

# name -> (restype, argtypes)
_SIGS = {
    "fic_status_string": (C.c_char_p, [C.c_int]),
    "fic_version": (C.c_int, []),
    "fic_default_params": (C.c_int, [C.POINTER(fic_params)]),
    "fic_create": (C.c_int, [_PP, C.c_int]),
    "fic_destroy": (C.c_int, [_P]),
    "fic_build_domain_pool": (C.c_int, [_P, C.POINTER(fic_image), C.c_int, C.POINTER(fic_params),
                                        _P, _PP]),
    "fic_pool_info": (C.c_int, [_P, C.POINTER(fic_pool_info_t)]),
    "fic_pool_copy": (C.c_int, [_P, C.c_int, _P, C.c_size_t]),
    "fic_pool_free": (None, [_P]),
    "fic_match_level": (C.c_int, [_P, C.POINTER(fic_image), _P, _P, C.c_int,
                                  C.POINTER(fic_params), _P, _PP]),
    "fic_matches_copy": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "fic_matches_free": (None, [_P]),
    "fic_encode": (C.c_int, [_P, C.POINTER(fic_image), C.c_int, C.POINTER(fic_params), _P, _PP]),
    "fic_encode_again": (C.c_int, [_P, C.POINTER(fic_image), C.c_int, C.POINTER(fic_params), _P,
                                   _P]),
    "fic_code_count": (C.c_int, [_P, C.c_int, C.POINTER(C.c_size_t)]),
    "fic_code_get": (C.c_int, [_P, C.c_int, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "fic_code_stats": (C.c_int, [_P, C.c_int, C.POINTER(fic_level_stats), C.c_int]),
    "fic_code_quantize_o": (C.c_int, [_P, C.c_int]),
    "fic_code_bits": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int64)]),
    "fic_code_free": (None, [_P]),
    "fic_code_set_profiling": (C.c_int, [_P, C.c_int]),
    "fic_code_profile": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int]),
    "fic_code_graph_kernels": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "fic_code_pool_profile": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int]),
    "fic_code_schedule": (C.c_int, [_P, C.POINTER(C.c_int32), C.c_int]),
    "fic_decode": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_double, _P, C.c_int, C.c_int, _P,
                             C.POINTER(C.c_int)]),
    "fic_decode_static": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_double, _P,
                                    C.c_int, _P, C.POINTER(C.c_int)]),
    "fic_debug_inject": (C.c_int, [_P, C.c_int]),
}

_lib = None


class FicError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def header_functions(path: str = HEADER):
    """Names of the functions include/fic.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fic_[a-z0-9_]+)\s*\(", txt)))


def load(path: str = LIB_PATH):
    """Load libfic.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_1501_04140_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def status_string(s: int) -> str:
    try:
        return load().fic_status_string(s).decode()
    except Exception:  # library not loadable: still name the code
        return str(s)


def _check(rc: int, what: str):
    if rc != FIC_OK:
        raise FicError(rc, what)


def default_params(**kw) -> fic_params:
    p = fic_params()
    _check(load().fic_default_params(C.byref(p)), "fic_default_params")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, int(v) if isinstance(getattr(p, k), int) else float(v))
    return p


def make_image(img) -> tuple[fic_image, object]:
    """fic_image for a 2-D uint8 torch tensor (CUDA: device pointer; CPU:
    host pointer) or numpy array (host).  Returns (descriptor, keep-alive)."""
    try:
        import torch
        if isinstance(img, torch.Tensor):
            if img.dtype != torch.uint8 or img.dim() != 2:
                raise TypeError("image must be a 2-D uint8 tensor")
            if img.stride(1) != 1:
                img = img.contiguous()
            H, W = img.shape
            d = fic_image(img.data_ptr(), W, H, img.stride(0), 0 if img.is_cuda else 1)
            return d, img
    except ImportError:
        pass
    a = np.ascontiguousarray(img, dtype=np.uint8)
    if a.ndim != 2:
        raise TypeError("image must be 2-D")
    H, W = a.shape
    return fic_image(a.ctypes.data, W, H, a.strides[0], 1), a


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def decode_static(codes_dev, n_codes: int, width: int, height: int, out_dev, out_pitch: int,
                  max_iters: int = 300, tol: float = 1e-7, stream=None) -> int:
    """fic_decode_static: decode `n_codes` maps held in device memory at
    `codes_dev` (a pointer or a CUDA tensor) into the device buffer `out_dev`
    without any device allocation.  Returns the iteration count.

    The library runs on the calling thread's current CUDA device and on the
    given stream.  When `codes_dev` is a CUDA tensor the call makes its device
    current for the call and, with no stream given, runs on torch's current
    stream of that device, so work torch queued there (writing the codes or
    the output buffer) is ordered before the decode.  With raw pointers the
    caller sets the device and passes the stream (None: the legacy default
    stream)."""
    it = C.c_int()
    cp = codes_dev.data_ptr() if hasattr(codes_dev, "data_ptr") else codes_dev
    op = out_dev.data_ptr() if hasattr(out_dev, "data_ptr") else out_dev
    dev = getattr(codes_dev, "device", None)
    if dev is not None and getattr(dev, "type", None) == "cuda":
        import torch
        with torch.cuda.device(dev):
            st = stream if stream is not None else torch.cuda.current_stream(dev)
            _check(load().fic_decode_static(cp, n_codes, width, height, max_iters, tol, op,
                                            out_pitch, _stream_ptr(st), C.byref(it)),
                   "fic_decode_static")
        return it.value
    _check(load().fic_decode_static(cp, n_codes, width, height, max_iters, tol, op, out_pitch,
                                    _stream_ptr(stream), C.byref(it)), "fic_decode_static")
    return it.value


class Context:
    """fic_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        _check(load().fic_create(C.byref(self._h), device), "fic_create")
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().fic_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def debug_inject(self, fault: int):
        """fic_debug_inject: arm a fault for the next tensor matcher launch
        (test hook of the bounded device waits)."""
        _check(load().fic_debug_inject(self._h, fault), "fic_debug_inject")

    # ---------------------------------------------------------------- pool
    def build_domain_pool(self, img, range_size: int, params: fic_params, stream=None) -> "Pool":
        d, keep = make_image(img)
        h = C.c_void_p()
        _check(load().fic_build_domain_pool(self._h, C.byref(d), range_size, C.byref(params),
                                            _stream_ptr(stream), C.byref(h)),
               "fic_build_domain_pool")
        return Pool(h, keep)

    # ---------------------------------------------------------------- one level
    def match_level(self, img, pool: "Pool", range_xy, params: fic_params, stream=None):
        d, keep = make_image(img)
        rxy = np.ascontiguousarray(range_xy, dtype=np.int32).reshape(-1, 2)
        h = C.c_void_p()
        _check(load().fic_match_level(self._h, C.byref(d), pool.handle, rxy.ctypes.data, len(rxy),
                                      C.byref(params), _stream_ptr(stream), C.byref(h)),
               "fic_match_level")
        try:
            out = np.zeros(max(len(rxy), 1), TRANSFORM_DTYPE)
            cnt = C.c_size_t()
            _check(load().fic_matches_copy(h, out.ctypes.data, len(out), C.byref(cnt)),
                   "fic_matches_copy")
            return out[:cnt.value].copy()
        finally:
            load().fic_matches_free(h)

    # ---------------------------------------------------------------- encoder
    def encode(self, imgs, params: fic_params, stream=None) -> "Code":
        if not isinstance(imgs, (list, tuple)):
            imgs = [imgs]
        descs, keeps = zip(*(make_image(i) for i in imgs))
        arr = (fic_image * len(descs))(*descs)
        h = C.c_void_p()
        _check(load().fic_encode(self._h, arr, len(descs), C.byref(params), _stream_ptr(stream),
                                 C.byref(h)), "fic_encode")
        return Code(self, h, [(d.width, d.height) for d in descs], list(keeps), params)

    def encode_again(self, code: "Code", imgs, params: fic_params, stream=None):
        if not isinstance(imgs, (list, tuple)):
            imgs = [imgs]
        descs, keeps = zip(*(make_image(i) for i in imgs))
        arr = (fic_image * len(descs))(*descs)
        _check(load().fic_encode_again(self._h, arr, len(descs), C.byref(params),
                                       _stream_ptr(stream), code.handle), "fic_encode_again")
        code._keep = list(keeps)
        return code


class Pool:
    def __init__(self, h, keep):
        self._h = h
        self._keep = keep

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = fic_pool_info_t()
        _check(load().fic_pool_info(self._h, C.byref(i)), "fic_pool_info")
        return {f: getattr(i, f) for f, _ in fic_pool_info_t._fields_}

    def copy(self, field: int) -> np.ndarray:
        info = self.info()
        if field == FIC_POOL_KEYS:
            out = np.zeros(max(info["pool_size"], 1), np.int64)
            n = info["pool_size"]
        elif field == FIC_POOL_KEPT:
            out = np.zeros(max(info["n_kept"], 1), np.int32)
            n = info["n_kept"]
        else:
            out = np.zeros(max(info["n_kept"], 1), np.int64)
            n = info["n_kept"]
        _check(load().fic_pool_copy(self._h, field, out.ctypes.data, out.nbytes), "fic_pool_copy")
        return out[:n].copy()

    def free(self):
        if self._h:
            load().fic_pool_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Code:
    def __init__(self, ctx: Context, h, sizes, keep, params):
        self._ctx = ctx
        self._h = h
        self.sizes = sizes
        self._keep = keep
        self.params = params

    @property
    def handle(self):
        return self._h

    def count(self, image_idx: int = 0) -> int:
        c = C.c_size_t()
        _check(load().fic_code_count(self._h, image_idx, C.byref(c)), "fic_code_count")
        return c.value

    def transforms(self, image_idx: int = 0, out=None) -> np.ndarray:
        """The saved maps of one image (fic_code_get).  With `out` (a 1-D
        TRANSFORM_DTYPE array, e.g. a view of page-locked memory, large enough
        for every map) the maps are copied into it and out[:count] is
        returned; otherwise a new array."""
        n = self.count(image_idx)
        fresh = out is None
        if fresh:
            out = np.zeros(max(n, 1), TRANSFORM_DTYPE)
        elif out.dtype != TRANSFORM_DTYPE or out.ndim != 1 or not out.flags.c_contiguous:
            raise TypeError("out must be a contiguous 1-D TRANSFORM_DTYPE array")
        c = C.c_size_t()
        _check(load().fic_code_get(self._h, image_idx, out.ctypes.data, len(out), C.byref(c)),
               "fic_code_get")
        return out[:c.value].copy() if fresh else out[:c.value]

    def stats(self, image_idx: int = 0) -> list[dict]:
        arr = (fic_level_stats * 4)()
        _check(load().fic_code_stats(self._h, image_idx, arr, 4), "fic_code_stats")
        nl = 1 if self.params.single_level else self.params.n_levels
        return [{f: getattr(arr[i], f) for f, _ in fic_level_stats._fields_} for i in range(nl)]

    def quantize_o(self, o_bits: int = 7):
        """Replace o by its stored form (o_bits bits) in every saved map."""
        _check(load().fic_code_quantize_o(self._h, o_bits), "fic_code_quantize_o")

    def bits(self, image_idx: int = 0, o_bits: int = 7) -> int:
        """Total bits of one image's stored form (8 W H / bits = compression ratio)."""
        b = C.c_int64()
        _check(load().fic_code_bits(self._h, image_idx, o_bits, C.byref(b)), "fic_code_bits")
        return int(b.value)

    def decode(self, image_idx: int = 0, max_iters: int = 300, tol: float = 1e-7, out=None,
               stream=None):
        """Decoded image: into `out` (2-D uint8 tensor/array) or a new host array."""
        W, H = self.sizes[image_idx]
        it = C.c_int()
        if out is None:
            out = np.zeros((H, W), np.uint8)
        d, keep = make_image(out)
        _check(load().fic_decode(self._ctx.handle, self._h, image_idx, max_iters, tol,
                                 d.pixels, d.pitch, d.host, _stream_ptr(stream), C.byref(it)),
               "fic_decode")
        self.iters = it.value
        return out

    def set_profiling(self, on: bool = True):
        _check(load().fic_code_set_profiling(self._h, int(on)), "fic_code_set_profiling")

    def profile(self) -> list[tuple[float, float]]:
        """Per level: (matcher kernel ms, whole level ms) of the last encode."""
        nl = 1 if self.params.single_level else self.params.n_levels
        arr = (C.c_float * (2 * nl))()
        _check(load().fic_code_profile(self._h, arr, 2 * nl), "fic_code_profile")
        return [(arr[2 * i], arr[2 * i + 1]) for i in range(nl)]

    def pool_profile(self) -> list[float]:
        """Per level: ms of the pool build of the last encode (profiling on)."""
        nl = 1 if self.params.single_level else self.params.n_levels
        arr = (C.c_float * nl)()
        _check(load().fic_code_pool_profile(self._h, arr, nl), "fic_code_pool_profile")
        return [arr[i] for i in range(nl)]

    def schedule(self) -> list[tuple[int, int]]:
        """Per level: (work items per CTA, epilogue groups per tile) of the matcher."""
        nl = 1 if self.params.single_level else self.params.n_levels
        arr = (C.c_int32 * (2 * nl))()
        _check(load().fic_code_schedule(self._h, arr, 2 * nl), "fic_code_schedule")
        return [(arr[2 * i], arr[2 * i + 1]) for i in range(nl)]

    def graph_kernels(self) -> int:
        n = C.c_int64()
        _check(load().fic_code_graph_kernels(self._h, C.byref(n)), "fic_code_graph_kernels")
        return n.value

    def free(self):
        if self._h:
            load().fic_code_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
