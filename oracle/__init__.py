"""CPU oracle of the fractal encoder (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import this package.  It wraps ``fic_oracle.c`` (plain C, written from the
paper's definitions: Sec. 2 Eq. 1-3, Sec. 3 Eq. 4-5, Sec. 3.1 S sets) through
ctypes.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

S_PREDEFINED = 0
S_GRID = 1
S_EXACT = 2


def build(force: bool = False) -> str:
    """Compile fic_oracle.c into liboracle.so with gcc (OpenMP when available)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "fic_oracle.h"))):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("range_size0", C.c_int), ("domain_step", C.c_int),
                ("rms_threshold", C.c_double), ("single_level", C.c_int), ("s_mode", C.c_int),
                ("grid_samples", C.c_int), ("entropy_percentile", C.c_double),
                ("n_threads", C.c_int), ("pool_size", C.c_int)]


class Code(C.Structure):
    _fields_ = [("level", C.c_int32), ("x", C.c_int32), ("y", C.c_int32), ("size", C.c_int32),
                ("dom_index", C.c_int32), ("dom_x", C.c_int32), ("dom_y", C.c_int32),
                ("iso", C.c_int32), ("s_idx", C.c_int32), ("p", C.c_int32), ("q", C.c_int32),
                ("pad", C.c_int32), ("e_num", C.c_int64), ("o_num", C.c_int64),
                ("e", C.c_double), ("s", C.c_double), ("o", C.c_double),
                ("s_num", C.c_int64), ("s_den", C.c_int64)]


class MatchResult(C.Structure):
    _fields_ = [("e_num", C.c_int64), ("key", C.c_int64), ("dom_index", C.c_int32),
                ("iso", C.c_int32), ("s_idx", C.c_int32), ("pad", C.c_int32)]


class LevelStats(C.Structure):
    _fields_ = [("size", C.c_int32), ("pool_size", C.c_int32), ("n_kept", C.c_int32),
                ("fallback", C.c_int32), ("thr_key", C.c_int64), ("n_active", C.c_int32),
                ("n_accepted", C.c_int32), ("matches", C.c_double)]


CODE_DTYPE = np.dtype([(n, "<i4") for n in ("level", "x", "y", "size", "dom_index", "dom_x",
                                             "dom_y", "iso", "s_idx", "p", "q", "pad")]
                      + [("e_num", "<i8"), ("o_num", "<i8"), ("e", "<f8"), ("s", "<f8"),
                         ("o", "<f8"), ("s_num", "<i8"), ("s_den", "<i8")])
MATCH_DTYPE = np.dtype([("e_num", "<i8"), ("key", "<i8"), ("dom_index", "<i4"),
                        ("iso", "<i4"), ("s_idx", "<i4"), ("pad", "<i4")])
MATCH_EXACT_DTYPE = np.dtype([("key", "<i8"), ("s_num", "<i8"), ("s_den", "<i8"),
                              ("dom_index", "<i4"), ("iso", "<i4"), ("e", "<f8"),
                              ("e_lo", "<u8"), ("e_hi", "<u8")])

_P = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.oracle_entropy.restype = C.c_double
            L.oracle_entropy.argtypes = [_P, C.c_long, C.c_int, C.c_int, C.c_int]
            L.oracle_entropy_key.restype = C.c_int64
            L.oracle_entropy_key.argtypes = [_P, C.c_long, C.c_int, C.c_int, C.c_int]
            L.oracle_key_table.restype = None
            L.oracle_key_table.argtypes = [_P, C.c_int]
            L.oracle_pool_size.restype = C.c_int
            L.oracle_pool_size.argtypes = [C.c_int] * 4 + [_P, _P]
            L.oracle_pool_filter.restype = C.c_int
            L.oracle_pool_filter.argtypes = [_P, C.c_long, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_double, C.c_int, _P, _P, _P, _P]
            L.oracle_decimate.restype = None
            L.oracle_decimate.argtypes = [_P, C.c_long, C.c_int, C.c_int, C.c_int, _P]
            L.oracle_isometry.restype = None
            L.oracle_isometry.argtypes = [_P, C.c_int, C.c_int, _P]
            L.oracle_error_num.restype = C.c_int64
            L.oracle_error_num.argtypes = [_P, _P, C.c_int, C.c_int, C.c_int]
            L.oracle_error_direct.restype = C.c_double
            L.oracle_error_direct.argtypes = [_P, _P, C.c_int, C.c_int, C.c_int]
            L.oracle_s_set.restype = C.c_int
            L.oracle_s_set.argtypes = [C.c_int, C.c_int, C.c_int, _P, _P]
            L.oracle_match.restype = None
            L.oracle_match.argtypes = [_P, C.c_long, C.c_int, C.c_int, C.c_int, C.c_int, _P,
                                       C.c_int, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int, _P]
            L.oracle_encode.restype = C.c_int
            L.oracle_encode.argtypes = [_P, C.c_long, C.c_int, C.c_int, C.POINTER(Params), _P,
                                        C.c_int, _P]
            L.oracle_decode.restype = C.c_int
            L.oracle_decode.argtypes = [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _P]
            L.oracle_quantize_o.restype = None
            L.oracle_quantize_o.argtypes = [_P, C.c_int, C.c_int]
            L.oracle_map_numerators.restype = None
            L.oracle_map_numerators.argtypes = [_P, C.c_long, C.c_int] + [_P] * 8 + [C.c_int, _P, _P]
            L.oracle_error_num128.restype = None
            L.oracle_error_num128.argtypes = [_P, _P, C.c_int, C.c_int64, C.c_int64, _P]
            L.oracle_s_exact.restype = None
            L.oracle_s_exact.argtypes = [_P, _P, C.c_int, _P, _P]
            L.oracle_mul_u128.restype = None
            L.oracle_mul_u128.argtypes = [C.c_uint64] * 4 + [_P]
            L.oracle_match_exact.restype = None
            L.oracle_match_exact.argtypes = [_P, C.c_long, C.c_int, C.c_int, C.c_int, C.c_int,
                                             _P, C.c_int, _P, C.c_int, C.c_int, _P]
            L.oracle_code_bits.restype = C.c_int64
            L.oracle_code_bits.argtypes = [_P, C.c_int, _P, C.c_int]
            _lib = L
    return _lib


def _u8(img):
    a = np.ascontiguousarray(img, dtype=np.uint8)
    assert a.ndim == 2
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def entropy(img, x, y, size):
    a = _u8(img)
    return lib().oracle_entropy(_ptr(a), a.shape[1], x, y, size)


def entropy_key(img, x, y, size):
    a = _u8(img)
    return int(lib().oracle_entropy_key(_ptr(a), a.shape[1], x, y, size))


def key_table(qmax):
    t = np.zeros(qmax + 1, np.int64)
    lib().oracle_key_table(_ptr(t), qmax)
    return t


def pool_size(W, H, B, L):
    nx, ny = C.c_int(), C.c_int()
    P = lib().oracle_pool_size(W, H, B, L, C.byref(nx), C.byref(ny))
    return P, nx.value, ny.value


def pool_filter(img, B, L, percentile, top_k=0):
    """Returns (keys[P], kept[n_kept], thr_key, fallback); top_k K > 0 keeps
    the K highest entropies (Tables 1-2's pool size) instead of the
    percentile."""
    a = _u8(img)
    H, W = a.shape
    P, _, _ = pool_size(W, H, B, L)
    keys = np.zeros(max(P, 1), np.int64)
    kept = np.zeros(max(P, 1), np.int32)
    thr = C.c_int64()
    fb = C.c_int()
    n = lib().oracle_pool_filter(_ptr(a), W, W, H, B, L, percentile, top_k, _ptr(keys),
                                 _ptr(kept), C.byref(thr), C.byref(fb))
    return keys[:P], kept[:n].copy(), int(thr.value), int(fb.value)


def decimate(img, x, y, B):
    a = _u8(img)
    out = np.zeros(B * B, np.int64)
    lib().oracle_decimate(_ptr(a), a.shape[1], x, y, B, _ptr(out))
    return out.reshape(B, B)


def isometry(block, k):
    b = np.ascontiguousarray(block, dtype=np.int64)
    B = b.shape[0]
    out = np.zeros_like(b)
    lib().oracle_isometry(_ptr(b), B, k, _ptr(out))
    return out


def error_num(R, Ds, p, q):
    r = np.ascontiguousarray(R, dtype=np.int64).ravel()
    d = np.ascontiguousarray(Ds, dtype=np.int64).ravel()
    return int(lib().oracle_error_num(_ptr(r), _ptr(d), r.size, p, q))


def map_numerators(img, maps, n_threads=1):
    """(e_num, o_num) of Eq. 1 / Eq. 3 for each map of `maps` (fields x, y,
    size, dom_x, dom_y, iso, p, q; e.g. an encoder's output), whatever chose
    them."""
    a = _u8(img)
    cols = [np.ascontiguousarray(maps[f], dtype=np.int32)
            for f in ("x", "y", "size", "dom_x", "dom_y", "iso", "p", "q")]
    n = len(cols[0])
    e = np.zeros(max(n, 1), np.int64)
    o = np.zeros(max(n, 1), np.int64)
    lib().oracle_map_numerators(_ptr(a), a.shape[1], n, *[_ptr(c) for c in cols], n_threads,
                                _ptr(e), _ptr(o))
    return e[:n], o[:n]


def error_direct(R, Ds, p, q):
    r = np.ascontiguousarray(R, dtype=np.int64).ravel()
    d = np.ascontiguousarray(Ds, dtype=np.int64).ravel()
    return float(lib().oracle_error_direct(_ptr(r), _ptr(d), r.size, p, q))


def error_num128(R, Ds, p, q):
    """16 q^2 n^2 E of Eq. 1 for 64-bit p, q, as a Python integer."""
    r = np.ascontiguousarray(R, dtype=np.int64).ravel()
    d = np.ascontiguousarray(Ds, dtype=np.int64).ravel()
    out = np.zeros(2, np.uint64)
    lib().oracle_error_num128(_ptr(r), _ptr(d), r.size, int(p), int(q), _ptr(out))
    return int(out[0]) | (int(out[1]) << 64)


def s_exact(R, Ds):
    """Eq. 2's s of the pair, clamped to [0, 1], as (s_num, s_den)."""
    r = np.ascontiguousarray(R, dtype=np.int64).ravel()
    d = np.ascontiguousarray(Ds, dtype=np.int64).ravel()
    sn, sd = C.c_int64(), C.c_int64()
    lib().oracle_s_exact(_ptr(r), _ptr(d), r.size, C.byref(sn), C.byref(sd))
    return int(sn.value), int(sd.value)


def mul_u128(a, b):
    """a * b of two unsigned 128-bit integers, through the oracle's limbs."""
    out = np.zeros(4, np.uint64)
    m = (1 << 64) - 1
    lib().oracle_mul_u128(a & m, a >> 64, b & m, b >> 64, _ptr(out))
    return sum(int(out[i]) << (64 * i) for i in range(4))


def match_exact(img, B, L, kept, range_xy, n_threads=1):
    a = _u8(img)
    H, W = a.shape
    kept = np.ascontiguousarray(kept, dtype=np.int32)
    rxy = np.ascontiguousarray(range_xy, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(max(len(rxy), 1), MATCH_EXACT_DTYPE)
    lib().oracle_match_exact(_ptr(a), W, W, H, B, L, _ptr(kept), len(kept), _ptr(rxy), len(rxy),
                             n_threads, _ptr(out))
    return out[:len(rxy)]


def s_set(s_mode, grid_samples, B):
    p = np.zeros(64, np.int32)
    q = C.c_int32()
    n = lib().oracle_s_set(s_mode, grid_samples, B, _ptr(p), C.byref(q))
    return p[:n].copy(), int(q.value)


def match(img, B, L, kept, range_xy, s_p, q, n_threads=1):
    a = _u8(img)
    H, W = a.shape
    kept = np.ascontiguousarray(kept, dtype=np.int32)
    rxy = np.ascontiguousarray(range_xy, dtype=np.int32).reshape(-1, 2)
    sp = np.ascontiguousarray(s_p, dtype=np.int32)
    out = np.zeros(max(len(rxy), 1), MATCH_DTYPE)
    lib().oracle_match(_ptr(a), W, W, H, B, L, _ptr(kept), len(kept), _ptr(rxy), len(rxy),
                       _ptr(sp), len(sp), q, n_threads, _ptr(out))
    return out[:len(rxy)]


def make_params(n_levels=4, range_size0=16, domain_step=2, rms_threshold=8.0,
                single_level=False, s_mode=S_PREDEFINED, grid_samples=16,
                entropy_percentile=0.5, n_threads=1, pool_size=0):
    return Params(n_levels, range_size0, domain_step, rms_threshold, int(single_level),
                  s_mode, grid_samples, entropy_percentile, n_threads, pool_size)


def encode(img, params: Params):
    """Returns (codes structured array, list of per-level stats dicts)."""
    a = _u8(img)
    H, W = a.shape
    cap = 2 * W * H // 4 + 16
    codes = np.zeros(cap, CODE_DTYPE)
    stats = (LevelStats * 4)()
    n = lib().oracle_encode(_ptr(a), W, W, H, C.byref(params), _ptr(codes), cap, stats)
    if n < 0:
        raise ValueError(f"oracle_encode failed: {n}")
    nl = 1 if params.single_level else params.n_levels
    st = [{f: getattr(stats[i], f) for f, _ in LevelStats._fields_} for i in range(nl)]
    return codes[:n].copy(), st


def decode(codes, W, H, max_iters=300, tol=1e-7):
    c = np.ascontiguousarray(codes, dtype=CODE_DTYPE)
    out = np.zeros(W * H, np.float64)
    it = lib().oracle_decode(_ptr(c), len(c), W, H, max_iters, tol, _ptr(out))
    return out.reshape(H, W), it


def quantize_o(codes, o_bits=7):
    """Copy of the codes with o stored in o_bits bits (the stored form)."""
    c = np.ascontiguousarray(codes, dtype=CODE_DTYPE).copy()
    lib().oracle_quantize_o(_ptr(c), len(c), o_bits)
    return c


def code_bits(stats, s_mode=S_PREDEFINED, grid_samples=16, o_bits=7):
    """Total bits of an encode's stored form, from its per-level stats."""
    n = len(stats)
    st = (LevelStats * n)()
    for i, d in enumerate(stats):
        for f, _ in LevelStats._fields_:
            setattr(st[i], f, d[f])
    ns = (C.c_int * n)(*[len(s_set(s_mode, grid_samples, d["size"])[0]) for d in stats])
    return int(lib().oracle_code_bits(st, n, ns, o_bits))


def compression_ratio(W, H, bits):
    return 8.0 * W * H / bits


def to_u8(img_f64):
    """Round half to even and clamp, as the decoder's final step."""
    return np.clip(np.rint(img_f64), 0, 255).astype(np.uint8)


def psnr(a, b):
    d = a.astype(np.float64) - b.astype(np.float64)
    mse = float(np.mean(d * d))
    if mse == 0.0:
        return float("inf")
    return 10.0 * np.log10(255.0 * 255.0 / mse)
