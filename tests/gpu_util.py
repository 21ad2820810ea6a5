"""Helpers shared by the GPU tests: the CUDA library handle and the oracle
readings the parity checks compare against."""
from __future__ import annotations

import functools

import numpy as np
import pytest

import oracle


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@functools.lru_cache(maxsize=1)
def _built():
    from paper_1501_04140_gb300 import build
    return build.build()


def ctx():
    torch_cuda()
    _built()
    from paper_1501_04140_gb300 import fic
    return _ctx_cached(fic)


_CTX = {}


def _ctx_cached(fic):
    if "c" not in _CTX:
        _CTX["c"] = fic.Context(0)
    return _CTX["c"]


def dev(img):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(img)).cuda()


def params(fic, **kw):
    return fic.default_params(**kw)


def oracle_params(p):
    """Oracle params from a fic_params."""
    return oracle.make_params(n_levels=p.n_levels, range_size0=p.range_size0,
                              domain_step=p.domain_step, rms_threshold=p.rms_threshold,
                              single_level=bool(p.single_level), s_mode=p.s_mode,
                              grid_samples=p.grid_samples,
                              entropy_percentile=p.entropy_percentile, n_threads=8,
                              pool_size=p.pool_size)


def keys_of(m, n_s):
    """Tie-break key of GPU match records: (dom_index * 8 + iso) * |S| + s_idx."""
    return (m["dom_index"].astype(np.int64) * 8 + m["iso"]) * n_s + m["s_idx"]


def fp32_enum_tol(B, p_list, q):
    """Bound on how far the FP32 path's choice can be above the exact minimum,
    in units of e_num = 16 q^2 n^2 E: two FP32 scores, each within
    2^-22 (p^2 U + p Y) score units of exact (see the match kernels), one
    score unit being 8 q n of E' and e_num = n (16 q^2 A + E')."""
    n = B * B
    Y = 131072.0 * n
    U = 260100.0 * n / (8.0 * q)
    pm = max(p_list)
    return 2 * n * 8 * q * n * 2.0 ** -20 * (pm * pm * U + pm * Y)
