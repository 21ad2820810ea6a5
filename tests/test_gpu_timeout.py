"""The bounded device waits of the tensor matcher, driven to their limit.

A fault armed from the host (fic_debug_inject) makes the matcher's producer
leave one stage of shared memory unfilled; nothing else is wrong and the GPU
is never faulted.  The waits on that stage give up after their limit (2 s),
the kernel abandons its work and returns, and the handle reports
FIC_ETIMEOUT.  The context and the handle stay usable: the next encode, into
a new handle or into the same one, equals the oracle's again.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from paper_1501_04140_gb300.synth import synth_image
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def _fic():
    G.ctx()
    from paper_1501_04140_gb300 import fic
    return fic


@pytest.mark.parametrize("B0", [16, 8])
def test_encode_wait_runs_out_then_recovers(B0):
    fic = _fic()
    ctx = fic.Context(0)
    img = synth_image(128, 96, 90 + B0, n_textured=1)
    p = fic.default_params(range_size0=B0, n_levels=4 if B0 == 16 else 3)
    ref, _ = oracle.encode(img, G.oracle_params(p))
    d = G.dev(img)

    ctx.debug_inject(fic.FIC_FAULT_DROP_TILE_COPY)
    t0 = time.monotonic()
    code = ctx.encode(d, p)
    with pytest.raises(fic.FicError) as e:
        code.transforms(0)
    assert e.value.status == fic.FIC_ETIMEOUT
    assert time.monotonic() - t0 < 60.0  # every wait ended

    # the same handle, re-encoded: a clear status and the oracle's maps
    ctx.encode_again(code, d, p)
    got = code.transforms(0)
    np.testing.assert_array_equal(got["e_num"], ref["e_num"])
    np.testing.assert_array_equal(got["dom_index"], ref["dom_index"])
    np.testing.assert_array_equal(got["iso"], ref["iso"])
    code.free()

    # and a new handle on the same context
    code2 = ctx.encode(d, p)
    got2 = code2.transforms(0)
    for f in ("level", "x", "y", "dom_index", "iso", "s_idx", "e_num", "o_num"):
        np.testing.assert_array_equal(got2[f], ref[f], err_msg=f)
    code2.free()
    ctx.close()


def test_match_level_wait_runs_out_then_recovers():
    fic = _fic()
    ctx = fic.Context(0)
    img = synth_image(96, 96, 95, n_textured=1)
    p = fic.default_params()
    d = G.dev(img)
    pool = ctx.build_domain_pool(d, 8, p)
    rxy = np.array([(x, y) for y in range(0, 96, 8) for x in range(0, 96, 8)], np.int32)
    ctx.debug_inject(fic.FIC_FAULT_DROP_TILE_COPY)
    with pytest.raises(fic.FicError) as e:
        ctx.match_level(d, pool, rxy, p)
    assert e.value.status == fic.FIC_ETIMEOUT
    # the pool is intact and the next match is exact
    got = ctx.match_level(d, pool, rxy, p)
    _, kept, _, _ = oracle.pool_filter(img, 8, 2, 0.5)
    sp, q = oracle.s_set(0, 16, 8)
    ref = oracle.match(img, 8, 2, kept, rxy, sp, q, n_threads=8)
    np.testing.assert_array_equal(got["e_num"], ref["e_num"])
    np.testing.assert_array_equal(G.keys_of(got, len(sp)), ref["key"])
    pool.free()
    ctx.close()


def test_inject_rejects_unknown_fault():
    fic = _fic()
    ctx = fic.Context(0)
    with pytest.raises(fic.FicError) as e:
        ctx.debug_inject(7)
    assert e.value.status == fic.FIC_EINVAL
    ctx.debug_inject(fic.FIC_FAULT_NONE)
    ctx.close()
