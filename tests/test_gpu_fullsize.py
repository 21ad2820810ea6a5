"""GPU parity at the benchmark's sizes: the CUDA path through the C ABI against
the CPU oracle on the workloads the benchmark times.

- 512 x 512 (seed 1, one textured quadrant), quadtree 16 -> 2, L = 2, RMS 8:
  every field of every saved map and every level statistic, and the decoded
  image, for the predefined S sets of Sec. 3.1 at the median and at the 75th
  percentile of the entropy (live oracle encodes), and for the 16-sample
  grid of Sec. 2 (stored oracle encode, written by
  tests/golden/make_oracle_golden.py, re-derived on a sample live); the FP32
  comparison path within its rounding bound and at the oracle's PSNR
  +-0.01 dB.
- The 64-image batch of uneven sizes (256^2 ... 1024^2) in one encode: every
  image's thresholds and kept counts in full, every 256 x 256 member map by
  map, and sampled maps of a 1024 x 1024 and a 768 x 1024 member against the
  oracle's exhaustive search over its own pool.
- 4096 x 4096, L = 1 (the full pool of 16.5 M positions per level): every
  level's threshold key and kept count in full and sampled maps per level
  against the oracle's exhaustive search.
- fic_match_level over every range of a 1024 x 1024 image at B = 8, 4 and 2
  (more ranges than one pass of the range operand kernel's grid-stride loop
  takes), with sampled ranges against the oracle's search.

In the batch, the 4096 x 4096 encode and the every-range matches, every map's
e_num and o_num also equal the oracle's Eq. 1 / Eq. 3 at the map's own range,
domain, isometry and s (oracle.map_numerators).

Bars: integer work bit-exact (keys, thresholds, kept counts, e_num, o_num,
tie-break keys); doubles equal (the same operations in the same order); the
decoded image identical; the FP32 path within the rounding bound of its
scores.
"""
from __future__ import annotations

import concurrent.futures as cf
import functools
import os

import numpy as np
import pytest

import oracle
from paper_1501_04140_gb300.synth import batch_specs, synth_image
from tests import gpu_util as G
from tests.golden import make_oracle_golden as golden

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1
ALL_FIELDS = ("level", "x", "y", "size", "dom_index", "dom_x", "dom_y", "iso", "s_idx", "p", "q",
              "e_num", "o_num", "e", "s", "o")
STAT_FIELDS = ("size", "pool_size", "n_kept", "fallback", "thr_key", "n_active", "n_accepted")


def _fic():
    G.ctx()
    from paper_1501_04140_gb300 import fic
    return fic


def _img512():
    return synth_image(512, 512, 1, n_textured=1)


@functools.lru_cache(maxsize=None)
def _oracle_512(pct: float):
    """The oracle's whole encode of the 512 x 512 headline image (predefined S)."""
    return oracle.encode(_img512(), oracle.make_params(n_threads=NT, entropy_percentile=pct))


def _assert_maps_equal(got, ref, fields=ALL_FIELDS):
    n_ref = len(ref["level"])  # a structured array or a dict of field arrays
    assert len(got) == n_ref, (len(got), n_ref)
    for f in fields:
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)


def _assert_exact_maps(img, t):
    """Every map's e_num and o_num are Eq. 1 / Eq. 3 at its own domain,
    isometry and s (the oracle's arithmetic on the GPU's choices)."""
    e, o = oracle.map_numerators(img, t, n_threads=NT)
    bad = np.nonzero((t["e_num"] != e) | (t["o_num"] != o))[0]
    assert bad.size == 0, (bad.size, len(t), t[bad[:4]], e[bad[:4]], o[bad[:4]])


def _assert_stats_equal(st, rstats):
    assert len(st) == len(rstats)
    for a, b in zip(st, rstats):
        for f in STAT_FIELDS:
            assert a[f] == b[f], (f, a, b)


def _as_oracle_codes(maps):
    """Map records as the oracle's code array (for oracle.decode)."""
    out = np.zeros(len(maps["level"]), oracle.CODE_DTYPE)
    for f in ALL_FIELDS:
        out[f] = maps[f]
    return out


def _match_chunked(img, B, L, kept, rxy, sp, q, chunk=1 << 19, ex=None):
    """oracle.match over the whole kept pool, a bounded slice of the kept list
    at a time (the oracle decimates every kept domain of a call up front: a
    4096^2 pool would hold 17 GB), the slices searched side by side when an
    executor is given; the best of the slices' bests by (exact error,
    tie-break key) is the best over the pool."""
    def one(c0):
        return oracle.match(img, B, L, kept[c0:c0 + chunk], rxy, sp, q, n_threads=NT)

    starts = range(0, len(kept), chunk)
    best = None
    for r in (ex.map(one, starts) if ex is not None else map(one, starts)):
        if best is None:
            best = r
        else:
            better = (r["e_num"] < best["e_num"]) | ((r["e_num"] == best["e_num"])
                                                     & (r["key"] < best["key"]))
            best = np.where(better, r, best)
    return best


def _check_sampled_maps(img, t, lv, B, L, kept, n, rng, smode=0, M=16, ex=None):
    """n saved maps of level lv re-derived by the oracle's exhaustive search
    over the level's kept pool: the exact error and the tie-break key equal."""
    rows = t[t["level"] == lv]
    if len(rows) == 0:
        return 0
    pick = rows[rng.choice(len(rows), size=min(n, len(rows)), replace=False)]
    sp, q = oracle.s_set(smode, M, B)
    rxy = np.stack([pick["x"], pick["y"]], 1).astype(np.int32)
    ref = _match_chunked(img, B, L, kept, rxy, sp, q, ex=ex)
    np.testing.assert_array_equal(pick["e_num"], ref["e_num"])
    np.testing.assert_array_equal(G.keys_of(pick, len(sp)), ref["key"])
    return len(pick)


# ------------------------------------------------------------------ 512 x 512
@pytest.mark.parametrize("pct", [0.5, 0.75])
def test_512_every_map_predefined_s(pct):
    """The headline encode (median) and the 75th-percentile threshold: every
    field of every map, every level statistic, the decoded image and its
    iteration count equal the oracle's."""
    fic = _fic()
    ctx = G.ctx()
    img = _img512()
    code = ctx.encode(G.dev(img), fic.default_params(entropy_percentile=pct))
    got = code.transforms(0)
    ref, rstats = _oracle_512(pct)
    _assert_maps_equal(got, ref)
    _assert_stats_equal(code.stats(0), rstats)
    dec = code.decode(0)
    ref_f, it = oracle.decode(ref, 512, 512)
    np.testing.assert_array_equal(dec, oracle.to_u8(ref_f))
    assert code.iters == it
    assert abs(oracle.psnr(img, dec) - oracle.psnr(img, oracle.to_u8(ref_f))) <= 0.01
    code.free()


def test_512_every_map_grid16_stored_oracle():
    """The 16-sample s grid (s = k / 15): every map and statistic against the
    stored oracle encode, the decoded image against the oracle's decoder on
    those maps, and 8 maps per level re-derived by a live oracle search (a
    stored file that no longer matches the oracle fails here)."""
    fic = _fic()
    ctx = G.ctx()
    name = "enc512_grid16"
    img = golden.case_image(name)
    maps, rstats = golden.load(name)
    code = ctx.encode(G.dev(img), fic.default_params(s_mode=fic.FIC_S_GRID, grid_samples=16))
    got = code.transforms(0)
    _assert_maps_equal(got, maps)
    _assert_stats_equal(code.stats(0), rstats)
    dec = code.decode(0)
    ref_f, it = oracle.decode(_as_oracle_codes(maps), 512, 512)
    np.testing.assert_array_equal(dec, oracle.to_u8(ref_f))
    assert code.iters == it
    rng = np.random.default_rng(5)
    for lv in range(4):
        B = 16 >> lv
        _, kept, thr, _ = oracle.pool_filter(img, B, 2, 0.5)
        assert thr == rstats[lv]["thr_key"] and len(kept) == rstats[lv]["n_kept"]
        _check_sampled_maps(img, got, lv, B, 2, kept, 8, rng, smode=1, M=16)
    code.free()


def test_512_fp32_path_within_bound_and_psnr():
    """The plain FP32 path on the headline: the same pools; on every range
    both encoders saved, the FP32 choice's exact error is at or above the
    exact minimum and within the FP32 scores' rounding bound; the decoded
    PSNR within 0.01 dB of the oracle's."""
    fic = _fic()
    ctx = G.ctx()
    img = _img512()
    code = ctx.encode(G.dev(img), fic.default_params(precision=fic.FIC_PREC_FP32))
    got = code.transforms(0)
    ref, rstats = _oracle_512(0.5)
    st = code.stats(0)
    for a, b in zip(st, rstats):
        assert (a["thr_key"], a["n_kept"], a["pool_size"]) == (b["thr_key"], b["n_kept"],
                                                                b["pool_size"])
    common = 0
    for lv in range(4):
        B = 16 >> lv
        sp, q = oracle.s_set(0, 16, B)
        tol = G.fp32_enum_tol(B, sp, q)
        g = got[got["level"] == lv]
        r = ref[ref["level"] == lv]
        gi = {(int(x), int(y)): e for x, y, e in zip(g["x"], g["y"], g["e_num"])}
        for x, y, e in zip(r["x"], r["y"], r["e_num"]):
            if (int(x), int(y)) in gi:
                d = int(gi[(int(x), int(y))]) - int(e)
                assert 0 <= d <= tol, (lv, x, y, d, tol)
                common += 1
    assert common >= 0.95 * len(ref)
    ref_f, _ = oracle.decode(ref, 512, 512)
    a = oracle.psnr(img, code.decode(0))
    b = oracle.psnr(img, oracle.to_u8(ref_f))
    assert abs(a - b) <= 0.01, (a, b)
    code.free()


# ------------------------------------------------------------------ batch
def _batch64():
    return [(W, H, sd, synth_image(W, H, sd, n_textured=1))
            for (W, H, sd) in batch_specs(64, 1000, 42)]


def test_batch64_uneven_sizes():
    """The 64-image uneven batch in one encode: every image's per-level
    threshold and kept count equal the oracle's pool filter; every 256 x 256
    member's maps and statistics equal the oracle's encode; 24 maps per level
    of a 1024 x 1024 and of a 768 x 1024 member re-derived by the oracle's
    exhaustive search over that image's pool."""
    fic = _fic()
    ctx = G.ctx()
    batch = _batch64()
    p = fic.default_params()
    code = ctx.encode([G.dev(im) for (_, _, _, im) in batch], p)
    stats = [code.stats(i) for i in range(len(batch))]
    for i, (_, _, _, im) in enumerate(batch):
        _assert_exact_maps(im, code.transforms(i))

    def pool_of(args):
        i, lv = args
        im = batch[i][3]
        _, kept, thr, fb = oracle.pool_filter(im, 16 >> lv, 2, 0.5)
        return i, lv, kept, thr, fb

    jobs = [(i, lv) for i in range(len(batch)) for lv in range(4)]
    pools = {}
    with cf.ThreadPoolExecutor(max_workers=NT) as ex:
        for i, lv, kept, thr, fb in ex.map(pool_of, jobs):
            s = stats[i][lv]
            assert (s["thr_key"], s["n_kept"], s["fallback"]) == (thr, len(kept), fb), (i, lv)
            pools[(i, lv)] = kept
    small = [i for i, (W, H, _, _) in enumerate(batch) if (W, H) == (256, 256)]
    assert small
    for i in small:
        ref, rstats = oracle.encode(batch[i][3], G.oracle_params(p))
        _assert_maps_equal(code.transforms(i), ref)
        _assert_stats_equal(stats[i], rstats)
    rng = np.random.default_rng(7)
    for size in ((1024, 1024), (768, 1024)):
        i = next(k for k, (W, H, _, _) in enumerate(batch) if (W, H) == size)
        t = code.transforms(i)
        for lv in range(4):
            _check_sampled_maps(batch[i][3], t, lv, 16 >> lv, 2, pools[(i, lv)], 24, rng)
    code.free()


# ------------------------------------------------------------------ many ranges
@pytest.mark.parametrize("B", [8, 4, 2])
def test_match_level_more_ranges_than_one_pass(B):
    """fic_match_level over every range of a 1024 x 1024 image (16 384,
    65 536 and 262 144 ranges: more than the range operand kernel's blocks
    take in one pass of their grid-stride loop): every range's exact map
    (Eq. 1 / Eq. 3 at its chosen domain, isometry and s), and the best E of
    sampled ranges equal the oracle's exhaustive search."""
    fic = _fic()
    ctx = G.ctx()
    img = synth_image(1024, 1024, 77, n_textured=2)
    p = fic.default_params()
    d = G.dev(img)
    pool = ctx.build_domain_pool(d, B, p)
    rxy = np.array([(x, y) for y in range(0, 1024, B) for x in range(0, 1024, B)], np.int32)
    got = ctx.match_level(d, pool, rxy, p)
    pool.free()
    assert len(got) == len(rxy)
    _assert_exact_maps(img, got)
    rng = np.random.default_rng(5 + B)
    pick = np.sort(rng.choice(len(rxy), 24, replace=False))
    _, kept, _, _ = oracle.pool_filter(img, B, 2, 0.5)
    sp, q = oracle.s_set(0, 16, B)
    ref = oracle.match(img, B, 2, kept, rxy[pick], sp, q, n_threads=NT)
    np.testing.assert_array_equal(got["e_num"][pick], ref["e_num"])
    np.testing.assert_array_equal(G.keys_of(got[pick], len(sp)), ref["key"])


# ------------------------------------------------------------------ 4096 x 4096
def test_4096_full_pool_sampled():
    """4096 x 4096 with L = 1: per level the threshold key and the kept count
    of the full 16.5 M-position pool equal the oracle's, and saved maps of
    every level re-derived by the oracle's exhaustive search over the level's
    7-8 M kept domains (6 maps at B = 16 and 8, 16 at B = 4 and 2; the
    oracle's pool filters and searches of the four levels run side by
    side)."""
    fic = _fic()
    ctx = G.ctx()
    img = synth_image(4096, 4096, 1, n_textured=8)
    code = ctx.encode(G.dev(img), fic.default_params(domain_step=1))
    t = code.transforms(0)
    st = code.stats(0)
    code.free()
    _assert_exact_maps(img, t)
    n_pick = {0: 6, 1: 6, 2: 16, 3: 16}

    def pool(lv):
        return oracle.pool_filter(img, 16 >> lv, 1, 0.5)

    # the four pool filters side by side, then each level's search with its
    # domain slices side by side (8 at a time: a slice holds up to 1 GB)
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        pools = list(ex.map(pool, range(4)))
    checked = []
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        for lv, (_, kept, thr, fb) in enumerate(pools):
            B = 16 >> lv
            assert st[lv]["pool_size"] == oracle.pool_size(4096, 4096, B, 1)[0]
            assert (st[lv]["thr_key"], st[lv]["n_kept"], st[lv]["fallback"]) == (thr, len(kept),
                                                                                  fb)
            checked.append(_check_sampled_maps(img, t, lv, B, 1, kept, n_pick[lv],
                                               np.random.default_rng(11 + lv), ex=ex))
    assert all(c > 0 for c in checked), checked
