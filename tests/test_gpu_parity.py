"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars (from the method's arithmetic): integer work (entropy keys, kept lists,
moments, the exact tensor path's chosen error numerators and tie-break keys)
bit-exact; the FP32 path's choice within its derived rounding bound; decoded
images identical (same FP64 operation order) or PSNR within 0.01 dB.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_1501_04140_gb300.synth import synth_image
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

PREC = {"tensor": 0, "fp32": 1}


def _fic():
    G.ctx()
    from paper_1501_04140_gb300 import fic
    return fic


def _ramp(W, H):
    x = np.arange(W)[None, :].repeat(H, 0)
    return (x % 256).astype(np.uint8)


def _flat(W, H, v=77):
    return np.full((H, W), v, np.uint8)


POOL_CASES = [
    # (image, B, L, percentile)
    (lambda: synth_image(64, 64, 3), 8, 2, 0.5),
    (lambda: synth_image(96, 64, 4, n_textured=1), 16, 1, 0.75),
    (lambda: synth_image(128, 128, 1), 8, 4, 0.5),
    (lambda: synth_image(40, 32, 6), 2, 2, 0.5),
    (lambda: synth_image(48, 32, 7), 4, 3, 0.25),
    (lambda: _flat(32, 32), 8, 2, 0.5),
    (lambda: synth_image(64, 64, 8), 16, 2, 1.0),
    (lambda: synth_image(64, 64, 8), 16, 2, 0.0),
]


@pytest.mark.parametrize("case", range(len(POOL_CASES)))
@pytest.mark.parametrize("prec", ["tensor", "fp32"])
def test_pool_parity(case, prec):
    fic = _fic()
    mk, B, L, pct = POOL_CASES[case]
    img = mk()
    ctx = G.ctx()
    p = fic.default_params(domain_step=L, entropy_percentile=pct, precision=PREC[prec])
    pool = ctx.build_domain_pool(G.dev(img), B, p)
    info = pool.info()
    keys_o, kept_o, thr_o, fb_o = oracle.pool_filter(img, B, L, pct)
    P, px, py = oracle.pool_size(img.shape[1], img.shape[0], B, L)
    assert info["pool_size"] == P and info["px"] == px and info["py"] == py
    np.testing.assert_array_equal(pool.copy(fic.FIC_POOL_KEYS), keys_o)
    assert info["thr_key"] == thr_o
    assert info["fallback"] == fb_o
    kept = pool.copy(fic.FIC_POOL_KEPT)
    np.testing.assert_array_equal(kept, kept_o)
    sums = pool.copy(fic.FIC_POOL_SUMS)
    sq = pool.copy(fic.FIC_POOL_SQSUMS)
    for j in range(0, len(kept_o), max(1, len(kept_o) // 50)):
        d = int(kept_o[j])
        Ds = oracle.decimate(img, (d % px) * L, (d // px) * L, B)
        assert sums[j] == Ds.sum()
        assert sq[j] == (Ds * Ds).sum()
    pool.free()


@pytest.mark.parametrize("B,L,K", [(8, 2, 32), (4, 1, 256), (16, 2, 1), (2, 2, 10 ** 6),
                                   (8, 3, 100)])
def test_pool_parity_pool_size(B, L, K):
    """Tables 1-2's pool size: the K highest entropies, bit-exact with the
    oracle (K >= P keeps the whole pool)."""
    fic = _fic()
    ctx = G.ctx()
    img = synth_image(96, 64, 12, n_textured=1)
    p = fic.default_params(domain_step=L, pool_size=K)
    pool = ctx.build_domain_pool(G.dev(img), B, p)
    info = pool.info()
    keys_o, kept_o, thr_o, fb_o = oracle.pool_filter(img, B, L, 0.5, top_k=K)
    np.testing.assert_array_equal(pool.copy(fic.FIC_POOL_KEYS), keys_o)
    assert info["thr_key"] == thr_o and info["fallback"] == fb_o
    np.testing.assert_array_equal(pool.copy(fic.FIC_POOL_KEPT), kept_o)
    pool.free()


MATCH_CASES = [
    # (W, H, seed, B, L, s_mode, grid, n_ranges or None (all))
    (64, 64, 5, 8, 2, 0, 16, None),
    (64, 64, 5, 8, 1, 0, 16, 37),
    (96, 96, 9, 16, 2, 0, 16, None),
    (64, 48, 10, 4, 2, 0, 16, 150),
    (32, 32, 11, 2, 1, 0, 16, 200),
    (64, 64, 12, 8, 2, 1, 16, None),
    (64, 64, 13, 8, 3, 1, 32, 50),
    (96, 64, 14, 16, 1, 1, 16, 20),
    (48, 48, 15, 2, 2, 1, 10, 120),
    (64, 64, 16, 4, 1, 1, 16, 90),
    # many domain tiles per work item and many items per range tile: the
    # thresholds shared between isometry rows, warp pairs and CTAs
    (256, 256, 31, 4, 1, 0, 16, 300),
    (256, 192, 32, 8, 1, 1, 16, 60),
    (256, 256, 33, 16, 2, 0, 16, None),
    (320, 160, 34, 2, 1, 0, 16, 500),
    (256, 256, 35, 16, 1, 1, 32, 12),
]


def _ranges(W, H, B, n, seed):
    xy = np.array([(x, y) for y in range(0, H - B + 1, B) for x in range(0, W - B + 1, B)],
                  np.int32)
    if n is None or n >= len(xy):
        return xy
    rng = np.random.default_rng(seed)
    # arbitrary positions too (not only the range grid)
    out = []
    for i in range(n):
        if i % 3 == 0:
            out.append((rng.integers(0, W - B + 1), rng.integers(0, H - B + 1)))
        else:
            out.append(tuple(xy[rng.integers(0, len(xy))]))
    return np.array(out, np.int32)


@pytest.mark.parametrize("case", range(len(MATCH_CASES)))
@pytest.mark.parametrize("prec", ["tensor", "fp32"])
def test_match_level_parity(case, prec):
    fic = _fic()
    W, H, seed, B, L, smode, M, nr = MATCH_CASES[case]
    img = synth_image(W, H, seed, n_textured=1)
    ctx = G.ctx()
    p = fic.default_params(domain_step=L, s_mode=smode, grid_samples=M, precision=PREC[prec])
    d = G.dev(img)
    pool = ctx.build_domain_pool(d, B, p)
    rxy = _ranges(W, H, B, nr, seed)
    got = ctx.match_level(d, pool, rxy, p)
    pool.free()
    _, kept, _, _ = oracle.pool_filter(img, B, L, 0.5)
    sp, q = oracle.s_set(smode, M, B)
    ref = oracle.match(img, B, L, kept, rxy, sp, q, n_threads=8)
    assert len(got) == len(ref)
    n_s = len(sp)
    if prec == "tensor":
        np.testing.assert_array_equal(got["e_num"], ref["e_num"])
        np.testing.assert_array_equal(G.keys_of(got, n_s), ref["key"])
    else:
        tol = G.fp32_enum_tol(B, sp, q)
        assert np.all(got["e_num"] >= ref["e_num"])
        assert np.all(got["e_num"] - ref["e_num"] <= tol), (got["e_num"] - ref["e_num"]).max()
    # the exact map of the chosen candidate (Eq. 1, Eq. 3) for every range
    n = B * B
    for i in range(0, len(got), max(1, len(got) // 20)):
        g = got[i]
        R = img[g["y"]:g["y"] + B, g["x"]:g["x"] + B].astype(np.int64)
        Ds = oracle.isometry(oracle.decimate(img, g["dom_x"], g["dom_y"], B), g["iso"])
        assert g["e_num"] == oracle.error_num(R, Ds, int(g["p"]), int(g["q"]))
        assert g["o_num"] == 4 * g["q"] * R.sum() - g["p"] * Ds.sum()
        assert g["e"] == g["e_num"] / (16.0 * g["q"] * g["q"] * n * n)


def _extreme_image(name):
    rng = np.random.default_rng(71)
    if name == "black":
        return np.zeros((96, 96), np.uint8)
    if name == "sparse_white":
        img = np.zeros((128, 128), np.uint8)
        img[rng.random((128, 128)) < 0.03] = 255
        return img
    return ((rng.random((128, 128)) < 0.5) * 255).astype(np.uint8)  # "binary"


@pytest.mark.parametrize("name", ["black", "sparse_white", "binary"])
@pytest.mark.parametrize("smode", [0, 1])
def test_match_level_b16_correlations_at_the_bound(name, smode):
    """B = 16 accumulates the whole K = 256 in one f32 accumulator: every
    partial sum is an integer of magnitude at most 256 * 128 * 512 = 2^24.
    Black ranges against black domains (the black image keeps every domain:
    the entropy filter's fallback) reach exactly 2^24, sparse white pixels
    stay just below it, random 0/255 pixels mix large terms of both signs;
    the best E and key of every range equal the oracle's."""
    fic = _fic()
    img = _extreme_image(name)
    H, W = img.shape
    ctx = G.ctx()
    p = fic.default_params(s_mode=smode, grid_samples=16)
    d = G.dev(img)
    pool = ctx.build_domain_pool(d, 16, p)
    rxy = np.array([(x, y) for y in range(0, H, 16) for x in range(0, W, 16)], np.int32)
    got = ctx.match_level(d, pool, rxy, p)
    pool.free()
    _, kept, _, _ = oracle.pool_filter(img, 16, 2, 0.5)
    sp, q = oracle.s_set(smode, 16, 16)
    ref = oracle.match(img, 16, 2, kept, rxy, sp, q, n_threads=8)
    np.testing.assert_array_equal(got["e_num"], ref["e_num"])
    np.testing.assert_array_equal(G.keys_of(got, len(sp)), ref["key"])


ENC_CASES = [
    # (W, H, seed, textured, params)
    (96, 96, 21, 1, dict()),
    (64, 96, 22, 1, dict(s_mode=1, grid_samples=16)),
    (64, 64, 23, 0, dict(range_size0=8, n_levels=3, domain_step=1)),
    (128, 128, 1, 0, dict(range_size0=8, n_levels=1, single_level=1, domain_step=4, s_mode=1,
                          grid_samples=16)),
    (48, 80, 24, 1, dict(entropy_percentile=0.75, rms_threshold=5.0)),
    (64, 64, 25, 1, dict(range_size0=4, n_levels=2, domain_step=2, rms_threshold=3.0)),
    (96, 96, 26, 1, dict(pool_size=64)),
    (64, 64, 27, 1, dict(pool_size=32, s_mode=1, grid_samples=10)),
    # exact s (Eq. 2 per pair, clamped to [0, 1])
    (96, 96, 28, 1, dict(s_mode=2)),
    (64, 64, 29, 1, dict(s_mode=2, range_size0=8, n_levels=3, domain_step=1)),
    (64, 96, 30, 0, dict(s_mode=2, rms_threshold=4.0, entropy_percentile=0.25)),
]


def _enc_params(fic, prec, kw):
    p = fic.default_params(precision=PREC[prec])
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("case", range(len(ENC_CASES)))
def test_encode_parity_tensor(case):
    fic = _fic()
    W, H, seed, tex, kw = ENC_CASES[case]
    img = synth_image(W, H, seed, n_textured=tex)
    ctx = G.ctx()
    p = _enc_params(fic, "tensor", kw)
    code = ctx.encode(G.dev(img), p)
    got = code.transforms(0)
    ref, rstats = oracle.encode(img, G.oracle_params(p))
    assert len(got) == len(ref)
    for f in ("level", "x", "y", "size", "dom_index", "dom_x", "dom_y", "iso", "s_idx", "p", "q",
              "e_num", "o_num", "e", "s", "o"):
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
    st = code.stats(0)
    for a, b in zip(st, rstats):
        for f in ("size", "pool_size", "n_kept", "fallback", "thr_key", "n_active", "n_accepted"):
            assert a[f] == b[f], (f, a, b)
    # decoder: identical iterate to the oracle's on the same codes
    dec = code.decode(0)
    ref_f, it = oracle.decode(ref, W, H)
    np.testing.assert_array_equal(dec, oracle.to_u8(ref_f))
    assert code.iters == it
    code.free()


def test_encode_exact_s_ramp_and_errors():
    """Exact s on the GPU: the ramp f(x, y) = x is exact at the first level
    (s = 1/2, E = 0, as the oracle); FP32 precision is refused and the stored
    form's bit count is undefined for it."""
    fic = _fic()
    ctx = G.ctx()
    img = np.tile(np.arange(64, dtype=np.uint8), (64, 1))
    p = _enc_params(fic, "tensor", dict(s_mode=2, rms_threshold=0.0))
    code = ctx.encode(G.dev(img), p)
    got = code.transforms(0)
    ref, _ = oracle.encode(img, G.oracle_params(p))
    assert len(got) == len(ref) == 16
    assert np.all(got["e"] == 0.0) and np.all(got["s"] == 0.5)
    for f in ("dom_index", "iso", "s", "o", "e"):
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
    np.testing.assert_array_equal(code.decode(0), img)
    with pytest.raises(fic.FicError) as e:
        code.bits(0, 7)
    assert e.value.status == fic.FIC_EINVAL
    code.free()
    with pytest.raises(fic.FicError) as e:
        ctx.encode(G.dev(img), _enc_params(fic, "fp32", dict(s_mode=2)))
    assert e.value.status == fic.FIC_EUNSUPPORTED


@pytest.mark.parametrize("case", [0, 1, 4])
def test_encode_fp32_psnr(case):
    fic = _fic()
    W, H, seed, tex, kw = ENC_CASES[case]
    img = synth_image(W, H, seed, n_textured=tex)
    ctx = G.ctx()
    p = _enc_params(fic, "fp32", kw)
    code = ctx.encode(G.dev(img), p)
    dec = code.decode(0)
    ref, _ = oracle.encode(img, G.oracle_params(p))
    ref_f, _ = oracle.decode(ref, W, H)
    a = oracle.psnr(img, dec)
    b = oracle.psnr(img, oracle.to_u8(ref_f))
    assert abs(a - b) <= 0.01, (a, b)
    code.free()


def test_encode_batch_uneven_sizes():
    fic = _fic()
    ctx = G.ctx()
    sizes = [(64, 64), (96, 48), (32, 32), (128, 64)]
    imgs = [synth_image(W, H, 40 + i, n_textured=1) for i, (W, H) in enumerate(sizes)]
    p = fic.default_params()
    code = ctx.encode([G.dev(im) for im in imgs], p)
    for i, im in enumerate(imgs):
        got = code.transforms(i)
        ref, rstats = oracle.encode(im, G.oracle_params(p))
        np.testing.assert_array_equal(got["e_num"], ref["e_num"])
        np.testing.assert_array_equal(got["dom_index"], ref["dom_index"])
        np.testing.assert_array_equal(got["x"], ref["x"])
        np.testing.assert_array_equal(got["level"], ref["level"])
        st = code.stats(i)
        assert [s["n_active"] for s in st] == [s["n_active"] for s in rstats]
    code.free()


def test_encode_host_image_and_again():
    fic = _fic()
    ctx = G.ctx()
    img = synth_image(64, 64, 50, n_textured=1)
    p = fic.default_params()
    code = ctx.encode(img, p)  # host numpy array: the library copies it
    ref, _ = oracle.encode(img, G.oracle_params(p))
    np.testing.assert_array_equal(code.transforms(0)["e_num"], ref["e_num"])
    img2 = synth_image(64, 64, 51, n_textured=1)
    ctx.encode_again(code, img2, p)
    ref2, _ = oracle.encode(img2, G.oracle_params(p))
    got2 = code.transforms(0)
    np.testing.assert_array_equal(got2["e_num"], ref2["e_num"])
    np.testing.assert_array_equal(got2["dom_index"], ref2["dom_index"])
    code.free()


def test_flat_image_exact():
    fic = _fic()
    ctx = G.ctx()
    img = _flat(64, 64, 90)
    p = fic.default_params(rms_threshold=0.0)
    code = ctx.encode(G.dev(img), p)
    t = code.transforms(0)
    st = code.stats(0)
    assert st[0]["fallback"] == 1
    assert np.all(t["e_num"] == 0)
    assert len(t) == 16  # every 16x16 range accepted at level 0 with E = 0
    dec = code.decode(0)
    np.testing.assert_array_equal(dec, img)
    code.free()


def test_ramp_reconstructs_exactly():
    """An integer ramp f = x: the decimated domain has twice the slope, so
    s = 0.5 (Sec. 3.1's step-4 set) with the identity reproduces it with
    E = 0 at the 2x2 level (threshold 0 forces the descent)."""
    fic = _fic()
    ctx = G.ctx()
    img = _ramp(128, 64)
    p = fic.default_params(rms_threshold=0.0)
    code = ctx.encode(G.dev(img), p)
    t = code.transforms(0)
    ref, _ = oracle.encode(img, G.oracle_params(p))
    np.testing.assert_array_equal(t["e_num"], ref["e_num"])
    assert np.all(t["e_num"][t["level"] == 3] == 0)
    code.free()


def test_invalid_arguments():
    fic = _fic()
    ctx = G.ctx()
    img = synth_image(64, 64, 1)
    p = fic.default_params()
    with pytest.raises(fic.FicError) as e:
        ctx.encode(G.dev(img[:, :40]), p)  # width not a multiple of 16
    assert e.value.status == fic.FIC_EINVAL
    bad = fic.default_params(range_size0=3)
    with pytest.raises(fic.FicError):
        ctx.encode(G.dev(img), bad)
    pool = ctx.build_domain_pool(G.dev(img), 8, p)
    with pytest.raises(fic.FicError):
        ctx.match_level(G.dev(img), pool, np.array([[60, 60]], np.int32), p)  # outside
    pool.free()


def test_graph_replay_and_profiling():
    """fic_encode_again on a stream captures the encode once and replays it:
    same maps as the direct encode; the level timers report positive times."""
    fic = _fic()
    torch = G.torch_cuda()
    ctx = G.ctx()
    img = synth_image(96, 64, 60, n_textured=1)
    d = G.dev(img)
    p = fic.default_params()
    ref = ctx.encode(d, p)
    want = ref.transforms(0)
    ref.free()
    st = torch.cuda.Stream()
    code = ctx.encode(d, p, stream=st)
    code.set_profiling(True)
    for _ in range(3):
        ctx.encode_again(code, d, p, stream=st)
        torch.cuda.synchronize()
        got = code.transforms(0)
        np.testing.assert_array_equal(got, want)
        prof = code.profile()
        assert len(prof) == 4 and all(m > 0 and lv >= m for m, lv in prof), prof
    assert code.graph_kernels() > 20
    code.free()


def test_pool_parity_large_multi_kernel_select():
    """A pool above 2^20 positions (1104 x 1104, L = 1, B = 2: 1,212,201
    positions) takes the multi-kernel radix select; keys, threshold and the
    kept list match the oracle bit-exactly, for two percentiles."""
    fic = _fic()
    ctx = G.ctx()
    img = synth_image(1104, 1104, 77, n_textured=2)
    for B, pct in ((2, 0.5), (4, 0.75)):
        p = fic.default_params(domain_step=1, entropy_percentile=pct)
        pool = ctx.build_domain_pool(G.dev(img), B, p)
        info = pool.info()
        keys_o, kept_o, thr_o, fb_o = oracle.pool_filter(img, B, 1, pct)
        assert info["pool_size"] == len(keys_o) > (1 << 20)
        np.testing.assert_array_equal(pool.copy(fic.FIC_POOL_KEYS), keys_o)
        assert info["thr_key"] == thr_o and info["fallback"] == fb_o
        np.testing.assert_array_equal(pool.copy(fic.FIC_POOL_KEPT), kept_o)
        pool.free()


# (W, H, seed, B, L, percentile, pool size K, extra pitch): pools between the
# shared-memory sizes of the one-block select -- up to 12288 keys whole, up to
# 81920 through two sample splitters, above that two passes over L2 -- at
# B = 16 (one warp per sliding run) and below; odd L (every other position
# per run, odd x offsets) and an odd row pitch (single-byte pixel loads).
MEDIUM_POOLS = [
    (512, 512, 11, 16, 2, 0.5, 0, 0),      # 58081 positions: sample splitters
    (512, 512, 12, 16, 2, 0.5, 20000, 0),  # the same path, top-K
    (320, 304, 13, 16, 1, 0.3, 0, 1),      # 78897, odd L, pitch 321
    (304, 256, 14, 16, 3, 0.9, 0, 0),      # 6825, odd L: whole pool in shared memory
    (384, 384, 15, 8, 1, 0.5, 0, 0),       # 136161: two L2 passes
    (296, 296, 16, 4, 1, 0.75, 0, 3),      # 83521: two L2 passes, pitch 299
]


@pytest.mark.parametrize("case", range(len(MEDIUM_POOLS)))
def test_pool_parity_medium(case):
    """Keys, threshold, kept list and moments of medium pools match the oracle
    bit-exactly on every path of the one-block select."""
    fic = _fic()
    W, H, seed, B, L, pct, K, pad = MEDIUM_POOLS[case]
    img = synth_image(W, H, seed, n_textured=1)
    ctx = G.ctx()
    p = fic.default_params(domain_step=L, entropy_percentile=pct, pool_size=K)
    dev = G.dev(np.pad(img, ((0, 0), (0, pad))))[:, :W]  # row pitch W + pad
    assert dev.stride(0) == W + pad
    pool = ctx.build_domain_pool(dev, B, p)
    info = pool.info()
    keys_o, kept_o, thr_o, fb_o = oracle.pool_filter(img, B, L, pct, top_k=K)
    P, px, py = oracle.pool_size(W, H, B, L)
    assert info["pool_size"] == P and info["px"] == px and info["py"] == py
    np.testing.assert_array_equal(pool.copy(fic.FIC_POOL_KEYS), keys_o)
    assert info["thr_key"] == thr_o and info["fallback"] == fb_o
    kept = pool.copy(fic.FIC_POOL_KEPT)
    np.testing.assert_array_equal(kept, kept_o)
    sums = pool.copy(fic.FIC_POOL_SUMS)
    sq = pool.copy(fic.FIC_POOL_SQSUMS)
    for j in range(0, len(kept_o), max(1, len(kept_o) // 200)):
        d = int(kept_o[j])
        Ds = oracle.decimate(img, (d % px) * L, (d // px) * L, B)
        assert sums[j] == Ds.sum() and sq[j] == (Ds * Ds).sum()
    pool.free()


@pytest.mark.parametrize("o_bits", [7, 5])
def test_stored_form_quantized_offset_and_bits(o_bits):
    """The stored form (o in o_bits bits, the bit count behind the compression
    ratio) equals the oracle's: quantised o bit-exact, the decoded image of the
    quantised maps identical, the same total bits."""
    fic = _fic()
    ctx = G.ctx()
    img = synth_image(96, 64, 28, n_textured=1)
    p = fic.default_params()
    code = ctx.encode(G.dev(img), p)
    ref, rstats = oracle.encode(img, G.oracle_params(p))
    np.testing.assert_array_equal(code.transforms(0)["e_num"], ref["e_num"])
    assert code.bits(0, o_bits) == oracle.code_bits(rstats, o_bits=o_bits)
    code.quantize_o(o_bits)
    got = code.transforms(0)
    refq = oracle.quantize_o(ref, o_bits)
    np.testing.assert_array_equal(got["o"], refq["o"])
    dec = code.decode(0)
    ref_f, _ = oracle.decode(refq, 96, 64)
    np.testing.assert_array_equal(dec, oracle.to_u8(ref_f))
    code.free()


def test_autotune_keeps_results():
    """autotune = 1 times several schedules on the first encode and keeps the
    fastest; the maps are the same as with the default schedule, also on the
    graph replay that follows."""
    fic = _fic()
    torch = G.torch_cuda()
    ctx = G.ctx()
    imgs = [synth_image(W, H, 70 + i, n_textured=1) for i, (W, H) in enumerate([(96, 64), (64, 64)])]
    d = [G.dev(im) for im in imgs]
    p0 = fic.default_params()
    ref = ctx.encode(d, p0)
    want = [ref.transforms(i) for i in range(2)]
    ref.free()
    p1 = fic.default_params(autotune=1)
    st = torch.cuda.Stream()
    code = ctx.encode(d, p1, stream=st)
    torch.cuda.synchronize()
    for i in range(2):
        np.testing.assert_array_equal(code.transforms(i), want[i])
    ctx.encode_again(code, d, p1, stream=st)
    torch.cuda.synchronize()
    for i in range(2):
        np.testing.assert_array_equal(code.transforms(i), want[i])
    code.free()
