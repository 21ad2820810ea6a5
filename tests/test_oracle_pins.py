"""Pins of the CPU oracle against things other than itself (CPU only).

Each test checks one oracle function against what the paper or mathematics
fixes: values printed in the paper (tests/golden), library routines
(scipy.stats.entropy, numpy.rot90), exact rational brute force of Eq. 1-3,
closed forms, and special images whose encoding is known exactly.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.stats

import oracle
from paper_1501_04140_gb300.synth import synth_image

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- Eq. 4-5

def test_entropy_special_cases():
    flat = np.full((8, 8), 77, np.uint8)
    assert oracle.entropy(flat, 0, 0, 8) == 0.0
    distinct = np.arange(256, dtype=np.uint8).reshape(16, 16)
    assert oracle.entropy(distinct, 0, 0, 16) == pytest.approx(math.log(256), abs=1e-12)
    half = np.zeros((4, 4), np.uint8)
    half[:2] = 200
    assert oracle.entropy(half, 0, 0, 4) == pytest.approx(math.log(2), abs=1e-12)


def test_entropy_matches_scipy_natural_log():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 40, size=(40, 40)).astype(np.uint8)
    for (x, y, size) in [(0, 0, 4), (3, 5, 8), (10, 2, 16), (8, 8, 32)]:
        blk = img[y:y + size, x:x + size].ravel()
        counts = np.bincount(blk, minlength=256)
        ref = scipy.stats.entropy(counts)  # natural log, p = q / sum(q)
        assert oracle.entropy(img, x, y, size) == pytest.approx(ref, abs=1e-12)


def test_key_table_correctly_rounded():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    t = oracle.key_table(1024)
    for q in range(0, 1025):
        if q == 0:
            assert t[0] == 0
            continue
        exact = mpmath.mpf(q) * mpmath.log(q) * mpmath.mpf(2) ** 32
        ref = int(mpmath.nint(exact))
        assert int(t[q]) == ref, q
        # margin from the rounding boundary, so no platform's long double
        # can round the other way
        frac = exact - mpmath.floor(exact)
        assert abs(frac - mpmath.mpf(0.5)) > mpmath.mpf(1e-3), q


def test_entropy_key_orders_like_entropy():
    img = synth_image(96, 96, 11, n_textured=1)
    keys, ents = [], []
    for y in range(0, 96 - 8, 3):
        for x in range(0, 96 - 8, 5):
            keys.append(oracle.entropy_key(img, x, y, 8))
            ents.append(oracle.entropy(img, x, y, 8))
    keys = np.array(keys)
    ents = np.array(ents)
    n = 64.0
    recon = np.log(n) - keys / (n * 2.0 ** 32)
    np.testing.assert_allclose(recon, ents, atol=1e-9)
    order = np.argsort(keys, kind="stable")
    assert np.all(np.diff(ents[order]) <= 1e-12)


# ---------------------------------------------------------------- Sec. 2 pool

def test_pool_counts_golden():
    for N, n, L, n_ranges, n_domains in _read_golden("pool_counts.txt"):
        N, n, L = int(N), int(n), int(L)
        P, nx, ny = oracle.pool_size(N, N, n, L)
        assert P == int(n_domains)
        assert (N // n) ** 2 == int(n_ranges)
        if L == 1:
            assert P == (N - 2 * n + 1) ** 2


def test_pool_keys_positions_and_threshold():
    img = synth_image(64, 48, 4)
    for B, L, pct in [(8, 2, 0.5), (4, 3, 0.75), (2, 1, 0.5), (16, 2, 0.25)]:
        keys, kept, thr, fb = oracle.pool_filter(img, B, L, pct)
        H, W = img.shape
        xs = list(range(0, W - 2 * B + 1, L))
        ys = list(range(0, H - 2 * B + 1, L))
        assert len(keys) == len(xs) * len(ys)
        ents = []
        for iy, y in enumerate(ys):
            for ix, x in enumerate(xs):
                assert keys[iy * len(xs) + ix] == oracle.entropy_key(img, x, y, 2 * B)
                blk = img[y:y + 2 * B, x:x + 2 * B].ravel()
                ents.append(scipy.stats.entropy(np.bincount(blk, minlength=256)))
        ents = np.array(ents)
        # threshold = the entropy at the percentile position of the sorted pool
        srt = np.sort(ents)
        thr_h = srt[int(math.floor(pct * (len(ents) - 1)))]
        strict = np.nonzero(ents > thr_h + 1e-9)[0]
        ambiguous = np.abs(ents - thr_h) <= 1e-9
        kept_set = set(kept.tolist())
        assert set(strict.tolist()) <= kept_set
        assert kept_set <= set(np.nonzero((ents > thr_h + 1e-9) | ambiguous)[0].tolist())
        assert fb == 0
        assert np.all(np.diff(kept) > 0)


def test_pool_size_keeps_the_highest_entropies():
    """Tables 1-2's pool size K: the kept set is the K domains of highest
    entropy (scipy entropies; ties at the boundary dropped), K >= P keeps the
    whole pool."""
    img = synth_image(64, 48, 4, n_textured=1)
    H, W = img.shape
    for B, L, K in [(8, 2, 32), (4, 2, 64), (2, 1, 256), (4, 3, 7), (8, 4, 10 ** 6)]:
        keys, kept, thr, fb = oracle.pool_filter(img, B, L, 0.5, top_k=K)
        xs = list(range(0, W - 2 * B + 1, L))
        ys = list(range(0, H - 2 * B + 1, L))
        ents = np.array([scipy.stats.entropy(np.bincount(img[y:y + 2 * B, x:x + 2 * B].ravel(),
                                                          minlength=256))
                         for y in ys for x in xs])
        P = len(ents)
        if K >= P:
            assert len(kept) == P and fb == 1
            continue
        # entropy of the (K+1)-th highest: keep what lies strictly above it
        thr_h = np.sort(ents)[::-1][K]
        strict = set(np.nonzero(ents > thr_h + 1e-9)[0].tolist())
        near = set(np.nonzero(np.abs(ents - thr_h) <= 1e-9)[0].tolist())
        kept_set = set(kept.tolist())
        assert strict <= kept_set <= strict | near
        assert len(kept) <= K
        assert np.all(np.diff(kept) > 0)


def test_pool_fallback_on_flat_image():
    img = np.full((32, 32), 9, np.uint8)
    keys, kept, thr, fb = oracle.pool_filter(img, 4, 2, 0.5)
    assert fb == 1
    assert len(kept) == len(keys)


# ---------------------------------------------------------------- decimation, isometries

def test_decimate_is_2x2_sum():
    img = synth_image(40, 40, 7)
    for (x, y, B) in [(0, 0, 2), (3, 5, 4), (7, 1, 8), (4, 4, 16)]:
        blk = img[y:y + 2 * B, x:x + 2 * B].astype(np.int64)
        ref = blk.reshape(B, 2, B, 2).sum(axis=(1, 3))
        np.testing.assert_array_equal(oracle.decimate(img, x, y, B), ref)


def test_isometries_are_clockwise_rotations_and_mirrors():
    rng = np.random.default_rng(3)
    for B in (2, 4, 8, 16):
        D = rng.integers(0, 1021, size=(B, B))
        for k in range(8):
            ref = np.rot90(D, k=-(k % 4))  # clockwise by 90 k degrees
            if k >= 4:
                ref = np.fliplr(ref)
            np.testing.assert_array_equal(oracle.isometry(D, k), ref)
    # hand-worked 2x2 case: [[a, b], [c, d]] rotated clockwise is [[c, a], [d, b]]
    D = np.array([[1, 2], [3, 4]])
    np.testing.assert_array_equal(oracle.isometry(D, 1), [[3, 1], [4, 2]])
    np.testing.assert_array_equal(oracle.isometry(D, 4), [[2, 1], [4, 3]])


def test_isometry_group_closure_and_invariants():
    rng = np.random.default_rng(4)
    B = 4
    D = rng.permutation(B * B).reshape(B, B)  # distinct entries
    imgs = [oracle.isometry(D, k) for k in range(8)]
    keys = {tuple(m.ravel()) for m in imgs}
    assert len(keys) == 8
    for a in range(8):
        for b in range(8):
            comp = oracle.isometry(oracle.isometry(D, b), a)
            assert tuple(comp.ravel()) in keys
        # every map has an inverse in the set
        assert any(np.array_equal(oracle.isometry(imgs[a], b), D) for b in range(8))
    for m in imgs:
        assert m.sum() == D.sum() and (m * m).sum() == (D * D).sum()


# ---------------------------------------------------------------- Eq. 1-3

def _eq1_fraction(R, Ds, s):
    """Eq. 1 with Eq. 3's offset, in exact rationals; d_i = Ds_i / 4."""
    R = [Fraction(int(v)) for v in np.ravel(R)]
    d = [Fraction(int(v), 4) for v in np.ravel(Ds)]
    n = len(R)
    o = sum(R) / n - s * (sum(d) / n)
    return sum((s * di + o - ri) ** 2 for di, ri in zip(d, R))


def test_error_num_is_exact_eq1():
    rng = np.random.default_rng(8)
    for B in (2, 4, 8, 16):
        n = B * B
        for _ in range(5):
            R = rng.integers(0, 256, size=n)
            Ds = rng.integers(0, 1021, size=n)
            for (p, q) in [(1, 10), (9, 10), (0, 15), (15, 15), (7, 31)]:
                e = _eq1_fraction(R, Ds, Fraction(p, q))
                num = oracle.error_num(R, Ds, p, q)
                assert Fraction(num, 16 * q * q * n * n) == e
                assert oracle.error_direct(R, Ds, p, q) == pytest.approx(float(e), rel=1e-12, abs=1e-9)


def test_map_numerators_against_exact_eq1_eq3():
    """oracle.map_numerators (batched Eq. 1 / Eq. 3 of given maps) against
    exact rationals on a decimation by numpy reshape and isometries by
    numpy.rot90 / fliplr, on maps of every size at arbitrary positions."""
    rng = np.random.default_rng(21)
    img = rng.integers(0, 256, size=(96, 80), dtype=np.uint8)
    H, W = img.shape
    rows = []
    for _ in range(120):
        B = int(rng.choice([2, 4, 8, 16]))
        q = int(rng.choice([10, 15, 31]))
        rows.append((int(rng.integers(0, W - B + 1)), int(rng.integers(0, H - B + 1)), B,
                     int(rng.integers(0, W - 2 * B + 1)), int(rng.integers(0, H - 2 * B + 1)),
                     int(rng.integers(0, 8)), int(rng.integers(0, q + 1)), q))
    maps = np.array(rows, dtype=[(f, "<i4") for f in ("x", "y", "size", "dom_x", "dom_y", "iso",
                                                      "p", "q")])
    e_num, o_num = oracle.map_numerators(img, maps, n_threads=4)
    for m, e, o in zip(maps, e_num, o_num):
        x, y, B, dx, dy, k, p, q = (int(m[f]) for f in maps.dtype.names)
        n = B * B
        R = img[y:y + B, x:x + B].astype(np.int64)
        Ds = img[dy:dy + 2 * B, dx:dx + 2 * B].astype(np.int64).reshape(B, 2, B, 2).sum(axis=(1, 3))
        T = np.rot90(Ds, k=-(k % 4))
        if k >= 4:
            T = np.fliplr(T)
        assert Fraction(int(e), 16 * q * q * n * n) == _eq1_fraction(R, T, Fraction(p, q))
        assert int(o) == 4 * q * int(R.sum()) - p * int(T.sum())  # 4 q n times Eq. 3's o
    assert oracle.map_numerators(img, maps[:0])[0].size == 0


def test_closed_form_optimum_eq2():
    """With s = s* of Eq. 2 the error is Var_R - Cov^2 / Var_D (sum form) and
    every other s gives more."""
    rng = np.random.default_rng(9)
    B = 4
    n = B * B
    for _ in range(20):
        Ds = rng.integers(0, 1021, size=n)
        R = rng.integers(0, 256, size=n)
        d = [Fraction(int(v), 4) for v in Ds]
        r = [Fraction(int(v)) for v in R]
        db, rb = sum(d) / n, sum(r) / n
        cov = sum((a - rb) * (b - db) for a, b in zip(r, d))
        vd = sum((b - db) ** 2 for b in d)
        vr = sum((a - rb) ** 2 for a in r)
        s_star = cov / vd
        e_star = _eq1_fraction(R, Ds, s_star)
        assert e_star == vr - cov * cov / vd
        # the oracle's integer form at s = p/q is never below E(s*)
        for p in range(0, 11):
            assert Fraction(oracle.error_num(R, Ds, p, 10), 16 * 100 * n * n) >= e_star


def test_s_sets_golden():
    for row in _read_golden("s_sets.txt"):
        B = int(row[0])
        want = [Fraction(v) for v in row[1:]]
        p, q = oracle.s_set(oracle.S_PREDEFINED, 0, B)
        assert [Fraction(int(a), q) for a in p] == want
    p, q = oracle.s_set(oracle.S_GRID, 16, 8)
    assert q == 15 and list(p) == list(range(16))


# ---------------------------------------------------------------- matching

def _brute_match(img, B, L, kept, ranges, s_values):
    """Exhaustive argmin of Eq. 1 in rationals; isometries from numpy."""
    H, W = img.shape
    nx = (W - 2 * B) // L + 1
    out = []
    for (rx, ry) in ranges:
        R = img[ry:ry + B, rx:rx + B].astype(np.int64)
        best = None
        for d in kept:
            dx, dy = (d % nx) * L, (d // nx) * L
            Ds = img[dy:dy + 2 * B, dx:dx + 2 * B].astype(np.int64).reshape(B, 2, B, 2).sum(axis=(1, 3))
            for k in range(8):
                T = np.rot90(Ds, k=-(k % 4))
                if k >= 4:
                    T = np.fliplr(T)
                for si, s in enumerate(s_values):
                    e = _eq1_fraction(R, T, s)
                    key = (d * 8 + k) * len(s_values) + si
                    if best is None or (e, key) < best:
                        best = (e, key)
        out.append(best)
    return out


@pytest.mark.parametrize("B,L,mode", [(2, 2, oracle.S_PREDEFINED), (4, 3, oracle.S_PREDEFINED),
                                      (2, 1, oracle.S_GRID)])
def test_match_equals_rational_brute_force(B, L, mode):
    img = synth_image(24, 24, 21)
    keys, kept, thr, fb = oracle.pool_filter(img, B, L, 0.5)
    kept = kept[:12]
    p, q = oracle.s_set(mode, 5, B)
    ranges = [(x, y) for y in range(0, 24, B * 3) for x in range(0, 24, B * 2)][:10]
    got = oracle.match(img, B, L, kept, ranges, p, q)
    want = _brute_match(img, B, L, kept, ranges, [Fraction(int(a), q) for a in p])
    n = B * B
    for g, (e, key) in zip(got, want):
        assert Fraction(int(g["e_num"]), 16 * q * q * n * n) == e
        assert int(g["key"]) == key


def test_match_ties_take_lowest_key():
    # a flat image: every candidate has E = 0; the first key must win
    img = np.full((16, 16), 50, np.uint8)
    kept = np.arange(9, dtype=np.int32)
    got = oracle.match(img, 4, 2, kept, [(4, 4), (8, 12)], [3, 8], 10)
    assert all(int(g["e_num"]) == 0 and int(g["key"]) == 0 for g in got)


# ---------------------------------------------------------------- encoder / decoder

def _brute_quadtree(img, B0, n_levels, L, pct, T, mode, grid):
    """Quadtree of Sec. 2 on top of the rational brute-force matcher."""
    H, W = img.shape
    active = [(x, y) for y in range(0, H, B0) for x in range(0, W, B0)]
    codes = []
    for lv in range(n_levels):
        B = B0 >> lv
        n = B * B
        keys, kept, thr, fb = oracle.pool_filter(img, B, L, pct)
        # the kept set itself is pinned by test_pool_keys_positions_and_threshold
        p, q = oracle.s_set(mode, grid, B)
        res = _brute_match(img, B, L, kept, active, [Fraction(int(a), q) for a in p])
        nxt = []
        for (x, y), (e, key) in zip(active, res):
            if lv == n_levels - 1 or e <= n * Fraction(T) ** 2:
                codes.append((lv, x, y, e, key))
            else:
                h = B // 2
                nxt += [(x, y), (x + h, y), (x, y + h), (x + h, y + h)]
        active = nxt
    return codes


def test_encode_equals_brute_force_quadtree():
    img = synth_image(16, 16, 31)
    prm = oracle.make_params(n_levels=2, range_size0=4, domain_step=2, rms_threshold=4.0)
    codes, stats = oracle.encode(img, prm)
    want = _brute_quadtree(img, 4, 2, 2, 0.5, 4.0, oracle.S_PREDEFINED, 0)
    assert len(codes) == len(want)
    for c, (lv, x, y, e, key) in zip(codes, want):
        n = int(c["size"]) ** 2
        q = int(c["q"])
        assert (int(c["level"]), int(c["x"]), int(c["y"])) == (lv, x, y)
        assert Fraction(int(c["e_num"]), 16 * q * q * n * n) == e
        ns = 1 if c["size"] == 16 else 2
        assert (int(c["dom_index"]) * 8 + int(c["iso"])) * ns + int(c["s_idx"]) == key
        # Eq. 3 offset
        R = img[c["y"]:c["y"] + c["size"], c["x"]:c["x"] + c["size"]].astype(np.int64)
        B = int(c["size"])
        Ds = img[c["dom_y"]:c["dom_y"] + 2 * B, c["dom_x"]:c["dom_x"] + 2 * B].astype(np.int64)
        Ds = Ds.reshape(B, 2, B, 2).sum(axis=(1, 3))
        o = Fraction(int(R.sum()), n) - Fraction(int(c["p"]), q) * Fraction(int(Ds.sum()), 4 * n)
        assert Fraction(int(c["o_num"]), 4 * q * n) == o
    assert sum(s["n_accepted"] for s in stats) == len(codes)


# ---------------------------------------------------------------- exact s (Eq. 2)

def _eq1_min_over_unit_interval(R, Ds):
    """min over s in [0, 1] of Eq. 1 (with Eq. 3's o) from Eq. 1 alone: E(s)
    is a quadratic in s, fitted exactly through s = 0, 1/2, 1."""
    e0 = _eq1_fraction(R, Ds, Fraction(0))
    eh = _eq1_fraction(R, Ds, Fraction(1, 2))
    e1 = _eq1_fraction(R, Ds, Fraction(1))
    a = 2 * (e1 - 2 * eh + e0)          # E(s) = a s^2 + b s + c
    b = e1 - e0 - a
    if a == 0:
        s = Fraction(0) if b >= 0 else Fraction(1)
    else:
        s = min(max(-b / (2 * a), Fraction(0)), Fraction(1))
    return s, _eq1_fraction(R, Ds, s)


def test_s_exact_minimises_eq1_on_unit_interval():
    """oracle_s_exact's s is the minimiser of Eq. 1 over [0, 1] (found here
    from Eq. 1 alone), including the clamped ends and the flat block."""
    rng = np.random.default_rng(31)
    cases = []
    for B in (2, 4, 8, 16):
        n = B * B
        for _ in range(4):
            cases.append((rng.integers(0, 256, size=n), rng.integers(0, 1021, size=n)))
        base = rng.integers(0, 1021, size=n)
        cases.append((255 - base // 4, base))                       # anti-correlated: s = 0
        cases.append((np.clip(2 * (base // 4) - 100, 0, 255), base))  # slope 2: s = 1
        cases.append((rng.integers(0, 256, size=n), np.full(n, 400)))   # flat: s = 0
        cases.append((base // 8 + 30, base))                        # slope 1/2: s = 1/2
    seen = set()
    for R, Ds in cases:
        sn, sd = oracle.s_exact(R, Ds)
        s_or = Fraction(sn, sd)
        s_bf, e_bf = _eq1_min_over_unit_interval(R, Ds)
        assert _eq1_fraction(R, Ds, s_or) == e_bf
        if e_bf > 0 and s_bf != s_or:  # several minimisers only when E is flat in s
            assert _eq1_fraction(R, Ds, s_bf) == _eq1_fraction(R, Ds, s_or)
        seen.add("0" if s_or == 0 else "1" if s_or == 1 else "mid")
        # the oracle's 128-bit integer form of Eq. 1 at that s is exact
        n = len(R)
        assert Fraction(oracle.error_num128(R, Ds, sn, sd), 16 * sd * sd * n * n) == e_bf
    assert seen == {"0", "1", "mid"}


def test_mul_u128_matches_python_integers():
    rng = np.random.default_rng(32)
    for _ in range(200):
        a = int(rng.integers(0, 1 << 62)) << int(rng.integers(0, 66))
        b = int(rng.integers(0, 1 << 62)) << int(rng.integers(0, 66))
        a &= (1 << 128) - 1
        b &= (1 << 128) - 1
        assert oracle.mul_u128(a, b) == a * b
    top = (1 << 128) - 1
    assert oracle.mul_u128(top, top) == top * top


@pytest.mark.parametrize("B,L", [(2, 2), (4, 3), (8, 4)])
def test_match_exact_equals_rational_brute_force(B, L):
    """The exact-s search equals the exhaustive argmin over (domain,
    isometry) of each pair's minimum of Eq. 1 over s in [0, 1] (found from
    Eq. 1 alone), ties to the lowest key dom_index * 8 + k."""
    img = synth_image(40, 40, 33, n_textured=1)
    keys, kept, thr, fb = oracle.pool_filter(img, B, L, 0.5)
    kept = kept[:10]
    H, W = img.shape
    nx = (W - 2 * B) // L + 1
    ranges = [(x, y) for y in range(0, 40, B * 3) for x in range(0, 40, B * 2)][:8]
    got = oracle.match_exact(img, B, L, kept, ranges)
    n = B * B
    for g, (rx, ry) in zip(got, ranges):
        R = img[ry:ry + B, rx:rx + B].astype(np.int64)
        best = None
        for d in kept:
            dx, dy = (d % nx) * L, (d // nx) * L
            Ds = img[dy:dy + 2 * B, dx:dx + 2 * B].astype(np.int64).reshape(B, 2, B, 2).sum(axis=(1, 3))
            for k in range(8):
                T = np.rot90(Ds, k=-(k % 4))
                if k >= 4:
                    T = np.fliplr(T)
                s_bf, e_bf = _eq1_min_over_unit_interval(R.ravel(), T.ravel())
                key = int(d) * 8 + k
                if best is None or (e_bf, key) < best:
                    best = (e_bf, key)
        e_or = Fraction(int(g["e_lo"]) | (int(g["e_hi"]) << 64), 16 * int(g["s_den"]) ** 2 * n * n)
        assert (e_or, int(g["key"])) == best


def test_encode_exact_s_ramp_is_exact_at_the_first_level():
    """f(x, y) = x: with s free in [0, 1] the first level already finds
    s = 1/2 and E = 0 for every 16 x 16 range (the predefined sets need the
    2 x 2 level for that), and the decoder returns f."""
    img = np.tile(np.arange(64, dtype=np.uint8), (64, 1))
    codes, stats = oracle.encode(img, oracle.make_params(rms_threshold=0.0, s_mode=oracle.S_EXACT))
    assert [st["n_accepted"] for st in stats] == [16, 0, 0, 0]
    assert np.all(codes["e"] == 0.0)
    assert np.all(codes["s"] == 0.5) and np.all(codes["s_num"] * 2 == codes["s_den"])
    dec, it = oracle.decode(codes, 64, 64)
    assert np.max(np.abs(dec - img)) < 1e-6


def test_encode_exact_s_codes_follow_eq1_to_eq3():
    """Every saved map of an exact-s encode: s is Eq. 2's value clamped to
    [0, 1], o is Eq. 3 (both as doubles of the exact fractions) and the
    reported E (moment form in double) is Eq. 1's exact error to 1e-12."""
    img = synth_image(64, 64, 34, n_textured=1)
    codes, stats = oracle.encode(img, oracle.make_params(s_mode=oracle.S_EXACT))
    assert len(codes) > 20
    for c in codes[::3]:
        B = int(c["size"])
        n = B * B
        R = img[c["y"]:c["y"] + B, c["x"]:c["x"] + B].astype(np.int64)
        Ds = img[c["dom_y"]:c["dom_y"] + 2 * B, c["dom_x"]:c["dom_x"] + 2 * B].astype(np.int64)
        Ds = Ds.reshape(B, 2, B, 2).sum(axis=(1, 3))
        k = int(c["iso"])
        T = np.rot90(Ds, k=-(k % 4))
        if k >= 4:
            T = np.fliplr(T)
        r = [Fraction(int(v)) for v in R.ravel()]
        d = [Fraction(int(v), 4) for v in T.ravel()]
        rb, db = sum(r) / n, sum(d) / n
        vd = sum((x - db) ** 2 for x in d)
        cov = sum((a - rb) * (x - db) for a, x in zip(r, d))
        s_ls = cov / vd if vd else Fraction(0)       # Eq. 2
        s_cl = min(max(s_ls, Fraction(0)), Fraction(1))
        assert Fraction(int(c["s_num"]), int(c["s_den"])) == s_cl
        assert c["s"] == float(s_cl)
        assert c["o"] == pytest.approx(float(rb - s_cl * db), rel=1e-15, abs=1e-12)  # Eq. 3
        e = _eq1_fraction(R.ravel(), T.ravel(), s_cl)
        assert c["e"] == pytest.approx(float(e), rel=1e-12, abs=1e-9)


def test_encode_flat_image_is_exact():
    img = np.full((64, 64), 173, np.uint8)
    codes, stats = oracle.encode(img, oracle.make_params(rms_threshold=0.0))
    assert len(codes) == 16 and np.all(codes["e_num"] == 0)
    assert np.all(codes["dom_index"] == 0) and np.all(codes["iso"] == 0)
    dec, it = oracle.decode(codes, 64, 64)
    assert oracle.psnr(oracle.to_u8(dec), img) == float("inf")


def test_encode_ramp_reconstructs_exactly():
    """f(x, y) = x: the decimated domain has slope 2, so only s = 0.5 (in the
    step-4 set) with the identity isometry gives E = 0; with threshold 0 every
    range descends to 2 x 2 and the decoder (contraction 0.5) returns f."""
    img = np.tile(np.arange(64, dtype=np.uint8), (64, 1))
    codes, stats = oracle.encode(img, oracle.make_params(rms_threshold=0.0))
    assert [s["n_accepted"] for s in stats] == [0, 0, 0, 1024]
    assert np.all(codes["e_num"] == 0)
    assert np.all(codes["p"] == 5) and np.all(codes["q"] == 10)
    dec, it = oracle.decode(codes, 64, 64)
    assert np.max(np.abs(dec - img)) < 1e-6
    assert oracle.psnr(oracle.to_u8(dec), img) == float("inf")


def test_encode_matches_float_brute_force_min():
    """A 64x64 four-level encode: every code's E is the minimum of Eq. 1 over
    the kept pool (numpy float64 brute force, all 8 isometries, all s)."""
    img = synth_image(64, 64, 41, n_textured=1)
    prm = oracle.make_params(n_levels=4, range_size0=16, domain_step=4, rms_threshold=6.0)
    codes, stats = oracle.encode(img, prm)
    H, W = img.shape
    for c in codes[::3]:
        B = int(c["size"])
        n = B * B
        keys, kept, thr, fb = oracle.pool_filter(img, B, 4, 0.5)
        nx = (W - 2 * B) // 4 + 1
        R = img[c["y"]:c["y"] + B, c["x"]:c["x"] + B].astype(np.float64).ravel()
        p, q = oracle.s_set(oracle.S_PREDEFINED, 0, B)
        best = np.inf
        for d in kept:
            dx, dy = (d % nx) * 4, (d // nx) * 4
            D = img[dy:dy + 2 * B, dx:dx + 2 * B].astype(np.float64).reshape(B, 2, B, 2).mean(axis=(1, 3))
            for k in range(8):
                T = np.rot90(D, k=-(k % 4))
                if k >= 4:
                    T = np.fliplr(T)
                t = T.ravel()
                for a in p:
                    s = a / q
                    o = R.mean() - s * t.mean()
                    best = min(best, float(np.sum((s * t + o - R) ** 2)))
        assert c["e"] == pytest.approx(best, rel=1e-9, abs=1e-9)


def test_decoder_fixed_point_satisfies_codes():
    img = synth_image(64, 64, 51)
    codes, _ = oracle.encode(img, oracle.make_params(domain_step=4))
    dec, it = oracle.decode(codes, 64, 64, max_iters=400, tol=1e-10)
    assert it < 400
    for c in codes:
        B = int(c["size"])
        D = dec[c["dom_y"]:c["dom_y"] + 2 * B, c["dom_x"]:c["dom_x"] + 2 * B]
        D = D.reshape(B, 2, B, 2).mean(axis=(1, 3))
        T = np.rot90(D, k=-(int(c["iso"]) % 4))
        if c["iso"] >= 4:
            T = np.fliplr(T)
        want = np.clip(c["s"] * T + c["o"], 0.0, 255.0)
        got = dec[c["y"]:c["y"] + B, c["x"]:c["x"] + B]
        np.testing.assert_allclose(got, want, atol=1e-8)


# ---------------------------------------------------------------- stored form

def test_quantized_offset_grid_error_and_endpoints():
    """o stored in b bits over [-255, 255]: every value lands on the grid
    k * step - 255, within half a step of the original, monotone, endpoints
    exact, and quantising twice changes nothing."""
    for b in (5, 7, 8):
        step = 510.0 / (2 ** b - 1)
        o = np.concatenate([np.linspace(-255, 255, 2001), [-255.0, 255.0, 0.0, 3.3, -17.25]])
        codes = np.zeros(len(o), oracle.CODE_DTYPE)
        codes["o"] = o
        q1 = oracle.quantize_o(codes, b)["o"]
        k = (q1 + 255.0) / step
        assert np.allclose(k, np.round(k), atol=1e-9)
        assert np.all(np.abs(q1 - o) <= step / 2 + 1e-9)
        srt = np.argsort(o, kind="stable")
        assert np.all(np.diff(q1[srt]) >= -1e-12)
        assert q1[-5] == -255.0 and abs(q1[-4] - 255.0) < 1e-9
        q2 = oracle.quantize_o(oracle.quantize_o(codes, b), b)["o"]
        np.testing.assert_array_equal(q2, q1)


def test_code_bits_flat_image_by_hand():
    """Flat 64 x 64 image, T = 0: the 16 ranges of 16 x 16 are all kept at the
    first of four levels with E = 0.  By hand: 16 quadtree bits, and per map
    ceil(log2 289) = 9 position bits (17 x 17 positions at L = 2), 3 isometry
    bits, 0 bits of s (|S| = 1) and 7 bits of o: 16 + 16 * 19 = 320 bits."""
    img = np.full((64, 64), 90, np.uint8)
    codes, stats = oracle.encode(img, oracle.make_params(rms_threshold=0.0))
    assert len(codes) == 16 and stats[0]["pool_size"] == 289
    bits = oracle.code_bits(stats, o_bits=7)
    assert bits == 320
    assert abs(oracle.compression_ratio(64, 64, bits) - 8 * 64 * 64 / 320) < 1e-12


def test_psnr_and_u8_rounding_textbook_values():
    """PSNR = 10 log10(255^2 / MSE): an error of 1 at every pixel gives MSE 1,
    i.e. 20 log10 255 = 48.1308 dB; an error of 16 at one pixel of 256 gives
    the same MSE; errors of 255 everywhere give 0 dB.  The decoder's final
    rounding is half to even, clamped to [0, 255]."""
    a = np.full((16, 16), 100, dtype=np.uint8)
    b = a + 1
    assert abs(oracle.psnr(a, b) - 48.13080360867909) < 1e-12
    c = a.copy()
    c[3, 5] = 116
    assert abs(oracle.psnr(a, c) - 48.13080360867909) < 1e-12
    assert oracle.psnr(np.zeros((4, 4), np.uint8), np.full((4, 4), 255, np.uint8)) == 0.0
    assert oracle.psnr(a, b) == oracle.psnr(b, a)
    v = np.array([0.5, 1.5, 2.5, -3.0, 300.0, 254.5, 254.6, -0.4])
    np.testing.assert_array_equal(oracle.to_u8(v), [0, 2, 2, 0, 255, 254, 255, 0])
