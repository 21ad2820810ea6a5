"""The stored oracle encode that the full-size GPU parity test reads
(tests/golden/enc512_grid16.npz, written by make_oracle_golden.py) still
agrees with the oracle: its per-level thresholds, kept counts and quadtree
counts, and a sample of its maps re-derived by a live exhaustive search."""
import os

import numpy as np

import oracle
from tests.golden import make_oracle_golden as golden


def test_stored_grid16_encode_agrees_with_the_oracle():
    name = "enc512_grid16"
    img = golden.case_image(name)
    maps, stats = golden.load(name)
    assert len(stats) == 4
    assert sum(s["n_accepted"] for s in stats) == len(maps["level"])
    # Sec. 2's quadtree: every range not saved at a level is split into 4
    for a, b in zip(stats, stats[1:]):
        assert b["n_active"] == 4 * (a["n_active"] - a["n_accepted"])
    assert stats[0]["n_active"] == (512 // 16) ** 2
    assert np.all(maps["q"] == 15) and np.all(maps["p"] == maps["s_idx"])
    rng = np.random.default_rng(3)
    for lv in (2, 3):  # the cheap levels: a live search of a few maps
        B = 16 >> lv
        _, kept, thr, fb = oracle.pool_filter(img, B, 2, 0.5)
        assert (thr, len(kept), fb) == (stats[lv]["thr_key"], stats[lv]["n_kept"],
                                         stats[lv]["fallback"])
        idx = np.flatnonzero(maps["level"] == lv)
        pick = rng.choice(idx, size=4, replace=False)
        sp, q = oracle.s_set(oracle.S_GRID, 16, B)
        rxy = np.stack([maps["x"][pick], maps["y"][pick]], 1).astype(np.int32)
        ref = oracle.match(img, B, 2, kept, rxy, sp, q, n_threads=os.cpu_count() or 1)
        np.testing.assert_array_equal(maps["e_num"][pick], ref["e_num"])
        np.testing.assert_array_equal(maps["dom_index"][pick], ref["dom_index"])
        np.testing.assert_array_equal(maps["iso"][pick], ref["iso"])
        np.testing.assert_array_equal(maps["s_idx"][pick], ref["s_idx"])
