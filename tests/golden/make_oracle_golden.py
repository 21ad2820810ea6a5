"""Writes the stored oracle results that the full-size GPU parity tests read.

Every value in the files it writes comes from `oracle/` (the plain C encoder
of Sec. 2-3.1) on the seeded synthetic images of
`paper_1501_04140_gb300.synth`; nothing here runs or reads the CUDA path.
The tests compare the GPU encoder's maps with these files element by
element, and re-derive a sample of them with a live oracle call, so that a
stale file fails.

The stored encodes are the ones too slow for the oracle to redo inside a GPU
test run (minutes of CPU each):

  enc512_grid16.npz  512 x 512 (seed 1, one textured quadrant), quadtree
                     16 -> 8 -> 4 -> 2, L = 2, RMS 8, median entropy
                     threshold, s from the 16-sample grid k / 15 (Sec. 2's
                     pre-sampled set of [0, 1]).

Each file holds, per saved map in the oracle's output order, every field of
the oracle's map record (range, domain, isometry, s index, p / q, the exact
numerators of E and o, and E, s, o as doubles), and per level the statistics
size, pool_size, n_kept, fallback, thr_key, n_active and n_accepted.

  python tests/golden/make_oracle_golden.py [--threads N]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1501_04140_gb300.synth import synth_image  # noqa: E402

MAP_FIELDS = ("level", "x", "y", "size", "dom_index", "dom_x", "dom_y", "iso", "s_idx", "p", "q",
              "e_num", "o_num", "e", "s", "o")
STAT_FIELDS = ("size", "pool_size", "n_kept", "fallback", "thr_key", "n_active", "n_accepted")

# name -> (W, H, seed, n_textured, oracle params without the thread count)
CASES = {
    "enc512_grid16": (512, 512, 1, 1, dict(s_mode=oracle.S_GRID, grid_samples=16)),
}


def path_of(name: str) -> str:
    return os.path.join(HERE, name + ".npz")


def case_image(name: str) -> np.ndarray:
    W, H, seed, tex, _ = CASES[name]
    return synth_image(W, H, seed, n_textured=tex)


def case_params(name: str, n_threads: int):
    return oracle.make_params(n_threads=n_threads, **CASES[name][4])


def write(name: str, n_threads: int) -> str:
    img = case_image(name)
    codes, stats = oracle.encode(img, case_params(name, n_threads))
    arrays = {f: np.ascontiguousarray(codes[f]) for f in MAP_FIELDS}
    for f in STAT_FIELDS:
        arrays["stat_" + f] = np.array([s[f] for s in stats], np.int64)
    out = path_of(name)
    np.savez_compressed(out, **arrays)
    return out


def load(name: str) -> tuple[dict, list[dict]]:
    """(maps: field -> array, stats: list of per-level dicts)."""
    z = np.load(path_of(name))
    maps = {f: z[f] for f in MAP_FIELDS}
    n_lv = len(z["stat_size"])
    stats = [{f: int(z["stat_" + f][i]) for f in STAT_FIELDS} for i in range(n_lv)]
    return maps, stats


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("names", nargs="*", default=sorted(CASES))
    args = ap.parse_args()
    for name in args.names:
        t0 = time.time()
        out = write(name, args.threads)
        print(f"{out}: {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
