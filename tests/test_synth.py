"""The seeded input generator (shared by the oracle-side tests and the CUDA
path; it holds none of the encoder's arithmetic): its counter-based hash
against SplitMix64's published outputs, its distributions, and determinism."""
import numpy as np

from paper_1501_04140_gb300 import synth
from paper_1501_04140_gb300.synth import batch_specs, synth_image

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def test_splitmix64_first_outputs_of_seed_zero():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0 first returns
    # 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f; the i-th
    # output is the finaliser of the state i * gamma
    states = np.array([0, GAMMA, (2 * GAMMA) & M64], np.uint64)
    got = [int(v) for v in synth._splitmix64(states)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_streams():
    s = synth._Stream(7, 3)
    u = s.uniform(200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12.0) < 0.002
    # counters continue: the next draw is new numbers, not a repeat
    assert not np.array_equal(s.uniform(8), u[:8])
    z = synth._Stream(7, 4).normal(100000)  # Irwin-Hall: mean 0, variance 1
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.03
    assert np.abs(z).max() <= 6.0


def test_images_are_seeded_and_deterministic():
    a = synth_image(96, 64, 5, n_textured=1)
    b = synth_image(96, 64, 5, n_textured=1)
    c = synth_image(96, 64, 6, n_textured=1)
    assert a.dtype == np.uint8 and a.shape == (64, 96)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.std() > 5.0  # not flat: ramps, edges, noise and a texture tile


def test_batch_specs_are_seeded_sizes_from_the_set():
    s1 = batch_specs(64, 1000, 42)
    assert s1 == batch_specs(64, 1000, 42)
    assert len(s1) == 64
    sizes = {(w, h) for (w, h, _) in s1}
    assert sizes <= {(256, 256), (384, 512), (512, 512), (768, 1024), (1024, 1024)}
    assert len(sizes) > 1  # uneven sizes
    assert [sd for (_, _, sd) in s1] == list(range(1000, 1064))
