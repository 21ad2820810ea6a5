"""Seeded synthetic 8-bit grayscale images (input generation only).

Stand-ins for the natural test images of the paper's experiments (Sec. 4:
Lena, Baboon, F16 -- not available here): a sum of smooth 2-D ramps, step
edges of random orientation (height h split as +-h/2 about the
edge), Gaussian-like noise and optional band-limited
texture tiles, clipped to 0..255.

The generator uses a counter-based hash (splitmix64) and only IEEE basic
arithmetic and square roots, so the same seed gives the same image on every
platform.  This module holds none of the encoder's arithmetic; both the
oracle-side tests and the CUDA path consume its images.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on uint64 counters."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


class _Stream:
    """Uniform doubles in [0, 1) from hash(seed, stream, counter)."""

    def __init__(self, seed: int, stream: int):
        with np.errstate(over="ignore"):
            self.base = _splitmix64(np.array([(seed * 0x100000001B3 + stream * 0x9E37) & 0xFFFFFFFFFFFFFFFF],
                                             dtype=np.uint64))[0]
        self.ctr = 0

    def uniform(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            c = np.arange(self.ctr, self.ctr + n, dtype=np.uint64) + self.base * np.uint64(2)
        self.ctr += n
        bits = _splitmix64(c) >> np.uint64(11)
        return bits.astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """Irwin-Hall approximation: sum of 12 uniforms minus 6 (unit variance)."""
        u = self.uniform(12 * n).reshape(12, n)
        acc = u[0].copy()
        for i in range(1, 12):
            acc = acc + u[i]
        return acc - 6.0


def _binomial_blur(a: np.ndarray, taps: int = 11) -> np.ndarray:
    """Separable binomial low-pass (C(10,k)/2^10, sigma ~1.58), edge-padded."""
    w = np.array([1, 10, 45, 120, 210, 252, 210, 120, 45, 10, 1], np.float64) / 1024.0
    r = taps // 2
    p = np.pad(a, r, mode="edge")
    h = np.zeros((p.shape[0], a.shape[1]))
    for k in range(taps):
        h = h + w[k] * p[:, k:k + a.shape[1]]
    v = np.zeros(a.shape)
    for k in range(taps):
        v = v + w[k] * h[k:k + a.shape[0], :]
    return v


def synth_image(W: int, H: int, seed: int, n_textured: int = 0, noise_sigma: float = 6.0,
                texture_amp: float = 40.0) -> np.ndarray:
    """Return an (H, W) uint8 image.

    Components: 4 smooth ramps (random direction, amplitude U(20, 60), a
    smoothstep profile over a random span), 3 step edges (random orientation
    through a random point, height U(-60, 60)), per-pixel noise of standard
    deviation ``noise_sigma`` and ``n_textured`` tiles of band-limited noise
    (binomial-filtered white noise scaled to standard deviation
    ``texture_amp``).  One tile is a quadrant of the image; with more than one
    tile, each is W/8 x H/8 at a seeded position.
    """
    g = _Stream(seed, 1)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.full((H, W), 128.0)
    span = float(max(W, H))
    for _ in range(4):
        v = g.uniform(6)
        dx, dy = 2.0 * v[0] - 1.0, 2.0 * v[1] - 1.0
        nrm = np.sqrt(dx * dx + dy * dy) + 1e-9
        dx, dy = dx / nrm, dy / nrm
        amp = 20.0 + 40.0 * v[2]
        sign = 1.0 if v[3] < 0.5 else -1.0
        width = span * (0.5 + 1.5 * v[4])
        centre = (v[5] - 0.5) * span
        t = ((xx - W / 2.0) * dx + (yy - H / 2.0) * dy - centre) / width + 0.5
        t = np.clip(t, 0.0, 1.0)
        img = img + sign * amp * (t * t * (3.0 - 2.0 * t) - 0.5)
    for _ in range(3):
        v = g.uniform(5)
        dx, dy = 2.0 * v[0] - 1.0, 2.0 * v[1] - 1.0
        nrm = np.sqrt(dx * dx + dy * dy) + 1e-9
        dx, dy = dx / nrm, dy / nrm
        x0, y0 = v[2] * W, v[3] * H
        h = -60.0 + 120.0 * v[4]
        img = img + np.where((xx - x0) * dx + (yy - y0) * dy > 0.0, 0.5 * h, -0.5 * h)
    img = img + noise_sigma * g.normal(W * H).reshape(H, W)
    if n_textured > 0:
        t = _Stream(seed, 2)
        # std of the 2-D binomial filter applied to unit white noise
        gain = 184756.0 / 1048576.0
        for k in range(n_textured):
            if n_textured == 1:
                q = int(t.uniform(1)[0] * 4.0) % 4
                tw, th = W // 2, H // 2
                x0, y0 = (q % 2) * tw, (q // 2) * th
            else:
                tw, th = max(W // 8, 8), max(H // 8, 8)
                v = t.uniform(2)
                x0 = int(v[0] * (W - tw))
                y0 = int(v[1] * (H - th))
            noise = t.normal(tw * th).reshape(th, tw)
            tex = _binomial_blur(noise) * (texture_amp / gain)
            img[y0:y0 + th, x0:x0 + tw] = img[y0:y0 + th, x0:x0 + tw] + tex
    return np.clip(np.rint(img), 0.0, 255.0).astype(np.uint8)


BATCH_SIZES = ((256, 256), (384, 512), (512, 512), (768, 1024), (1024, 1024))


def batch_specs(n_images: int = 64, first_seed: int = 1000, mix_seed: int = 42):
    """(W, H, seed) for the uneven-size batch: sizes drawn from BATCH_SIZES by
    a seeded stream, image seeds first_seed, first_seed + 1, ..."""
    u = _Stream(mix_seed, 3).uniform(n_images)
    out = []
    for i in range(n_images):
        W, H = BATCH_SIZES[int(u[i] * len(BATCH_SIZES)) % len(BATCH_SIZES)]
        out.append((W, H, first_seed + i))
    return out
