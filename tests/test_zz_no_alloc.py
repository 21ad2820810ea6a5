"""fic_decode_static, the decoder that allocates no device memory, against
fic_decode.

It exists for callers that cannot let a library call cudaMalloc: processes
whose device memory is managed by another allocator (a framework's caching
allocator, a pool sized at start-up) and loops that cannot afford the device
synchronisation of an allocation.  It runs the same decoder on a static
workspace inside the library, so its image must equal fic_decode's byte for
byte, as the decoder tests require, and stay equal from one call to the next
although every call reuses (and leaves behind) the same workspace.

This file is collected last on purpose: a failure here must not stop the
other GPU tests of a run that ends at the first failure.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1501_04140_gb300.synth import synth_image
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def _encode_and_decode(fic, ctx, img):
    """Codes of `img` on the device and fic_decode's image and iteration count."""
    torch = G.torch_cuda()
    code = ctx.encode(G.dev(img), fic.default_params())
    t = code.transforms(0)
    want = code.decode(0)
    iters = code.iters
    code.free()
    codes_dev = torch.from_numpy(t.view(np.uint8).copy()).cuda()
    return codes_dev, len(t), want, iters


def test_decode_static_equals_decode_on_two_calls():
    ctx = G.ctx()
    from paper_1501_04140_gb300 import fic
    torch = G.torch_cuda()
    # two images of different sizes, decoded one after the other: the second
    # call must not see anything the first left in the shared workspace
    cases = [synth_image(128, 96, 21, n_textured=1), synth_image(64, 64, 22)]
    prepared = [_encode_and_decode(fic, ctx, img) for img in cases]
    for img, (codes_dev, n, want, iters) in zip(cases, prepared):
        H, W = img.shape
        out = torch.full((H, W), 7, dtype=torch.uint8, device="cuda")
        got_iters = fic.decode_static(codes_dev, n, W, H, out, W)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        assert got_iters == iters
    # and the first image again, after the second overwrote the workspace
    img = cases[0]
    codes_dev, n, want, iters = prepared[0]
    out = torch.zeros(img.shape, dtype=torch.uint8, device="cuda")
    assert fic.decode_static(codes_dev, n, img.shape[1], img.shape[0], out, img.shape[1]) == iters
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_decode_static_at_its_size_limits():
    """The largest image the workspace takes (exactly its pixel maximum) and
    the largest iteration count, with a tolerance of zero so that every
    iteration runs: the last iterate and the last per-iteration maximum sit
    at the far end of the workspace, and the image must still equal
    fic_decode's with the same arguments byte for byte."""
    ctx = G.ctx()
    from paper_1501_04140_gb300 import fic
    torch = G.torch_cuda()
    side = int(round(fic.FIC_DECODE_STATIC_MAX_PIXELS ** 0.5))
    assert side * side == fic.FIC_DECODE_STATIC_MAX_PIXELS
    img = synth_image(side, side, 23, n_textured=2)
    code = ctx.encode(G.dev(img), fic.default_params())
    t = code.transforms(0)
    iters_max = fic.FIC_DECODE_STATIC_MAX_ITERS
    want = code.decode(0, max_iters=iters_max, tol=0.0)
    assert code.iters == iters_max
    code.free()
    codes_dev = torch.from_numpy(t.view(np.uint8).copy()).cuda()
    for _ in range(2):
        out = torch.zeros((side, side), dtype=torch.uint8, device="cuda")
        got = fic.decode_static(codes_dev, len(t), side, side, out, side, max_iters=iters_max,
                                tol=0.0)
        assert got == iters_max
        np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_decode_static_rejects_sizes_beyond_its_workspace():
    ctx = G.ctx()  # noqa: F841  (builds and loads the library)
    from paper_1501_04140_gb300 import fic
    torch = G.torch_cuda()
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    codes = torch.zeros(88, dtype=torch.uint8, device="cuda")
    with pytest.raises(fic.FicError) as e:  # one pixel more than the maximum
        fic.decode_static(codes, 0, 1024 * 1024 + 16, 1, out, 1024 * 1024 + 16)
    assert e.value.status == fic.FIC_EINVAL
    with pytest.raises(fic.FicError) as e:  # more iterations than the maximum
        fic.decode_static(codes, 0, 4, 4, out, 4, max_iters=1025)
    assert e.value.status == fic.FIC_EINVAL
    # a map whose domain block leaves the image is refused before decoding
    t = np.zeros(1, fic.TRANSFORM_DTYPE)
    t["size"], t["q"], t["p"] = 2, 10, 5
    t["dom_x"] = 3  # 2B = 4 columns from x = 3 leave a 4-wide image
    bad = torch.from_numpy(t.view(np.uint8).copy()).cuda()
    with pytest.raises(fic.FicError) as e:
        fic.decode_static(bad, 1, 4, 4, out, 4)
    assert e.value.status == fic.FIC_EINVAL
