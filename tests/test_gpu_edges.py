"""GPU edge cases through the C ABI: radii at the library's maximum, 1 x 1
and one-column frames, one-pixel blocks (which equal per-pixel foveation),
and an empty batch. Bars as in the forward tests: uint8 within 1 LSB,
float32 within 1e-5."""
import numpy as np
import pytest
import torch

import oracle
from paper_2012_08655_gb300 import workloads as wl
from _helpers import assert_f32_close, assert_u8_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_08655_gb300 import fovea
    return fovea


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def render(fv, img, fmt, B, fx, fy, s0, k, tc):
    x = to_dev(img)
    w, h, c = fv._shape_of(x, fmt)
    ctx = fv.Context(w, h, c, B, s0, k, fmt)
    ctx.set_config(256, 0, 16 if tc == 3 else 32, tensor_cores=tc)
    y = torch.empty_like(x)
    ctx.render(x, y, fx, fy)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_radius_near_the_maximum(fv, tc):
    """An 8 x 8 frame whose far corner block reaches r = 1013 (the library's
    bound is 1023): nearly every tap clamps onto the border."""
    img = wl.uniform_u8((8, 8, 3), seed=4)
    s0, k = 0.5, 39.7   # block (1, 1) of side 4 is centred at (6, 6): e = 6 sqrt(2), r = ceil(3 (0.5 + k e))
    _, rad = oracle.sigma_table(8, 8, 4, 0.0, 0.0, s0, k)
    assert 1000 < rad.max() <= 1023
    y = render(fv, img, fv.U8_HWC, 4, 0.0, 0.0, s0, k, tc)
    ref = oracle.forward_u8(img, 4, 0.0, 0.0, s0, k, "hwc")
    # 192 values: every one within 1 LSB, at most two of them off (a rounding
    # tie of the fp32 or fp16-split sums against the binary64 oracle)
    assert_u8_close(y, ref, min_equal=0.0)
    assert int((y.astype(int) != ref.astype(int)).sum()) <= 2


def test_radius_near_the_maximum_f32(fv):
    img = wl.uniform_f32((2, 8, 8), seed=5)
    y = render(fv, img, fv.F32_CHW, 4, 0.0, 0.0, 0.5, 39.7, 1)
    ref = oracle.forward(img, 4, 0.0, 0.0, 0.5, 39.7, "chw")
    assert_f32_close(y, ref, atol=1e-5)


@pytest.mark.parametrize("shape", [(1, 1, 3), (1, 40, 1), (37, 1, 2)])
@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_degenerate_frames(fv, shape, tc):
    H, W, C = shape
    img = wl.uniform_u8(shape, seed=H * W + C)
    y = render(fv, img, fv.U8_HWC, 32, W / 3.0, H / 2.0, 0.8, 0.3, tc)
    ref = oracle.forward_u8(img, 32, W / 3.0, H / 2.0, 0.8, 0.3, "hwc")
    # 3 to 74 values: every one within 1 LSB, at most two of them off
    assert_u8_close(y, ref, min_equal=0.0)
    assert int((y.astype(int) != ref.astype(int)).sum()) <= 2


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_one_pixel_blocks_equal_per_pixel_foveation(fv, tc):
    """With B = 1 every block is a pixel, so the block-wise map is the
    per-pixel map (the oracle's per-pixel function, a different code path)."""
    img = wl.uniform_u8((21, 26, 3), seed=6)
    y = render(fv, img, fv.U8_HWC, 1, 9.5, 12.25, 0.4, 0.2, tc)
    ref = oracle.forward_pixel_u8(img, 9.5, 12.25, 0.4, 0.2, "hwc")
    assert_u8_close(y, ref, min_equal=0.99)
    x = to_dev(img)
    yp = torch.empty_like(x)
    fv.Context(26, 21, 3, 32, 0.4, 0.2, fv.U8_HWC).render_pixelwise(x, yp, 9.5, 12.25)
    torch.cuda.synchronize()
    d = np.abs(yp.cpu().numpy().astype(int) - y.astype(int))
    assert d.max() <= 1


def test_empty_batch_is_refused(fv):
    with pytest.raises(ValueError):
        fv.foveate_batch([])
