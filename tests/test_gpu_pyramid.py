"""GPU parity of Gaussian-pyramid (mipmap) foveation against the FP64
oracle, through the C ABI. Bars: uint8 within 1 LSB (almost all equal),
float32 within 1e-5 absolute for values in [0, 1) (fp32 pyramid levels and
fp32 sigma: the level fraction is continuous in sigma)."""
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


def render(fv, img, fmt, fx, fy, s0, k):
    x = to_dev(img)
    w, h, c = fv._shape_of(x, fmt)
    ctx = fv.Context(w, h, c, 32, s0, k, fmt)
    y = torch.empty_like(x)
    ctx.render_pyramid(x, y, fx, fy)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("W,H,C,fx,fy,s0,k", [
    (100, 70, 3, 40.5, 33.25, 0.5, 0.05),
    (37, 29, 3, -12.0, 50.0, 0.3, 0.2),
    (64, 48, 1, 60.0, 2.0, 0.0, 0.1),
    (50, 41, 4, 25.0, 20.5, 1.2, 0.08),
    (1, 23, 2, 0.5, 11.5, 0.6, 0.3),
    (33, 17, 3, 0.0, 0.0, 0.5, 3.0),    # levels down to 1 x 1
])
def test_u8_pyramid_matches_oracle(fv, W, H, C, fx, fy, s0, k):
    img = wl.uniform_u8((H, W, C), seed=W * H)
    y = render(fv, img, fv.U8_HWC, fx, fy, s0, k)
    ref = oracle.forward_pyramid_u8(img, fx, fy, s0, k, "hwc")
    assert_u8_close(y, ref, min_equal=0.99)


def test_f32_pyramid_matches_oracle(fv):
    img = wl.uniform_f32((3, 45, 61), seed=2)
    y = render(fv, img, fv.F32_CHW, 20.0, 30.0, 0.4, 0.12)
    ref = oracle.forward_pyramid(img, 20.0, 30.0, 0.4, 0.12, "chw")
    assert_f32_close(y, ref, atol=1e-5)


def test_zero_sigma_is_the_identity(fv):
    img = wl.uniform_u8((30, 45, 3), seed=3)
    assert np.array_equal(render(fv, img, fv.U8_HWC, 10.0, 10.0, 0.0, 0.0), img)


def test_frame_1080p_u8_sampled(fv):
    s = wl.frame_1080p()
    y = render(fv, s.image, fv.U8_HWC, s.fix_x, s.fix_y, s.sigma0, s.k)
    g = np.random.Generator(np.random.PCG64(4))
    pix = np.unique(np.concatenate([[0, 1919, 1079 * 1920, 1920 * 1080 - 1, 540 * 1920 + 960],
                                    g.choice(1920 * 1080, size=4000, replace=False)])).astype(np.int64)
    ref = oracle.forward_pyramid_u8(s.image, s.fix_x, s.fix_y, s.sigma0, s.k, "hwc", pixels=pix)
    assert_u8_close(y.reshape(-1, 3)[pix], ref.reshape(-1, 3)[pix], min_equal=0.99)
