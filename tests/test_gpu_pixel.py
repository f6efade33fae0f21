"""GPU parity of per-pixel ("perfect") foveation and of the SSIM map against
the FP64 oracle, through the C ABI.

Bars: uint8 within 1 LSB of the oracle (and almost all equal), float32
within 1e-5 absolute for values in [0, 1); SSIM within 2e-4 absolute (the
kernel's moments are fp32 single-pass sums of values taken relative to L/2:
|error| <~ a few x L^2/4 x 2^-24 / C2 ~ 1e-4)."""
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


def render_pixelwise(fv, img, fmt, fx, fy, s0, k, tensor_cores=1):
    x = to_dev(img)
    w, h, c = fv._shape_of(x, fmt)
    ctx = fv.Context(w, h, c, 32, s0, k, fmt)
    ctx.set_config(256, 0, 32, tensor_cores=tensor_cores)
    y = torch.empty_like(x)
    ctx.render_pixelwise(x, y, fx, fy)
    torch.cuda.synchronize()
    return y.cpu().numpy()


U8_CASES = [
    # W, H, C, fx, fy, sigma0, k
    (100, 70, 3, 40.5, 33.25, 0.5, 0.05),       # several 16x16 tiles, ragged tail in both axes
    (37, 29, 3, -12.0, 50.0, 0.3, 0.2),         # W*C = 111: byte staging path; fixation outside
    (64, 48, 1, 60.0, 2.0, 0.0, 0.1),           # one channel, sigma0 = 0 at the fixation
    (50, 41, 4, 25.0, 20.5, 1.2, 0.08),         # four channels
    (16, 16, 2, 8.0, 8.0, 0.4, 0.6),            # one tile, radius up to ~17 > tile
    (1, 23, 3, 0.5, 11.5, 0.6, 0.3),            # one column
    (64, 48, 1, 0.0, 0.0, 0.5, 0.5),            # radius up to 120: windows longer than one accumulator chunk
]


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("W,H,C,fx,fy,s0,k", U8_CASES)
def test_u8_pixelwise_matches_oracle(fv, tc, W, H, C, fx, fy, s0, k):
    img = wl.uniform_u8((H, W, C), seed=W + H)
    y = render_pixelwise(fv, img, fv.U8_HWC, fx, fy, s0, k, tensor_cores=tc)
    ref = oracle.forward_pixel_u8(img, fx, fy, s0, k, "hwc")
    assert_u8_close(y, ref, min_equal=0.99)


@pytest.mark.parametrize("W,H,C,fx,fy,s0,k", [
    (64, 40, 1, 20.0, 30.0, 0.5, 0.07),
    (33, 27, 3, 40.0, -5.0, 0.2, 0.15),
])
def test_f32_pixelwise_matches_oracle(fv, W, H, C, fx, fy, s0, k):
    img = wl.uniform_f32((C, H, W), seed=W)
    y = render_pixelwise(fv, img, fv.F32_CHW, fx, fy, s0, k)
    ref = oracle.forward_pixel(img, fx, fy, s0, k, "chw")
    assert_f32_close(y, ref, atol=1e-5)


def test_zero_sigma_is_the_identity(fv):
    img = wl.uniform_u8((30, 45, 3), seed=3)
    for tc in (1, 0):
        y = render_pixelwise(fv, img, fv.U8_HWC, 10.0, 10.0, 0.0, 0.0, tensor_cores=tc)
        assert np.array_equal(y, img)


def sample_pixels(W, H, fx, fy, n=1500, seed=0):
    """Row-major pixel indices: the corners, the fixation pixel, tile borders
    (16-pixel tiles) and random pixels."""
    g = np.random.Generator(np.random.PCG64(seed))
    sel = {0, W - 1, (H - 1) * W, H * W - 1}
    fxp, fyp = min(max(int(fx), 0), W - 1), min(max(int(fy), 0), H - 1)
    sel.add(fyp * W + fxp)
    for t in range(0, W, 16):
        sel.update({fyp * W + t, fyp * W + min(t + 15, W - 1)})
    for t in range(0, H, 16):
        sel.update({t * W + fxp, min(t + 15, H - 1) * W + fxp})
    sel.update(int(p) for p in g.choice(W * H, size=n, replace=False))
    return np.array(sorted(sel), np.int64)


def test_frame_1080p_u8_sampled(fv):
    s = wl.frame_1080p()
    y = render_pixelwise(fv, s.image, fv.U8_HWC, s.fix_x, s.fix_y, s.sigma0, s.k)
    pix = sample_pixels(1920, 1080, s.fix_x, s.fix_y)
    ref = oracle.forward_pixel_u8(s.image, s.fix_x, s.fix_y, s.sigma0, s.k, "hwc", pixels=pix)
    got = y.reshape(-1, 3)[pix]
    assert_u8_close(got, ref.reshape(-1, 3)[pix], min_equal=0.99)


def test_tensor_core_and_fp32_kernels_agree_at_1080p(fv):
    s = wl.frame_1080p(seed=5)
    fx, fy = 300.5, 900.25
    a = render_pixelwise(fv, s.image, fv.U8_HWC, fx, fy, s.sigma0, s.k, tensor_cores=1)
    b = render_pixelwise(fv, s.image, fv.U8_HWC, fx, fy, s.sigma0, s.k, tensor_cores=0)
    d = np.abs(a.astype(np.int32) - b.astype(np.int32))
    assert d.max() <= 1 and np.mean(d == 0) > 0.99


def test_pixelwise_refuses_a_sigma_map_and_huge_radii(fv):
    x = to_dev(wl.uniform_u8((40, 40, 3), seed=1))
    y = torch.empty_like(x)
    ctx = fv.Context(40, 40, 3, 8, 0.5, 2.0, fv.U8_HWC)   # corner pixel radius 337 > 255
    with pytest.raises(fv.FoveaError):
        ctx.render_pixelwise(x, y, 0.0, 0.0)
    m = torch.full((5, 5), 1.5, dtype=torch.float32, device="cuda")
    cm = fv.Context(40, 40, 3, 8, 0.0, 0.0, fv.U8_HWC, law=fv.LAW_MAP, sigma_map=m, sigma_map_max=1.5)
    with pytest.raises(fv.FoveaError):
        cm.render_pixelwise(x, y, 20.0, 20.0)


# ---------------------------------------------------------------- SSIM

@pytest.mark.parametrize("W,H,C", [(70, 45, 3), (33, 17, 1), (8, 8, 4)])
def test_ssim_u8_matches_oracle(fv, W, H, C):
    a = wl.uniform_u8((H, W, C), seed=1)
    rng = np.random.Generator(np.random.PCG64(2))
    b = np.clip(a.astype(np.int32) + rng.integers(-30, 31, a.shape), 0, 255).astype(np.uint8)
    m, mean = fv.ssim(to_dev(a), to_dev(b))
    ref = oracle.ssim_map(a, b, 255.0, "hwc")
    np.testing.assert_allclose(m.cpu().numpy(), ref, rtol=0, atol=2e-4)
    assert abs(mean - ref.mean()) < 2e-4


def test_ssim_f32_matches_oracle_and_identity(fv):
    a = wl.uniform_f32((2, 40, 52), seed=6)
    b = np.clip(a + 0.05 * np.sin(np.arange(52))[None, None, :], 0, 1).astype(np.float32)
    m, mean = fv.ssim(to_dev(a), to_dev(b), data_range=1.0)
    ref = oracle.ssim_map(a, b, 1.0, "chw")
    np.testing.assert_allclose(m.cpu().numpy(), ref, rtol=0, atol=2e-4)
    m1, mean1 = fv.ssim(to_dev(a), to_dev(a), data_range=1.0)
    np.testing.assert_allclose(m1.cpu().numpy(), 1.0, rtol=0, atol=2e-4)
    assert abs(mean1 - 1.0) < 2e-4


def test_blockwise_against_pixelwise_ssim_1080p(fv):
    """The comparison of Section 3.1 on the synthetic 1080p frame: the block-
    wise output is close to the per-pixel reference, and the SSIM map on the
    GPU matches the oracle's on sampled rows."""
    s = wl.frame_1080p()
    x = to_dev(s.image)
    ref = fv.foveate_pixelwise(x, s.fix_x, s.fix_y, s.sigma0, s.k)
    blk = fv.foveate(x, s.fix_x, s.fix_y, s.sigma0, s.k)
    m, mean = fv.ssim(blk, ref)
    assert 0.9 < mean <= 1.0
    rows = slice(520, 560)
    o = oracle.ssim_map(blk.cpu().numpy()[rows], ref.cpu().numpy()[rows], 255.0, "hwc")
    # interior rows of the crop only (the crop's own border clamps differently)
    np.testing.assert_allclose(m.cpu().numpy()[rows][5:-5], o[5:-5], rtol=0, atol=2e-4)
