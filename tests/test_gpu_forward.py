"""GPU parity of the forward path (sigma table, halo-tile blur, uint8 codec)
against the FP64 oracle, through the C ABI.

Bars: radii bit-exact and sigma equal to the binary64 value rounded to
float32; float32 frames with values in [0, 1) within 1e-5 absolute; uint8
frames within 1 LSB (and almost all equal)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2012_08655_gb300 import workloads as wl
from _helpers import assert_f32_close, assert_u8_close, block_mask, sample_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_08655_gb300 import fovea
    return fovea


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------- sigma table

SIGMA_CASES = [
    (256, 256, 32, 128.0, 128.0, 0.5, 0.02),
    (1920, 1080, 32, 960.0, 540.0, 0.5, 0.02),
    (1920, 1080, 32, 12.25, 1070.5, 0.5, 0.04),
    (3840, 2160, 32, 3000.75, 100.125, 0.5, 0.04),
    (224, 224, 32, 17.0, 200.0, 0.5, 0.08),
    (100, 70, 16, 20.5, 61.25, 0.4, 0.05),
    (57, 41, 8, -10.0, 50.0, 0.0, 0.15),
    (640, 480, 32, 700.0, -30.0, 1.0, 0.0),
]


@pytest.mark.parametrize("W,H,B,fx,fy,s0,k", SIGMA_CASES)
def test_sigma_table_bit_exact(fv, W, H, B, fx, fy, s0, k):
    sig, rad = fv.sigma_table(W, H, fx, fy, s0, k, block=B)
    torch.cuda.synchronize()
    osig, orad = oracle.sigma_table(W, H, B, np.float32(fx), np.float32(fy), s0, k)
    assert np.array_equal(rad.cpu().numpy(), orad)
    assert np.array_equal(sig.cpu().numpy(), osig.astype(np.float32))


def test_sigma_table_random_fixations(fv):
    g = wl.rng(123)
    for _ in range(40):
        W, H = int(g.integers(1, 2000)), int(g.integers(1, 2000))
        fx, fy = np.float32(g.uniform(-200, W + 200)), np.float32(g.uniform(-200, H + 200))
        k = float(g.uniform(0.0, 0.1))
        B = int(g.choice([8, 16, 32]))
        sig, rad = fv.sigma_table(W, H, float(fx), float(fy), 0.5, k, block=B)
        osig, orad = oracle.sigma_table(W, H, B, fx, fy, 0.5, k)
        assert np.array_equal(rad.cpu().numpy(), orad)
        assert np.array_equal(sig.cpu().numpy(), osig.astype(np.float32))


# ---------------------------------------------------------------- plain 256x256 float32

def test_plain_f32_256(fv):
    s = wl.plain_f32()
    x = to_dev(s.image)
    y = fv.foveate(x, s.fix_x, s.fix_y, s.sigma0, s.k)
    torch.cuda.synchronize()
    ref = oracle.forward(s.image, 32, s.fix_x, s.fix_y, s.sigma0, s.k, "chw")
    assert_f32_close(y.cpu().numpy(), ref)


# ---------------------------------------------------------------- edge cases

EDGE = [
    # W, H, C, dtype, B, fx, fy, sigma0, k
    (37, 29, 1, "f32", 32, 10.0, 10.0, 0.5, 0.1),      # one partial block
    (100, 70, 3, "u8", 16, 20.5, 61.25, 0.4, 0.05),    # ragged, RGB, B = 16
    (57, 41, 2, "f32", 8, -10.0, 50.0, 0.0, 0.15),     # fixation outside, sigma0 = 0, B = 8
    (64, 64, 4, "u8", 32, 32.0, 32.0, 0.0, 0.0),       # sigma = 0: identity
    (64, 48, 3, "f32", 32, 0.0, 0.0, 3.0, 0.5),        # r ~ 100 > W, H: several slabs
    (1, 1, 1, "f32", 32, 0.5, 0.5, 1.0, 0.0),          # 1 x 1
    (300, 1, 3, "u8", 32, 150.0, 0.0, 0.5, 0.05),      # one row
    (1, 200, 1, "f32", 32, 0.0, 100.0, 0.5, 0.05),     # one column
    (84, 84, 1, "u8", 32, 42.0, 42.0, 0.5, 0.02),      # gray 84 x 84
    (96, 80, 3, "f32", 32, 5.0, 75.0, 0.5, 0.6),       # r ~ 220: many row chunks and slabs
    (160, 96, 2, "u8", 32, 150.0, 5.0, 0.5, 0.3),      # two channels, large r
    (33, 65, 4, "f32", 4, 16.0, 30.0, 0.3, 0.2),       # B = 4, RGBA
]


@pytest.mark.parametrize("W,H,C,dt,B,fx,fy,s0,k", EDGE)
def test_forward_edge_cases(fv, W, H, C, dt, B, fx, fy, s0, k):
    if dt == "u8":
        img = wl.uniform_u8((H, W, C), seed=W * 7 + H)
        x = to_dev(img)
    else:
        img = wl.uniform_f32((C, H, W), seed=W * 7 + H)
        x = to_dev(img)
    y = fv.foveate(x, fx, fy, s0, k, block=B)
    torch.cuda.synchronize()
    if dt == "u8":
        ref = oracle.forward_u8(img, B, fx, fy, s0, k, "hwc")
        assert_u8_close(y.cpu().numpy(), ref, min_equal=0.98)
    else:
        ref = oracle.forward(img, B, fx, fy, s0, k, "chw")
        assert_f32_close(y.cpu().numpy(), ref)
    if s0 == 0.0 and k == 0.0:
        assert torch.equal(y, x)


@pytest.mark.parametrize("W,H,C,dt,B,fx,fy,s0,k", EDGE[:10] + [(256, 256, 1, "f32", 32, 128.0, 128.0, 0.5, 0.02)])
def test_single_wave_frames_match_the_persistent_kernel(fv, W, H, C, dt, B, fx, fy, s0, k):
    """A frame with no more blocks than one wave of CTAs runs as one launch
    with one CTA per block (sigma evaluated in the CTA); the same frame in a
    batch runs the persistent kernel behind the sigma kernel. Same item body,
    same sigma: bit-equal outputs."""
    if dt == "u8":
        img = wl.uniform_u8((H, W, C), seed=W + 5 * H)
        fmt = fv.U8_HWC
    else:
        img = wl.uniform_f32((C, H, W), seed=W + 5 * H)
        fmt = fv.F32_CHW
    x = to_dev(img)
    ctx = fv.Context(W, H, C, B, s0, k, fmt)
    ctx.set_config(256, 0, 32, tensor_cores=0)
    y1 = torch.empty_like(x)
    ctx.render(x, y1, fx, fy)
    bctx = fv.batch_context(B)
    bctx.set_config(256, 0, 32, tensor_cores=0)
    y2 = torch.empty_like(x)
    bctx.render_batch([fv.BatchFrame(x, y2, fx, fy, s0, k)])
    torch.cuda.synchronize()
    assert ctx.check() == 0 and bctx.check() == 0
    assert torch.equal(y1, y2)


def test_u8_uniform_bytes_1080p_sampled(fv):
    img = wl.uniform_u8((1080, 1920, 3), seed=3)
    y = fv.foveate(to_dev(img), 700.25, 300.5, 0.5, 0.02).cpu().numpy()
    blocks = sample_blocks(1920, 1080, 32, 700.25, 300.5, n_random=48, seed=1)
    ref = oracle.forward_u8(img, 32, 700.25, 300.5, 0.5, 0.02, "hwc", blocks=blocks)
    assert_u8_close(y, ref, mask=block_mask(1920, 1080, 32, blocks, "hwc", 3))


# ---------------------------------------------------------------- 1080p RGB frame

def test_frame_1080p_u8(fv):
    s = wl.frame_1080p()
    y = fv.foveate(to_dev(s.image), s.fix_x, s.fix_y, s.sigma0, s.k).cpu().numpy()
    blocks = sample_blocks(1920, 1080, 32, s.fix_x, s.fix_y, n_random=64, seed=2, all_edges=True)
    ref = oracle.forward_u8(s.image, 32, s.fix_x, s.fix_y, s.sigma0, s.k, "hwc", blocks=blocks)
    assert_u8_close(y, ref, mask=block_mask(1920, 1080, 32, blocks, "hwc", 3), min_equal=0.995)


def test_render_host_and_batch_match_render(fv):
    s = wl.frame_1080p(seed=4)
    x = to_dev(s.image)
    ctx = fv.Context(1920, 1080, 3, 32, s.sigma0, s.k, fv.U8_HWC)
    y1 = torch.empty_like(x)
    ctx.render(x, y1, s.fix_x, s.fix_y)
    hin = torch.from_numpy(s.image).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    ctx.render_host(hin, hout, s.fix_x, s.fix_y)
    y3 = torch.empty_like(x)
    fv.foveate_batch([fv.BatchFrame(x, y3, s.fix_x, s.fix_y, s.sigma0, s.k)])
    torch.cuda.synchronize()
    assert torch.equal(y1.cpu(), hout)
    assert torch.equal(y1, y3)


@pytest.mark.parametrize("kind", ["f32_256", "u8_1080p"])
def test_render_captured_in_a_cuda_graph(fv, kind):
    """fovea_render captured into a CUDA graph (after one eager call at the
    same size and fixation, which sizes the context) and replayed: every
    replay writes the eager output bit for bit, with the input changed in
    place between replays."""
    if kind == "f32_256":
        spec = wl.plain_f32()
        x = to_dev(spec.image)
        ctx = fv.Context(256, 256, 1, 32, spec.sigma0, spec.k, fv.F32_CHW)
        fx, fy = spec.fix_x, spec.fix_y
        other = to_dev(wl.uniform_f32(spec.image.shape, seed=3))
    else:
        s = wl.frame_1080p(seed=6)
        x = to_dev(s.image)
        ctx = fv.Context(1920, 1080, 3, 32, s.sigma0, s.k, fv.U8_HWC)
        fx, fy = s.fix_x, s.fix_y
        other = to_dev(wl.uniform_u8(s.image.shape, seed=3))
    y = torch.empty_like(x)
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        ctx.render(x, y, fx, fy)
    cs.synchronize()
    src = x.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cs):
        ctx.render(src, y, fx, fy)
    for inp in (x, other, x):
        src.copy_(inp)
        y.zero_()
        g.replay()
        ref = torch.empty_like(inp)
        ctx.render(inp, ref, fx, fy)
        torch.cuda.synchronize()
        assert torch.equal(y, ref)


def test_render_host_pipelined_calls(fv):
    """Consecutive host calls alternate staging slots and overlap one another's
    copies and kernels; interleaved device-path calls on the same stream stay
    ordered with them. Every result equals the device path's."""
    frames = [wl.frame_1080p(seed=20 + i) for i in range(5)]
    fix = [(960.0, 540.0), (100.5, 1000.25), (1800.0, 30.0), (500.0, 500.0), (1919.0, 0.0)]
    s0 = frames[0]
    ctx = fv.Context(1920, 1080, 3, 32, s0.sigma0, s0.k, fv.U8_HWC)
    hin = [torch.from_numpy(f.image).pin_memory() for f in frames]
    hout = [torch.empty_like(h).pin_memory() for h in hin]
    dev_in = to_dev(frames[2].image)
    dev_out = torch.empty_like(dev_in)
    for i in range(5):
        ctx.render_host(hin[i], hout[i], *fix[i])
        if i == 2:
            ctx.render(dev_in, dev_out, 7.0, 9.0)
    torch.cuda.current_stream().synchronize()
    ref_ctx = fv.Context(1920, 1080, 3, 32, s0.sigma0, s0.k, fv.U8_HWC)
    for i in range(5):
        x = to_dev(frames[i].image)
        y = torch.empty_like(x)
        ref_ctx.render(x, y, *fix[i])
        torch.cuda.synchronize()
        assert torch.equal(y.cpu(), hout[i]), i
    y = torch.empty_like(dev_in)
    ref_ctx.render(dev_in, y, 7.0, 9.0)
    torch.cuda.synchronize()
    assert torch.equal(y, dev_out)


# ---------------------------------------------------------------- configurations

@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_every_config_gives_identical_output(fv, tc):
    """Within one kernel, the row chunk and the CTA count change nothing
    (kernel 3 stages 16-row chunks only and runs one CTA per SM whatever the
    requested count)."""
    s = wl.frame_1080p(seed=9)
    x = to_dev(s.image)
    ctx = fv.Context(1920, 1080, 3, 32, s.sigma0, s.k, fv.U8_HWC)
    outs = []
    for rb in ((16,) if tc == 3 else (16, 32) if tc == 2 else (16, 32, 64)):
        for ctas in (1, 2, 0):
            ctx.set_config(256, ctas, rb, tensor_cores=tc)
            y = torch.empty_like(x)
            ctx.render(x, y, s.fix_x, s.fix_y)
            outs.append(y)
    torch.cuda.synchronize()
    for y in outs[1:]:
        assert torch.equal(y, outs[0])
    if tc == 1:
        # 128 and 512 threads cut the halo tile into narrower / wider column
        # slabs, which regroups pass 2's fp32 sums: within 1 LSB, nearly all
        # equal; within one thread count the chunk and CTA count change nothing
        for nt in (128, 512):
            outs_nt = []
            for rb in (16, 64):
                for ctas in (1, 0):
                    ctx.set_config(nt, ctas, rb, tensor_cores=1)
                    y = torch.empty_like(x)
                    ctx.render(x, y, s.fix_x, s.fix_y)
                    outs_nt.append(y)
            torch.cuda.synchronize()
            for y in outs_nt[1:]:
                assert torch.equal(y, outs_nt[0])
            assert_u8_close(outs_nt[0].cpu().numpy(), outs[0].cpu().numpy(), min_equal=0.999)
    cfg = ctx.autotune(iters=3)
    assert cfg["rows_per_chunk"] in (16, 32, 64) and cfg["threads"] in (128, 256, 512)


# ---------------------------------------------------------------- argument errors

def test_argument_errors(fv):
    x = torch.zeros((64, 64, 3), dtype=torch.uint8, device="cuda")
    ctx = fv.Context(64, 64, 3, 32, 0.5, 0.02, fv.U8_HWC)
    with pytest.raises(fv.FoveaError) as e:
        ctx.render(x, x, 10.0, 10.0)  # aliasing
    assert e.value.status == fv.EINVAL
    with pytest.raises(fv.FoveaError) as e:
        ctx.render(x, torch.empty_like(x), float("nan"), 1.0)
    assert e.value.status == fv.EINVAL
    big = fv.Context(64, 64, 3, 32, 0.5, 20.0, fv.U8_HWC)  # radius far above the maximum
    with pytest.raises(fv.FoveaError) as e:
        big.render(x, torch.empty_like(x), 0.0, 0.0)
    assert e.value.status == fv.EUNSUPPORTED


# ---------------------------------------------------------------- tensor-core kernel vs fp32 kernel

@pytest.mark.parametrize("tc,threads", [(1, 256), (2, 256), (3, 256), (1, 128), (1, 512)])
@pytest.mark.parametrize("W,H,C,B,fx,fy,k", [
    (1920, 1080, 3, 32, 960.0, 540.0, 0.02),
    (333, 221, 1, 32, 10.0, 200.0, 0.1),
    (640, 480, 4, 16, 600.0, 30.0, 0.3),
    (129, 77, 2, 8, 64.0, 38.0, 0.05),
    (256, 200, 3, 32, 250.0, 10.0, 0.7),
])
def test_tensor_core_kernel_matches_fp32_kernel(fv, W, H, C, B, fx, fy, k, tc, threads):
    """The tensor-core kernels (1: mma.sync with 128, 256 or 512 threads;
    2: vertical pass on tcgen05; 3: both passes on tcgen05, RGB frames; the
    other channel counts fall back to 1) against the fp32 FMA kernel and the
    oracle; the last case has radii above the bound of kernel 2, which falls
    back to mma.sync."""
    img = wl.grating_frame(H, W, C, seed=W + C)
    x = to_dev(img)
    ctx = fv.Context(W, H, C, B, 0.5, k, fv.U8_HWC)
    ctx.set_config(256, 0, 32, tensor_cores=0)
    y32 = torch.empty_like(x)
    ctx.render(x, y32, fx, fy)
    ctx.set_config(threads, 0, 16 if tc == 3 else 32, tensor_cores=tc)
    ytc = torch.empty_like(x)
    ctx.render(x, ytc, fx, fy)
    torch.cuda.synchronize()
    assert_u8_close(ytc.cpu().numpy(), y32.cpu().numpy(), min_equal=0.995)
    blocks = sample_blocks(W, H, B, fx, fy, n_random=16, seed=3)
    ref = oracle.forward_u8(img, B, fx, fy, 0.5, k, "hwc", blocks=blocks)
    assert_u8_close(ytc.cpu().numpy(), ref, mask=block_mask(W, H, B, blocks, "hwc", C), min_equal=0.995)


# ---------------------------------------------------------------- FP32 FMA roof probe

def test_measured_fma_rate_is_plausible(fv):
    rate = fv.measure_fma_rate()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # at most 128 FP32 lanes per SM at a clock of at most 3 GHz; at least a
    # tenth of that at 1 GHz
    assert 0.1 * sms * 128 * 1e9 < rate < sms * 128 * 3e9
