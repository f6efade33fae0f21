"""GPU parity of the float32 tensor-core forward kernel (csrc/tcf_forward.cu:
the separable blur of Section 2 / Algorithm 1 on mma.sync with fp16 hi + lo
splits of data and taps) against the FP64 oracle and the fp32 FMA kernel.

Bar: within 1e-5 absolute of the oracle for values in [0, 1) (the split's
representation error is about 2^-21 of |x|), within 1e-5 relative for data
of larger magnitude; frames the kernel cannot load by TMA (W not a multiple
of 4) run the fp32 kernel instead and meet the same bar."""
import numpy as np
import pytest
import torch

import oracle
from paper_2012_08655_gb300 import workloads as wl
from _helpers import assert_f32_close, block_mask, sample_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_08655_gb300 import fovea
    return fovea


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def render_batch_with(fv, frames, tc, block=32):
    """Render (image, fix_x, fix_y, sigma0, k) float32 CHW frames as one batch
    with the given tensor_cores setting; returns the device outputs."""
    ctx = fv.batch_context(block)
    ctx.set_config(256, 0, 32, tensor_cores=tc)
    ins = [to_dev(f[0]) for f in frames]
    outs = [torch.empty_like(x) for x in ins]
    ctx.render_batch([fv.BatchFrame(ins[i], outs[i], *frames[i][1:]) for i in range(len(frames))])
    torch.cuda.synchronize()
    assert ctx.check() == 0
    return outs


CASES = [
    # W, H, C, B, fx, fy, sigma0, k
    (256, 256, 1, 32, 128.0, 128.0, 0.5, 0.02),   # the plain 256 x 256 workload
    (224, 224, 3, 32, 17.0, 200.0, 0.5, 0.08),    # a training image
    (64, 48, 3, 32, 0.0, 0.0, 3.0, 0.5),          # r ~ 100 > W, H: every edge folded
    (96, 80, 3, 32, 5.0, 75.0, 0.5, 0.6),         # r ~ 220: many row chunks
    (300, 200, 2, 16, 290.0, 10.0, 0.4, 0.1),     # ragged blocks, two channels, B = 16
    (1000, 60, 1, 32, 0.0, 30.0, 0.5, 0.3),       # wide halos: several column slabs
    (640, 40, 2, 32, 600.0, 20.0, 0.5, 0.4),      # several slabs in each of two planes
    (128, 96, 4, 8, 64.0, 48.0, 0.0, 0.15),       # sigma0 = 0, B = 8, four channels
    (400, 120, 3, 32, 380.0, 60.0, 0.5, 0.25),    # three planes per pass, several slabs
    (200, 64, 4, 32, 0.0, 32.0, 0.5, 0.3),        # four planes per pass, several slabs
    (4, 1, 1, 32, 2.0, 0.5, 1.0, 0.0),            # one row of four
    (8, 300, 1, 32, 4.0, 0.0, 0.5, 0.05),         # narrow column
    (37, 29, 1, 32, 10.0, 10.0, 0.5, 0.1),        # W not a multiple of 4: the fp32 kernel
]


@pytest.mark.parametrize("W,H,C,B,fx,fy,s0,k", CASES)
def test_tcf_matches_oracle_and_fp32_kernel(fv, W, H, C, B, fx, fy, s0, k):
    img = wl.uniform_f32((C, H, W), seed=W * 3 + H + C)
    frames = [(img, fx, fy, s0, k)]
    y_tc, = render_batch_with(fv, frames, 1, B)
    y32, = render_batch_with(fv, frames, 0, B)
    ref = oracle.forward(img, B, fx, fy, s0, k, "chw")
    assert_f32_close(y_tc.cpu().numpy(), ref)
    assert_f32_close(y_tc.cpu().numpy(), y32.cpu().numpy(), atol=2e-6)
    if s0 == 0.0 and k == 0.0:
        assert torch.equal(y_tc.cpu(), torch.from_numpy(img))


def test_tcf_signed_data_of_larger_magnitude(fv):
    """Standard-normal data times 1000 (signed, |x| up to a few thousand):
    relative 1e-5 of the frame's scale."""
    g = wl.rng(11)
    img = (g.standard_normal((3, 120, 160)) * 1000.0).astype(np.float32)
    y, = render_batch_with(fv, [(img, 40.0, 100.0, 0.5, 0.2)], 1)
    ref = oracle.forward(img, 32, 40.0, 100.0, 0.5, 0.2, "chw")
    err = np.abs(y.cpu().numpy().astype(np.float64) - ref) / 1000.0
    assert err.max() <= 1e-5, f"relative error {err.max():.3e}"


def test_tcf_mixed_batch_and_single_frame_agree(fv):
    """Frames of several sizes and channel counts in one tensor-core launch
    (one plane per slab pass); a frame too large for one wave also renders
    alone through fovea_render (its three planes together in each pass), bit
    for bit equal to a batch of that frame alone (same kernel, same sigma)
    and within 2e-6 of its output in the mixed batch (other slab widths
    regroup the fp32 sums)."""
    frames = [(wl.uniform_f32((3, 1080, 1920), seed=1), 700.5, 300.25, 0.5, 0.02),
              (wl.uniform_f32((1, 256, 256), seed=2), 128.0, 128.0, 0.5, 0.02),
              (wl.uniform_f32((3, 224, 224), seed=3), 200.0, 15.0, 0.5, 0.08),
              (wl.uniform_f32((2, 480, 640), seed=4), -30.0, 240.0, 0.3, 0.05)]
    outs = render_batch_with(fv, frames, 1)
    for (img, fx, fy, s0, k), y in zip(frames, outs):
        C, H, W = img.shape
        blocks = sample_blocks(W, H, 32, fx, fy, n_random=8, seed=W)
        ref = oracle.forward(img, 32, fx, fy, s0, k, "chw", blocks=blocks)
        assert_f32_close(y.cpu().numpy(), ref, mask=block_mask(W, H, 32, blocks, "chw", C))
    img, fx, fy, s0, k = frames[0]
    ctx = fv.Context(1920, 1080, 3, 32, s0, k, fv.F32_CHW)
    ctx.set_config(256, 0, 32, tensor_cores=1)
    x = to_dev(img)
    y = torch.empty_like(x)
    ctx.render(x, y, fx, fy)
    torch.cuda.synchronize()
    assert ctx.check() == 0
    alone, = render_batch_with(fv, frames[:1], 1)
    assert torch.equal(y, alone)
    assert float((y - outs[0]).abs().max()) <= 2e-6


@pytest.mark.parametrize("bad", [32760.0, -40000.0, float("nan"), float("-inf")])
def test_tcf_value_out_of_range_is_reported(fv, bad):
    """A staged value the fp16 split cannot carry (|x| >= 32760, which fp16
    rounds to 2^15 or more, or not finite) sets FOVEA_FAULT_VALUE_RANGE:
    fovea_check reports EINVAL (the caller's data); 32759 does not, and the
    context stays usable."""
    img = wl.uniform_f32((1, 64, 64), seed=5)
    ctx = fv.batch_context(32)
    ctx.set_config(256, 0, 32, tensor_cores=1)
    x = to_dev(img)
    y = torch.empty_like(x)
    img[0, 10, 20] = -32759.0
    x.copy_(torch.from_numpy(img))
    ctx.render_batch([fv.BatchFrame(x, y, 32.0, 32.0, 0.5, 0.1)])
    torch.cuda.synchronize()
    assert ctx.check() == 0
    img[0, 10, 20] = bad
    x.copy_(torch.from_numpy(img))
    ctx.render_batch([fv.BatchFrame(x, y, 32.0, 32.0, 0.5, 0.1)])
    with pytest.raises(fv.FoveaError) as e:
        ctx.check()
    assert e.value.status == fv.EINVAL and e.value.faults == fv.FAULT_VALUE_RANGE
    img[0, 10, 20] = 0.5
    x.copy_(torch.from_numpy(img))
    ctx.render_batch([fv.BatchFrame(x, y, 32.0, 32.0, 0.5, 0.1)])
    torch.cuda.synchronize()
    assert ctx.check() == 0
    assert_f32_close(y.cpu().numpy(), oracle.forward(img, 32, 32.0, 32.0, 0.5, 0.1, "chw"))


def test_tcf_training_forward_matches_fp32_kernel(fv):
    """The training batch (32 x 3 x 224 x 224) through foveate_train's
    forward on the default configuration (tensor cores on) against the fp32
    kernel and, on sampled blocks of two images, the oracle."""
    x_np, fix_np, s0, k = wl.train_batch(seed=5)
    x = to_dev(x_np)
    fix = torch.from_numpy(fix_np)
    y = fv.foveate_train(x, fix, s0, k)
    b = fv._batch_ctx(32)
    cfg = b.get_config()
    try:
        b.set_config(256, 0, 32, tensor_cores=0)
        y32 = fv.foveate_train(x, fix, s0, k)
    finally:
        b.set_config(cfg["threads"], cfg["ctas_per_sm"], cfg["rows_per_chunk"], cfg["tensor_cores"])
    torch.cuda.synchronize()
    assert float((y - y32).abs().max()) <= 2e-6
    for i in (0, 31):
        fx, fy = float(fix_np[i, 0]), float(fix_np[i, 1])
        blocks = sample_blocks(224, 224, 32, fx, fy, n_random=6, seed=i)
        ref = oracle.forward(x_np[i], 32, fx, fy, s0, k, "chw", blocks=blocks)
        assert_f32_close(y[i].cpu().numpy(), ref, mask=block_mask(224, 224, 32, blocks, "chw", 3))


def test_float32_batch_autotune_stays_within_the_bar(fv):
    """The batch autotuner times the float32 tensor-core kernel beside the
    fp32 kernel's row chunks; whichever it keeps renders within the bar."""
    frames = [(wl.uniform_f32((3, 224, 224), seed=40 + i), 20.0 + 40 * i, 200.0 - 30 * i, 0.5, 0.08)
              for i in range(6)]
    ins = [to_dev(f[0]) for f in frames]
    outs = [torch.empty_like(x) for x in ins]
    batch = [fv.BatchFrame(ins[i], outs[i], *frames[i][1:]) for i in range(len(frames))]
    ctx = fv.batch_context(32)
    cfg = ctx.autotune_batch(batch, iters=2)
    assert cfg["tensor_cores"] in (0, 1)
    ctx.render_batch(batch)
    torch.cuda.synchronize()
    assert ctx.check() == 0
    for (img, fx, fy, s0, k), y in zip(frames, outs):
        assert_f32_close(y.cpu().numpy(), oracle.forward(img, 32, fx, fy, s0, k, "chw"))
