"""GPU parity of the tensor-core adjoint (csrc/tca_adjoint.cu, selected by
tensor_cores = 2: the transpose of Section 2 / Algorithm 1's block-wise blur
on mma.sync, a power-of-two scale per block plane, fp16 hi + lo splits)
against the FP64 oracle's adjoint and the fp32 adjoint kernel (the default,
with vector reductions into grad_in).

Bar: error within 1e-5 of max(|reference|, the gradient's scale) per pixel
(the split's error is about 2^-21 of the block's largest |g|), at gradient
scales from 1e-20 to 1e20."""
import numpy as np
import pytest
import torch

import oracle
from paper_2012_08655_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_08655_gb300 import fovea
    return fovea


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def backward_with(fv, ctx, g, fx, fy, tc):
    ctx.set_config(256, 0, 32, tensor_cores=tc)
    gi = torch.full_like(g, float("nan"))  # every pixel must be written (zeroed, then accumulated)
    ctx.backward(g, gi, fx, fy)
    torch.cuda.synchronize()
    assert ctx.check() == 0
    return gi.cpu().numpy().astype(np.float64)


CASES = [
    # W, H, C, B, fx, fy, sigma0, k, gradient scale
    (224, 224, 3, 32, 17.0, 200.0, 0.5, 0.08, 1.0),     # a training image
    (64, 48, 3, 32, 0.0, 0.0, 3.0, 0.5, 1.0),           # r ~ 100 > W, H: every edge folded
    (96, 80, 3, 32, 5.0, 75.0, 0.5, 0.6, 1.0),          # r ~ 220: many row tiles
    (1000, 60, 1, 32, 0.0, 30.0, 0.5, 0.3, 1.0),        # halos wider than one 256-column slab
    (300, 200, 2, 16, 290.0, 10.0, 0.4, 0.1, 1e-20),    # tiny gradients, B = 16
    (128, 96, 4, 8, 64.0, 48.0, 0.0, 0.15, 1e20),       # huge gradients, sigma0 = 0, B = 8
    (37, 29, 1, 32, 10.0, 10.0, 0.5, 0.1, 1.0),         # ragged, one partial block
    (1, 1, 1, 32, 0.5, 0.5, 1.0, 0.0, 1.0),             # 1 x 1
    (8, 300, 1, 32, 4.0, 0.0, 0.5, 0.05, 1.0),          # narrow column
    (200, 64, 4, 64, 0.0, 32.0, 0.5, 0.3, 1.0),         # B = 64
]


@pytest.mark.parametrize("W,H,C,B,fx,fy,s0,k,scale", CASES)
def test_tca_adjoint_matches_oracle_and_fp32_adjoint(fv, W, H, C, B, fx, fy, s0, k, scale):
    g_np = ((2.0 * wl.uniform_f32((C, H, W), seed=W + 7 * H + C) - 1.0) * scale).astype(np.float32)
    g = to_dev(g_np)
    ctx = fv.Context(W, H, C, B, s0, k, fv.F32_CHW)
    gi_tc = backward_with(fv, ctx, g, fx, fy, 2)
    gi_32 = backward_with(fv, ctx, g, fx, fy, 0)
    ref = oracle.adjoint(g_np, B, fx, fy, s0, k, "chw")
    assert np.all(np.isfinite(gi_tc))
    den = np.maximum(np.abs(ref), scale)
    assert float((np.abs(gi_tc - ref) / den).max()) <= 1e-5
    assert float((np.abs(gi_tc - gi_32) / den).max()) <= 1e-5


def test_tca_adjoint_zero_planes_and_mixed_scales(fv):
    """A plane of zeros contributes nothing; planes of very different scale
    are scaled independently (each keeps its own relative error)."""
    W, H = 160, 96
    g_np = np.zeros((3, H, W), np.float32)
    g_np[1] = wl.uniform_f32((H, W), seed=1) * 1e-12
    g_np[2] = wl.uniform_f32((H, W), seed=2) * 1e6
    g = to_dev(g_np)
    ctx = fv.Context(W, H, 3, 32, 0.5, 0.1, fv.F32_CHW)
    gi = backward_with(fv, ctx, g, 40.0, 50.0, 2)
    ref = oracle.adjoint(g_np, 32, 40.0, 50.0, 0.5, 0.1, "chw")
    assert np.all(gi[0] == 0.0)
    for c, scale in ((1, 1e-12), (2, 1e6)):
        assert float((np.abs(gi[c] - ref[c]) / np.maximum(np.abs(ref[c]), scale)).max()) <= 1e-5


def test_tca_adjoint_training_batch_matches_fp32_adjoint(fv):
    """The training batch's backward (batched adjoint launch) on the tensor
    cores (tensor_cores = 2) against the fp32 adjoint (the default) and, for
    two images, the oracle."""
    x_np, fix_np, s0, k = wl.train_batch(seed=3)
    g_np = wl.uniform_f32(x_np.shape, seed=9)
    g = to_dev(g_np)
    b = fv.batch_context(32)
    outs = {}
    for tc in (2, 0):
        b.set_config(256, 0, 32, tensor_cores=tc)
        gi = torch.empty_like(g)
        frames = [fv.BatchFrame(g[i], gi[i], float(fix_np[i, 0]), float(fix_np[i, 1]), s0, k)
                  for i in range(g.shape[0])]
        b.backward_batch(frames)
        torch.cuda.synchronize()
        assert b.check() == 0
        outs[tc] = gi.cpu().numpy().astype(np.float64)
    # edge pixels collect the folded mass of many clamped taps (values up to
    # ~40 here): the bar is relative, as in the other gradient tests
    assert float((np.abs(outs[2] - outs[0]) / np.maximum(1.0, np.abs(outs[0]))).max()) <= 1e-5
    for i in (0, 31):
        ref = oracle.adjoint(g_np[i], 32, fix_np[i, 0], fix_np[i, 1], s0, k, "chw")
        for tc in (2, 0):
            assert float((np.abs(outs[tc][i] - ref) / np.maximum(1.0, np.abs(ref))).max()) <= 1e-5
