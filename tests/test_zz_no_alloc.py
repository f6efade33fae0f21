"""fovea_render_noalloc, the entry point for callers that cannot allocate GPU
memory (their device memory belongs to a host framework or a server, or they
must not allocate while driving the GPU): through the C ABI, two calls in a
row must give what the ordinary fovea_render entry point gives, within the
tolerances of the other parity tests (uint8: 1 LSB; float32: 1e-5).

This file is named to run last, so a run that stops at the first failure has
already run every other test; it passes alone in a fresh process too."""
import ctypes

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


def _noalloc(fv, x, y, W, H, C, fmt, B, s0, k, fx, fy):
    st = fv._lib.fovea_render_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), W, H, C, fmt, B,
                                      s0, k, fx, fy, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, fv._lib.fovea_strerror(st)


def test_noalloc_matches_render_u8_two_calls(fv):
    W, H, C, B, s0, k = 1920, 1080, 3, 32, 0.5, 0.02
    ctx = fv.Context(W, H, C, B, s0, k, fv.U8_HWC)
    for call, (seed, fx, fy) in enumerate([(21, 960.0, 540.0), (22, 100.5, 1000.25)]):
        img = wl.grating_frame(H, W, C, seed=seed)
        x = torch.from_numpy(img).cuda()
        ref = torch.empty_like(x)
        ctx.render(x, ref, fx, fy)
        y = torch.full_like(x, 7)
        _noalloc(fv, x, y, W, H, C, fv.U8_HWC, B, s0, k, fx, fy)
        assert fv.noalloc_check() == 0  # no device fault in this call
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert_u8_close(got, ref.cpu().numpy(), min_equal=0.995)
        # and directly against the FP64 oracle on sampled blocks (corners,
        # ragged bottom row, the fixation block, random blocks)
        blocks = sample_blocks(W, H, B, fx, fy, n_random=24, seed=call)
        want = oracle.forward_u8(img, B, fx, fy, s0, k, "hwc", blocks=blocks)
        mask = block_mask(W, H, B, blocks, "hwc", C)
        assert_u8_close(got, want, mask=mask, min_equal=0.995)


def test_noalloc_matches_render_f32_two_calls(fv):
    C, H, W, B, s0, k = 3, 224, 224, 32, 0.5, 0.08
    ctx = fv.Context(W, H, C, B, s0, k, fv.F32_CHW)
    for call, (seed, fx, fy) in enumerate([(5, 20.0, 200.0), (6, 111.5, 3.25)]):
        x = torch.from_numpy(wl.uniform_f32((C, H, W), seed=seed)).cuda()
        ref = torch.empty_like(x)
        ctx.render(x, ref, fx, fy)
        y = torch.full_like(x, -1.0)
        _noalloc(fv, x, y, W, H, C, fv.F32_CHW, B, s0, k, fx, fy)
        assert fv.noalloc_check() == 0
        torch.cuda.synchronize()
        assert_f32_close(y.cpu().numpy(), ref.cpu().numpy())
        assert_f32_close(y.cpu().numpy(), oracle.forward(x.cpu().numpy(), B, fx, fy, s0, k, "chw"))


def test_noalloc_refuses_frames_beyond_its_scratch(fv):
    n = 8192 * 8192
    x = torch.zeros(n, dtype=torch.uint8, device="cuda")
    y = torch.zeros(n, dtype=torch.uint8, device="cuda")
    # 8192 x 8192 at B = 32 is 65536 blocks, above FOVEA_NOALLOC_MAX_BLOCKS: refused before any work.
    st = fv._lib.fovea_render_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      8192, 8192, 1, fv.U8_HWC, 32, 0.5, 0.0, 10.0, 10.0, None)
    assert st == fv.EUNSUPPORTED
    # block sides above 32 are refused too (one work item per block)
    st = fv._lib.fovea_render_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      256, 256, 1, fv.U8_HWC, 64, 0.5, 0.0, 10.0, 10.0, None)
    assert st == fv.EUNSUPPORTED
    torch.cuda.synchronize()
    assert int(y.sum().item()) == 0
