"""The batch autotuner (fovea_autotune_batch) on a mixed batch of uint8 RGB
frames: it times the configurations (kernel, threads per CTA, rows per
chunk, CTAs per SM) on the batch itself, later batches of the same kind
render with the chosen one, and the results stay within the forward path's
bars (1 LSB of the FP64 oracle on sampled blocks, and of the default
configuration's output). Runs after the other GPU tests of the forward path
(file order), since the choice is cached for the whole process."""
import numpy as np
import pytest
import torch

import oracle
from paper_2012_08655_gb300 import workloads as wl
from _helpers import assert_u8_close, block_mask, sample_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_08655_gb300 import fovea
    return fovea


SIZES = [(640, 480), (1280, 720), (1920, 1080), (1920, 1080), (3840, 2160), (200, 130)]


def _batch(fv, seed):
    g = wl.rng(seed)
    frames, imgs = [], []
    for i, (w, h) in enumerate(SIZES):
        img = wl.grating_frame(h, w, 3, seed=seed + i)
        x = torch.from_numpy(img).cuda()
        fx, fy = float(np.float32(g.uniform(0, w))), float(np.float32(g.uniform(0, h)))
        k = float(g.uniform(0.01, 0.04))
        frames.append(fv.BatchFrame(x, torch.empty_like(x), fx, fy, 0.5, k))
        imgs.append(img)
    return frames, imgs


def test_batch_autotune_choice_is_used_and_stays_within_the_bars(fv):
    frames, imgs = _batch(fv, 300)
    ctx = fv.batch_context(32)
    ref = fv.batch_context(32)
    ref.set_config(256, 0, 32, tensor_cores=1)        # an explicit configuration: never the tuned one
    ref_frames = []
    for f in frames:
        y = torch.empty_like(f.out)
        ref_frames.append(fv.BatchFrame(f.inp, y, f.fix_x, f.fix_y, f.sigma0, f.k))
    ref.render_batch(ref_frames)
    cfg = ctx.autotune_batch(frames, iters=2)
    assert cfg["threads"] in (128, 256, 512) and cfg["rows_per_chunk"] in (16, 32, 64)
    assert cfg["tensor_cores"] in (0, 1, 2) and 0 <= cfg["ctas_per_sm"] <= 2
    # a later batch of the same kind (same sizes, other fixations within the
    # same radius bucket) renders with the tuned configuration
    for f in frames:
        f.out.zero_()
    ctx.render_batch(frames)
    ctx.check()
    torch.cuda.synchronize()
    for i, (f, r, img) in enumerate(zip(frames, ref_frames, imgs)):
        assert_u8_close(f.out.cpu().numpy(), r.out.cpu().numpy(), min_equal=0.999)
        h, w = img.shape[:2]
        blocks = sample_blocks(w, h, 32, f.fix_x, f.fix_y, n_random=6, seed=i)
        want = oracle.forward_u8(img, 32, f.fix_x, f.fix_y, f.sigma0, f.k, "hwc", blocks=blocks)
        assert_u8_close(f.out.cpu().numpy(), want, mask=block_mask(w, h, 32, blocks, "hwc", 3), min_equal=0.99)
    # asking again keeps the cached choice
    assert ctx.autotune_batch(frames, iters=2) == cfg


def test_explicit_configuration_wins_over_the_tuned_one(fv):
    frames, _ = _batch(fv, 300)
    ctx = fv.batch_context(32)
    tuned = ctx.autotune_batch(frames, iters=1)   # cached by the previous test
    other = {"threads": 512 if tuned["threads"] != 512 else 128, "ctas_per_sm": 0, "rows_per_chunk": 32,
             "tensor_cores": 1}
    ctx.set_config(**other)
    assert ctx.get_config() == other
    ctx.render_batch(frames)
    ctx.check()
