"""GPU parity of the batched, differentiable and served forms against the
FP64 oracle (and against the single-frame path), through the C ABI."""
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


# ---------------------------------------------------------------- mixed batch

def test_mixed_batch_full_size(fv):
    """The 64-frame mixed batch (16 VGA, 16 720p, 24 1080p, 8 4K) in one
    batched launch: sampled blocks of a subset of frames against the oracle,
    and every frame equal to the single-frame path bit for bit."""
    frames = wl.mixed_batch(seed=0)
    ins = [to_dev(f.image) for f in frames]
    outs = [torch.empty_like(x) for x in ins]
    fv.foveate_batch([fv.BatchFrame(ins[i], outs[i], f.fix_x, f.fix_y, f.sigma0, f.k)
                      for i, f in enumerate(frames)])
    torch.cuda.synchronize()
    for i in [0, 17, 40, 56, 63]:
        f = frames[i]
        single = fv.foveate(ins[i], f.fix_x, f.fix_y, f.sigma0, f.k)
        torch.cuda.synchronize()
        assert torch.equal(single, outs[i]), f"frame {i}: batch differs from single-frame render"
        blocks = sample_blocks(f.width, f.height, 32, f.fix_x, f.fix_y, n_random=12, seed=i)
        ref = oracle.forward_u8(f.image, 32, f.fix_x, f.fix_y, f.sigma0, f.k, "hwc", blocks=blocks)
        assert_u8_close(outs[i].cpu().numpy(), ref, mask=block_mask(f.width, f.height, 32, blocks, "hwc", 3),
                        min_equal=0.99)


@pytest.mark.parametrize("tc,threads", [(1, 256), (1, 128), (1, 512), (2, 256), (3, 256)])
def test_batch_mixing_tma_and_plain_frames(fv, tc, threads):
    """uint8 RGB frames of one batch whose rows TMA can load (16-byte
    aligned pitch) and whose rows it cannot (odd pitch: plain loads), in
    alternation, on both tensor-core kernels and every thread count: every
    frame within 1 LSB of the oracle and no device fault. (Plain-loaded items
    must not advance the TMA ring's phase count.)"""
    sizes = [(640, 480), (33, 65), (480, 320), (101, 77), (1280, 720), (7, 300), (224, 224)]
    g = wl.rng(77)
    frames, imgs = [], []
    for i, (w, h) in enumerate(sizes):
        img = wl.grating_frame(h, w, 3, seed=90 + i)
        x = to_dev(img)
        fx, fy = float(np.float32(g.uniform(0, w))), float(np.float32(g.uniform(0, h)))
        frames.append(fv.BatchFrame(x, torch.empty_like(x), fx, fy, 0.5, 0.03))
        imgs.append(img)
    ctx = fv.batch_context(32)
    ctx.set_config(threads, 0, 16 if tc == 3 else 32, tensor_cores=tc)
    for rep in range(2):  # the second launch starts from the barrier phases the first one left
        for f in frames:
            f.out.zero_()
        ctx.render_batch(frames)
        assert ctx.check() == 0
    torch.cuda.synchronize()
    for i, (f, img) in enumerate(zip(frames, imgs)):
        h, w = img.shape[:2]
        blocks = sample_blocks(w, h, 32, f.fix_x, f.fix_y, n_random=8, seed=i)
        ref = oracle.forward_u8(img, 32, f.fix_x, f.fix_y, 0.5, 0.03, "hwc", blocks=blocks)
        assert_u8_close(f.out.cpu().numpy(), ref, mask=block_mask(w, h, 32, blocks, "hwc", 3), min_equal=0.99)


def test_batch_of_mixed_formats_and_channels(fv):
    """A batch mixing uint8 HWC (1 and 3 channels) and float32 CHW frames of
    ragged sizes, checked frame by frame against the oracle."""
    specs = [
        ("u8", 84, 84, 1, 40.0, 44.0, 0.5, 0.02),
        ("u8", 224, 224, 3, 10.0, 200.0, 0.5, 0.03),
        ("f32", 70, 45, 2, 35.0, 22.5, 0.2, 0.1),
        ("u8", 129, 33, 4, 128.0, 0.0, 0.5, 0.05),
        ("f32", 31, 97, 3, -5.0, 120.0, 0.0, 0.2),
    ]
    batch, imgs = [], []
    for i, (dt, W, H, C, fx, fy, s0, k) in enumerate(specs):
        img = wl.uniform_u8((H, W, C), seed=i) if dt == "u8" else wl.uniform_f32((C, H, W), seed=i)
        x = to_dev(img)
        batch.append(fv.BatchFrame(x, torch.empty_like(x), fx, fy, s0, k))
        imgs.append(img)
    fv.foveate_batch(batch)
    torch.cuda.synchronize()
    for (dt, W, H, C, fx, fy, s0, k), img, bf in zip(specs, imgs, batch):
        if dt == "u8":
            assert_u8_close(bf.out.cpu().numpy(), oracle.forward_u8(img, 32, fx, fy, s0, k, "hwc"), min_equal=0.98)
        else:
            assert_f32_close(bf.out.cpu().numpy(), oracle.forward(img, 32, fx, fy, s0, k, "chw"))


def test_consecutive_batches_with_new_buffers(fv):
    """Back-to-back batches of the same shape through one batch context, each
    on freshly allocated frames (the per-frame descriptors, tensor maps
    included, are rewritten in place between launches): every frame equals
    its single-frame render."""
    shapes = [(224, 224), (640, 480), (1280, 720), (224, 224), (1920, 1080)]
    for rnd in range(4):
        ins = [torch.from_numpy(wl.grating_frame(h, w, 3, seed=100 * rnd + i)).cuda()
               for i, (w, h) in enumerate(shapes)]
        outs = [torch.empty_like(x) for x in ins]
        fix = [(0.25 * w + 17.0 * rnd, 0.6 * h) for (w, h) in shapes]
        fv.foveate_batch([fv.BatchFrame(ins[i], outs[i], fix[i][0], fix[i][1], 0.5, 0.03) for i in range(len(ins))])
        torch.cuda.synchronize()
        for i in range(len(ins)):
            single = fv.foveate(ins[i], fix[i][0], fix[i][1], 0.5, 0.03)
            torch.cuda.synchronize()
            assert torch.equal(single, outs[i]), f"round {rnd} frame {i}: batch differs from single-frame render"


def test_batch_buffers_grow_while_earlier_batches_are_queued(fv):
    """A fresh batch context given ever larger batches back to back on one
    stream, with no synchronisation between them: each launch outgrows the
    item workspace or the batch table, so the buffers the queued launches
    read are replaced (and kept) while those launches are still pending.
    Every frame equals its single-frame render; a context whose buffers were
    reserved up front renders the same bytes."""
    shapes = [(84, 84), (224, 224), (640, 480), (1280, 720), (1920, 1080), (3840, 2160)]
    jobs = []
    for n in (1, 3, 9, 24):
        ins = [torch.from_numpy(wl.grating_frame(shapes[i % 6][1], shapes[i % 6][0], 3, seed=7 * n + i)).cuda()
               for i in range(n)]
        fix = [(0.3 * x.shape[1] + n, 0.55 * x.shape[0]) for x in ins]
        jobs.append((ins, fix))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    grown, reserved = fv.batch_context(32), fv.batch_context(32)
    reserved.reserve(64, 1 << 20)
    results = []
    with torch.cuda.stream(stream):
        for ins, fix in jobs:
            outs = [torch.empty_like(x) for x in ins]
            grown.render_batch([fv.BatchFrame(x, o, f[0], f[1], 0.5, 0.02) for x, o, f in zip(ins, outs, fix)],
                               stream)
            outs_r = [torch.empty_like(x) for x in ins]
            reserved.render_batch([fv.BatchFrame(x, o, f[0], f[1], 0.5, 0.02) for x, o, f in zip(ins, outs_r, fix)],
                                  stream)
            results.append((outs, outs_r))
    stream.synchronize()
    for (ins, fix), (outs, outs_r) in zip(jobs, results):
        for i, x in enumerate(ins):
            single = fv.foveate(x, fix[i][0], fix[i][1], 0.5, 0.02)
            torch.cuda.synchronize()
            assert torch.equal(single, outs[i]), f"batch of {len(ins)}, frame {i}: differs after growth"
            assert torch.equal(single, outs_r[i]), f"batch of {len(ins)}, frame {i}: differs with reserved buffers"
    grown.close()
    reserved.close()


# ---------------------------------------------------------------- differentiable form

def test_train_batch_forward_backward_vs_oracle(fv):
    """32 x 3 x 224 x 224 float32 with random fixations, sigma = 0.5 + 0.08 e:
    forward and input gradient of 4 images against the oracle and its adjoint."""
    x, fix, s0, k = wl.train_batch(seed=0)
    xt = to_dev(x).requires_grad_(True)
    y = fv.foveate_train(xt, torch.from_numpy(fix), s0, k)
    g = wl.uniform_f32(x.shape, seed=5)
    y.backward(to_dev(g))
    torch.cuda.synchronize()
    for i in [0, 7, 19, 31]:
        fo = oracle.forward(x[i], 32, fix[i, 0], fix[i, 1], s0, k, "chw")
        assert_f32_close(y[i].detach().cpu().numpy(), fo)
        go = oracle.adjoint(g[i], 32, fix[i, 0], fix[i, 1], s0, k, "chw")
        got = xt.grad[i].cpu().numpy()
        # Absolute 1e-5 where the gradient is O(1); relative 1e-5 on the edge
        # pixels that collect the folded mass of many clamped taps.
        err = np.abs(got - go) / np.maximum(1.0, np.abs(go))
        assert err.max() <= 1e-5, f"image {i}: gradient error {err.max():.3e}"


@pytest.mark.parametrize("B", [32, 4])
def test_gradient_matches_fp64_finite_differences_on_crops(fv, B):
    """16x16x3 crops of the training batch as standalone images (fixation
    moved into crop coordinates, same sigma law): the backward kernel against
    FP64 central finite differences of L(x) = <A x, g> over all 768 inputs."""
    x, fix, s0, k = wl.train_batch(seed=0, n=2)
    g = wl.uniform_f32((3, 16, 16), seed=8).astype(np.float64)
    for i, (cy, cx) in enumerate([(100, 60), (0, 208)]):
        crop = np.ascontiguousarray(x[i, :, cy:cy + 16, cx:cx + 16])
        fx, fy = float(np.float32(fix[i, 0] - cx)), float(np.float32(fix[i, 1] - cy))
        h = 1e-3
        base = crop.astype(np.float64)
        fd = np.zeros_like(base)
        for idx in np.ndindex(base.shape):
            p, m = base.copy(), base.copy()
            p[idx] += h
            m[idx] -= h
            lp = np.sum(oracle.forward(p, B, fx, fy, s0, k, "chw", nthreads=1) * g)
            lm = np.sum(oracle.forward(m, B, fx, fy, s0, k, "chw", nthreads=1) * g)
            fd[idx] = (lp - lm) / (2 * h)
        xt = to_dev(crop[None]).requires_grad_(True)
        y = fv.foveate_train(xt, torch.tensor([[fx, fy]]), s0, k, block=B)
        y.backward(to_dev(g[None].astype(np.float32)))
        torch.cuda.synchronize()
        assert_f32_close(xt.grad[0].cpu().numpy(), fd, atol=1e-5)


def test_adjoint_identity_on_gpu(fv):
    g = wl.rng(3)
    x = g.standard_normal((2, 3, 96, 80)).astype(np.float32)
    yv = g.standard_normal((2, 3, 96, 80)).astype(np.float32)
    fix = np.array([[10.0, 90.0], [70.5, -3.0]], np.float32)
    ax = fv.foveate_train(to_dev(x), torch.from_numpy(fix), 0.5, 0.1)
    xt = to_dev(x).requires_grad_(True)
    out = fv.foveate_train(xt, torch.from_numpy(fix), 0.5, 0.1)
    out.backward(to_dev(yv))
    torch.cuda.synchronize()
    lhs = float(np.sum(ax.cpu().numpy().astype(np.float64) * yv))
    rhs = float(np.sum(x.astype(np.float64) * xt.grad.cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-5 * max(1.0, abs(lhs))


def test_single_frame_backward_matches_batch(fv):
    x, fix, s0, k = wl.train_batch(seed=2, n=1, size=100)
    g = to_dev(wl.uniform_f32((3, 100, 100), seed=4))
    ctx = fv.Context(100, 100, 3, 32, s0, k, fv.F32_CHW)
    gi = torch.empty_like(g)
    ctx.backward(g, gi, float(fix[0, 0]), float(fix[0, 1]))
    torch.cuda.synchronize()
    go = oracle.adjoint(g.cpu().numpy(), 32, fix[0, 0], fix[0, 1], s0, k, "chw")
    err = np.abs(gi.cpu().numpy() - go) / np.maximum(1.0, np.abs(go))
    assert err.max() <= 1e-5


# ---------------------------------------------------------------- serving

def test_server_result_alone_equals_result_in_the_mix(fv):
    """Frames served one at a time and the same frames served among a burst of
    other requests give identical outputs (each (format, channels) group is
    its own batch, so a frame always meets the same kernel), within 1 LSB of
    the single-frame path (which may run another kernel configuration)."""
    specs = [(84, 84, 1), (224, 224, 3), (1280, 720, 3), (1920, 1080, 3), (224, 224, 3), (84, 84, 1)]
    frames = []
    for i, (W, H, C) in enumerate(specs):
        img = wl.grating_frame(H, W, C, seed=30 + i)
        frames.append((torch.from_numpy(img).pin_memory(), float(W) * 0.3, float(H) * 0.6))
    with fv.Server(device_budget_bytes=256 << 20, max_batch=16) as srv:
        alone = []
        for inp, fx, fy in frames:
            out = torch.empty_like(inp).pin_memory()
            rid = srv.submit(inp, out, fx, fy, 0.5, 0.02)
            t = srv.wait(rid)
            assert t["status"] == 0 and t["batch_size"] == 1
            alone.append(out)
        # The burst: outputs allocated first so that the submissions follow one
        # another closely, and a 4K frame in front keeps the GPU busy while
        # the rest arrive (the loop launches a request as soon as it can).
        big = torch.from_numpy(wl.grating_frame(2160, 3840, 3, seed=29)).pin_memory()
        big_out = torch.empty_like(big).pin_memory()
        outs = [torch.empty_like(inp).pin_memory() for rep in range(3) for inp, _, _ in frames]
        rids = [srv.submit(big, big_out, 1000.0, 500.0, 0.5, 0.02)]
        for j, out in enumerate(outs):
            inp, fx, fy = frames[j % len(frames)]
            rids.append(srv.submit(inp, out, fx, fy, 0.5, 0.02))
        sizes = [srv.wait(r)["batch_size"] for r in rids][1:]
    assert max(sizes) > 1, "the burst was never batched"
    for j, out in enumerate(outs):
        assert torch.equal(out, alone[j % len(frames)])
    for (inp, fx, fy), out in zip(frames, alone):
        ref = fv.foveate(inp.cuda(), fx, fy, 0.5, 0.02)
        assert_u8_close(out.numpy(), ref.cpu().numpy(), min_equal=0.995)
    inp, fx, fy = frames[1]
    assert_u8_close(alone[1].numpy(), oracle.forward_u8(inp.numpy(), 32, fx, fy, 0.5, 0.02, "hwc"))


def test_server_admission_limits(fv):
    # budget smaller than one 1080p request: refused up front
    with fv.Server(device_budget_bytes=4 << 20, max_batch=4) as srv:
        big = torch.zeros((1080, 1920, 3), dtype=torch.uint8).pin_memory()
        with pytest.raises(fv.FoveaError) as e:
            srv.submit(big, torch.empty_like(big), 5.0, 5.0, 0.5, 0.02)
        assert e.value.status == fv.EBUSY
        # many small requests through a budget that holds only a few at once
        small = [torch.from_numpy(wl.uniform_u8((224, 224, 3), seed=i)).pin_memory() for i in range(12)]
        outs = [torch.empty_like(s) for s in small]
        rids = [srv.submit(s, o, 100.0, 100.0, 0.5, 0.02) for s, o in zip(small, outs)]
        for r in rids:
            assert srv.wait(r, timeout_ms=20000)["status"] == 0
    ref = fv.foveate(small[3].cuda(), 100.0, 100.0, 0.5, 0.02).cpu()
    assert torch.equal(ref, outs[3])


def test_server_holds_request_tensors_until_waited(fv):
    """The binding keeps a request's host tensors alive from submit until wait
    reports it done: a caller that drops its own references right after
    submitting still gets the right result back through the held output."""
    import gc
    img = wl.grating_frame(720, 1280, 3, seed=41)
    ref = fv.foveate(torch.from_numpy(img).cuda(), 400.0, 300.0, 0.5, 0.02).cpu()
    with fv.Server(device_budget_bytes=64 << 20, max_batch=8) as srv:
        rids = []
        for _ in range(4):
            inp = torch.from_numpy(img.copy()).pin_memory()
            out = torch.empty_like(inp).pin_memory()
            rids.append(srv.submit(inp, out, 400.0, 300.0, 0.5, 0.02))
            del inp, out
        gc.collect()
        held = [srv._held[r][1] for r in rids]
        for r in rids:
            assert srv.wait(r, timeout_ms=20000)["status"] == 0
        assert not srv._held
    for out in held:
        assert torch.equal(out, ref)


def test_server_request_log(fv, tmp_path):
    """Server(log_path=...) appends one JSON line per finished request: id,
    frame shape, fixation and the library's timestamps and status."""
    import json
    path = tmp_path / "served.jsonl"
    specs = [(84, 84, 1), (224, 224, 3), (1280, 720, 3)]
    with fv.Server(device_budget_bytes=64 << 20, max_batch=8, log_path=str(path)) as srv:
        rids = []
        for i, (W, H, C) in enumerate(specs):
            inp = torch.from_numpy(wl.grating_frame(H, W, C, seed=70 + i)).pin_memory()
            rids.append(srv.submit(inp, torch.empty_like(inp).pin_memory(), W / 2.0, H / 3.0, 0.5, 0.02))
        times = [srv.wait(r) for r in rids]
    recs = [json.loads(l) for l in path.read_text().splitlines()]
    assert [r["id"] for r in recs] == rids
    for rec, t, (W, H, C) in zip(recs, times, specs):
        assert (rec["width"], rec["height"], rec["channels"]) == (W, H, C)
        assert rec["status"] == 0 and rec["done_us"] == t["done_us"] >= rec["start_us"] >= rec["admit_us"]
