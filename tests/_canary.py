"""Guard-band (canary) checks of every output the library writes.

Each output buffer sits between two 4 KiB guard bands filled with the byte
0xA5, inside one larger allocation; after the call the bands must be
untouched and the context's device fault word must be 0. Frames are ragged
(1 x 1, one row, one column, 65 x 33, the 3840 x 2160 frame), some outputs
start at a misaligned address, and every forward kernel and thread count
runs. compute-sanitizer is not available to these tests, so this is the
out-of-bounds evidence for the vectorised 16-byte stores of the persistent
kernels.

`run_cases(fv, torch)` returns a list of failure descriptions. Run as a
script it exits non-zero on any failure: the bounds-checked build of the
library (-DFOVEA_BOUNDS, selected with the FOVEA_LIBRARY environment
variable) is exercised that way in a child process.
"""
import os
import sys

import numpy as np

GUARD = 4096
PATTERN = 0xA5


class Guarded:
    """A tensor of `shape` and `dtype` at byte offset GUARD + skew of a
    buffer whose other bytes hold PATTERN."""

    def __init__(self, torch, shape, dtype, skew=0, device="cuda", pin=False):
        esz = torch.tensor([], dtype=dtype).element_size()
        assert skew % esz == 0
        self.n = int(np.prod(shape)) * esz
        self.lo = GUARD + skew
        buf = torch.full((self.lo + self.n + GUARD,), PATTERN, dtype=torch.uint8)
        self.buf = buf.pin_memory() if pin else buf.to(device)
        self.t = self.buf[self.lo:self.lo + self.n].view(dtype).view(shape)

    def intact(self):
        b = self.buf.cpu().numpy()
        return bool((b[:self.lo] == PATTERN).all() and (b[self.lo + self.n:] == PATTERN).all())


def run_cases(fv, torch):
    from paper_2012_08655_gb300 import workloads as wl
    fails = []
    dev = "cuda"

    def expect(ok, what):
        if not ok:
            fails.append(what)

    def check_ctx(ctx, what):
        try:
            ctx.check()
        except fv.FoveaError as e:
            fails.append(f"{what}: device faults 0x{e.faults:x}")

    u8_shapes = [(1, 1, 3), (1, 300, 1), (300, 1, 1), (65, 33, 3), (33, 65, 4), (2160, 3840, 3)]
    # ---- single-frame uint8 renders: every kernel, the mma.sync kernel at each thread count
    for (h, w, c) in u8_shapes:
        img = wl.grating_frame(h, w, c, seed=h + w) if c == 3 and h > 1 and w > 1 else \
            wl.uniform_u8((h, w, c), seed=h + 3 * w)
        x = torch.from_numpy(img).to(dev)
        ctx = fv.Context(w, h, c, 32, 0.5, 0.04, fv.U8_HWC)
        kinds = [(0, 256), (1, 128), (1, 256), (1, 512), (2, 256), (3, 256)]
        for tc, nt in kinds:
            for skew in (0, 3):
                if (h, w) == (2160, 3840) and skew:
                    continue
                g = Guarded(torch, (h, w, c), torch.uint8, skew)
                ctx.set_config(nt, 0, 16 if tc == 3 else 32, tensor_cores=tc)
                ctx.render(x, g.t, 0.3 * w, 0.6 * h)
                torch.cuda.synchronize()
                expect(g.intact(), f"render u8 {h}x{w}x{c} tc={tc} threads={nt} skew={skew}")
        check_ctx(ctx, f"render u8 {h}x{w}x{c}")
    # ---- single-frame float32 render and adjoint
    for (c, h, w) in [(1, 1, 1), (2, 300, 1), (3, 65, 33), (3, 224, 224)]:
        x = torch.from_numpy(wl.uniform_f32((c, h, w), seed=c + h)).to(dev)
        ctx = fv.Context(w, h, c, 32, 0.5, 0.08, fv.F32_CHW)
        for skew in (0, 4):
            g = Guarded(torch, (c, h, w), torch.float32, skew)
            ctx.render(x, g.t, 0.2 * w, 0.7 * h)
            gb = Guarded(torch, (c, h, w), torch.float32, skew)
            ctx.backward(x, gb.t, 0.2 * w, 0.7 * h)
            torch.cuda.synchronize()
            expect(g.intact(), f"render f32 {c}x{h}x{w} skew={skew}")
            expect(gb.intact(), f"backward f32 {c}x{h}x{w} skew={skew}")
        check_ctx(ctx, f"f32 {c}x{h}x{w}")
    # ---- batches: uint8 (tensor-core kernels), mixed formats, adjoint
    frames, guards = [], []
    for i, (h, w, c) in enumerate([(65, 33, 3), (1, 300, 3), (480, 640, 3), (2160, 3840, 3)]):
        x = torch.from_numpy(wl.grating_frame(h, w, c, seed=50 + i)).to(dev)
        g = Guarded(torch, (h, w, c), torch.uint8, 0 if i % 2 == 0 else 5)
        frames.append(fv.BatchFrame(x, g.t, 0.9 * w, 0.1 * h, 0.5, 0.03))
        guards.append(g)
    bctx = fv.batch_context(32)
    for tc, nt in [(0, 256), (1, 128), (1, 512), (2, 256), (3, 256)]:
        bctx.set_config(nt, 0, 16 if tc == 3 else 32, tensor_cores=tc)
        bctx.render_batch(frames)
        torch.cuda.synchronize()
        for i, g in enumerate(guards):
            expect(g.intact(), f"batch u8 frame {i} tc={tc} threads={nt}")
    mixed, mguards = [], []
    for i, (fmt, shape) in enumerate([(fv.U8_HWC, (31, 17, 1)), (fv.F32_CHW, (2, 40, 9)), (fv.U8_HWC, (7, 300, 4))]):
        if fmt == fv.U8_HWC:
            x = torch.from_numpy(wl.uniform_u8(shape, seed=i)).to(dev)
            g = Guarded(torch, shape, torch.uint8, 1)
        else:
            x = torch.from_numpy(wl.uniform_f32(shape, seed=i)).to(dev)
            g = Guarded(torch, shape, torch.float32, 4)
        mixed.append(fv.BatchFrame(x, g.t, 3.0, 4.0, 0.5, 0.1))
        mguards.append(g)
    bctx.render_batch(mixed)
    adj, aguards = [], []
    for i, shape in enumerate([(3, 33, 65), (1, 1, 1), (2, 224, 100)]):
        x = torch.from_numpy(wl.uniform_f32(shape, seed=20 + i)).to(dev)
        g = Guarded(torch, shape, torch.float32, 4 * i)
        adj.append(fv.BatchFrame(x, g.t, 5.0, 6.0, 0.5, 0.08))
        aguards.append(g)
    bctx.backward_batch(adj)
    torch.cuda.synchronize()
    for i, g in enumerate(mguards):
        expect(g.intact(), f"mixed batch frame {i}")
    for i, g in enumerate(aguards):
        expect(g.intact(), f"adjoint batch frame {i}")
    # the adjoint on the tensor cores (tensor_cores = 2), same frames
    bctx.set_config(256, 0, 32, tensor_cores=2)
    aguards2 = []
    for i, f in enumerate(adj):
        g = Guarded(torch, tuple(f.inp.shape), torch.float32, 4 * ((i + 1) % 3))
        aguards2.append(g)
        adj[i] = fv.BatchFrame(f.inp, g.t, f.fix_x, f.fix_y, f.sigma0, f.k)
    bctx.backward_batch(adj)
    torch.cuda.synchronize()
    for i, g in enumerate(aguards2):
        expect(g.intact(), f"tensor-core adjoint batch frame {i}")
    # float32 batches on the tensor cores: three planes per pass (uniform
    # channel count), one plane per pass (mixed counts); widths a multiple of
    # 4 and frames at least one TMA box (32 x 16), so every frame of a batch
    # is TMA-loadable and the batch runs on the tensor-core kernel
    bctx.set_config(256, 0, 32, tensor_cores=1)
    for label, shapes in (("f32 tc batch, 3 planes", [(3, 33, 64), (3, 300, 32), (3, 96, 512), (3, 16, 36)]),
                          ("f32 tc batch, mixed planes", [(1, 70, 1000), (2, 45, 36), (4, 129, 100)])):
        fr, gs = [], []
        for i, shape in enumerate(shapes):
            x = torch.from_numpy(wl.uniform_f32(shape, seed=40 + i)).to(dev)
            g = Guarded(torch, shape, torch.float32, 4 * (i % 4))
            fr.append(fv.BatchFrame(x, g.t, 0.25 * shape[2], 0.75 * shape[1], 0.5, 0.3))
            gs.append(g)
        bctx.render_batch(fr)
        torch.cuda.synchronize()
        for i, g in enumerate(gs):
            expect(g.intact(), f"{label} frame {i}")
    check_ctx(bctx, "batches")
    # a float32 frame beyond one wave: the tensor-core kernel on the single-frame path
    x = torch.from_numpy(wl.uniform_f32((3, 512, 800), seed=77)).to(dev)
    ctx = fv.Context(800, 512, 3, 32, 0.5, 0.02, fv.F32_CHW)
    for skew in (0, 4):
        g = Guarded(torch, (3, 512, 800), torch.float32, skew)
        ctx.render(x, g.t, 700.0, 30.0)
        torch.cuda.synchronize()
        expect(g.intact(), f"render f32 3x512x800 (tensor cores) skew={skew}")
    check_ctx(ctx, "f32 3x512x800")
    # ---- per-pixel foveation, pyramid and SSIM map
    for (h, w, c) in [(65, 33, 3), (1, 300, 1), (120, 200, 4)]:
        img = wl.uniform_u8((h, w, c), seed=h * w)
        x = torch.from_numpy(img).to(dev)
        ctx = fv.Context(w, h, c, 32, 0.5, 0.05, fv.U8_HWC)
        for tc in (0, 1):
            ctx.set_config(256, 0, 16 if tc == 3 else 32, tensor_cores=tc)
            g = Guarded(torch, (h, w, c), torch.uint8, 3)
            ctx.render_pixelwise(x, g.t, 10.0, 20.0)
            torch.cuda.synchronize()
            expect(g.intact(), f"pixelwise u8 {h}x{w}x{c} tc={tc}")
        g = Guarded(torch, (h, w, c), torch.uint8, 7)
        ctx.render_pyramid(x, g.t, 10.0, 20.0)
        torch.cuda.synchronize()
        expect(g.intact(), f"pyramid u8 {h}x{w}x{c}")
        check_ctx(ctx, f"pixelwise/pyramid {h}x{w}x{c}")
        m = Guarded(torch, (h, w), torch.float32, 4)
        total = torch.empty(1, dtype=torch.float64, device=dev)
        st = fv._lib.fovea_ssim(w, h, c, fv.U8_HWC, x.data_ptr(), x.data_ptr(), 0.0, m.t.data_ptr(),
                                total.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        expect(st == 0 and m.intact(), f"ssim map {h}x{w}x{c}")
    x = torch.from_numpy(wl.uniform_f32((3, 45, 70), seed=9)).to(dev)
    ctx = fv.Context(70, 45, 3, 32, 0.5, 0.05, fv.F32_CHW)
    for name, fn in (("pixelwise", ctx.render_pixelwise), ("pyramid", ctx.render_pyramid)):
        g = Guarded(torch, (3, 45, 70), torch.float32, 4)
        fn(x, g.t, 30.0, 5.0)
        torch.cuda.synchronize()
        expect(g.intact(), f"{name} f32")
    check_ctx(ctx, "pixelwise/pyramid f32")
    # ---- the no-allocation entry point
    for (h, w, c), fmt in [((65, 33, 3), fv.U8_HWC), ((1, 1, 1), fv.U8_HWC), ((3, 50, 31), fv.F32_CHW)]:
        if fmt == fv.U8_HWC:
            x = torch.from_numpy(wl.uniform_u8((h, w, c), seed=7)).to(dev)
            g = Guarded(torch, (h, w, c), torch.uint8, 9)
        else:
            x = torch.from_numpy(wl.uniform_f32((h, w, c), seed=7)).to(dev)
            g = Guarded(torch, (h, w, c), torch.float32, 8)
        fv.render_noalloc(x, g.t, 5.0, 5.0)
        try:
            fv.noalloc_check()
        except fv.FoveaError as e:
            fails.append(f"noalloc {h}x{w}x{c}: device faults 0x{e.faults:x}")
        torch.cuda.synchronize()
        expect(g.intact(), f"noalloc {h}x{w}x{c}")
    # ---- host-buffer path (pinned guards)
    h, w, c = 65, 33, 3
    hin = torch.from_numpy(wl.uniform_u8((h, w, c), seed=11)).pin_memory()
    ctx = fv.Context(w, h, c, 32, 0.5, 0.04, fv.U8_HWC)
    outs = [Guarded(torch, (h, w, c), torch.uint8, s, pin=True) for s in (0, 1, 2)]
    for g in outs:
        ctx.render_host(hin, g.t, 12.0, 40.0)
    torch.cuda.synchronize()
    for i, g in enumerate(outs):
        expect(g.intact(), f"render_host call {i}")
    check_ctx(ctx, "render_host")
    return fails


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    from paper_2012_08655_gb300 import fovea
    # the library's own flag agrees with the build the environment names
    assert fovea.BOUNDS_BUILD == ("bounds" in os.path.basename(fovea.LIB_PATH)), fovea.LIB_PATH
    problems = run_cases(fovea, torch)
    for p in problems:
        print("FAIL", p)
    print(f"library {fovea.LIB_PATH}: {len(problems)} failures")
    sys.exit(1 if problems else 0)
