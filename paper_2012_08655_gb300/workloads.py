"""Seeded synthetic inputs for the foveation workloads.

This module generates input images, fixations and sigma-law parameters only;
it holds none of the method's arithmetic, and both the CUDA path's tests and
the oracle's tests draw their inputs from it. The paper's own test images
(its 1080p frame and its 30-image SSIM set) are not available; these
generators stand in for them with the same shapes, dtypes and value ranges.

Workloads (all numpy PCG64, seed 0 unless stated):

* ``plain_f32``      256x256x1 float32 U[0,1), fixation (128, 128),
                     sigma = 0.5 + 0.02 e.
* ``frame_1080p``    one 1920x1080 RGB uint8 frame (gratings + rectangles),
                     fixation at the centre, sigma = 0.5 + 0.02 e.
* ``mixed_batch``    64 RGB uint8 frames: 16x640x480, 16x1280x720,
                     24x1920x1080, 8x3840x2160; fixation uniform over the
                     frame, slope k ~ U[0.01, 0.04] per frame.
* ``served_stream``  Poisson arrivals at 2000 req/s for 10 s over 32 streams
                     (84x84 gray, 224x224 / 1280x720 / 1920x1080 RGB at
                     request weights 0.4/0.3/0.2/0.1); per-stream Gaussian
                     random-walk fixation (step 30 px) clamped to the frame.
* ``train_batch``    32x3x224x224 float32 U[0,1), fixations uniform over the
                     image, sigma = 0.5 + 0.08 e.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_f32(shape, seed: int = 0) -> np.ndarray:
    """i.i.d. U[0, 1) float32."""
    return rng(seed).random(shape, dtype=np.float32)


def uniform_u8(shape, seed: int = 0) -> np.ndarray:
    """i.i.d. uniform bytes 0..255."""
    return rng(seed).integers(0, 256, size=shape, dtype=np.uint8)


def grating_frame(height: int, width: int, channels: int = 3, seed: int = 0,
                  n_gratings: int = 8, n_rects: int = 50) -> np.ndarray:
    """Natural-looking synthetic frame, uint8 HWC.

    Base level 128; ``n_gratings`` sinusoid gratings with orientation
    U[0, pi), period log-uniform in [4, 200] px, phase U[0, 2 pi) and a
    per-channel amplitude U[0, 40]; then ``n_rects`` opaque rectangles with
    sides U[8, 400] px, uniform position and a per-channel colour U{0..255};
    clipped to [0, 255] and rounded.
    """
    g = rng(seed)
    img = np.full((height, width, channels), 128.0, np.float32)
    ys = np.arange(height, dtype=np.float64)
    xs = np.arange(width, dtype=np.float64)
    for _ in range(n_gratings):
        theta = g.uniform(0.0, np.pi)
        period = float(np.exp(g.uniform(np.log(4.0), np.log(200.0))))
        phase = g.uniform(0.0, 2.0 * np.pi)
        amp = g.uniform(0.0, 40.0, size=channels).astype(np.float32)
        f = 2.0 * np.pi / period
        ax = f * np.cos(theta) * xs
        ay = f * np.sin(theta) * ys + phase
        # sin(ax + ay) as a rank-2 outer product: cheap even for 4K frames.
        s = (np.outer(np.cos(ay), np.sin(ax)) + np.outer(np.sin(ay), np.cos(ax))).astype(np.float32)
        img += s[:, :, None] * amp[None, None, :]
    for _ in range(n_rects):
        rw = int(g.integers(8, 401))
        rh = int(g.integers(8, 401))
        x0 = int(g.integers(0, max(1, width)))
        y0 = int(g.integers(0, max(1, height)))
        col = g.integers(0, 256, size=channels).astype(np.float32)
        img[y0:y0 + rh, x0:x0 + rw, :] = col
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


@dataclass
class FrameSpec:
    """One frame of a workload: content, fixation and sigma law."""
    image: np.ndarray          # uint8 HWC or float32 CHW
    fix_x: float
    fix_y: float
    sigma0: float
    k: float
    layout: str                # "hwc" (uint8) or "chw" (float32)

    @property
    def height(self) -> int:
        return self.image.shape[0] if self.layout == "hwc" else self.image.shape[-2]

    @property
    def width(self) -> int:
        return self.image.shape[1] if self.layout == "hwc" else self.image.shape[-1]

    @property
    def channels(self) -> int:
        return self.image.shape[2] if self.layout == "hwc" else self.image.shape[0]


BLOCK = 32


def plain_f32(seed: int = 0) -> FrameSpec:
    """256x256 single-channel float32 U[0,1), centre fixation, sigma = 0.5 + 0.02 e."""
    return FrameSpec(uniform_f32((1, 256, 256), seed), 128.0, 128.0, 0.5, 0.02, "chw")


def frame_1080p(seed: int = 0) -> FrameSpec:
    """1920x1080 RGB uint8 frame, centre fixation, sigma = 0.5 + 0.02 e."""
    return FrameSpec(grating_frame(1080, 1920, 3, seed), 960.0, 540.0, 0.5, 0.02, "hwc")


MIXED_SIZES = [(640, 480)] * 16 + [(1280, 720)] * 16 + [(1920, 1080)] * 24 + [(3840, 2160)] * 8


def mixed_batch_params(seed: int = 0, sizes=None):
    """Fixations and slopes of the mixed batch: list of (W, H, fx, fy, k)."""
    g = rng(seed)
    out = []
    for (w, h) in (sizes or MIXED_SIZES):
        fx = float(np.float32(g.uniform(0.0, w)))
        fy = float(np.float32(g.uniform(0.0, h)))
        k = float(g.uniform(0.01, 0.04))
        out.append((w, h, fx, fy, k))
    return out


def mixed_batch(seed: int = 0, sizes=None) -> list[FrameSpec]:
    """64 RGB uint8 frames of mixed sizes with independent fixations and slopes."""
    frames = []
    for i, (w, h, fx, fy, k) in enumerate(mixed_batch_params(seed, sizes)):
        frames.append(FrameSpec(grating_frame(h, w, 3, seed * 1000 + 17 + i), fx, fy, 0.5, k, "hwc"))
    return frames


def train_batch(seed: int = 0, n: int = 32, size: int = 224):
    """(images float32 [n,3,size,size] U[0,1), fixations float32 [n,2]); sigma = 0.5 + 0.08 e."""
    g = rng(seed)
    x = g.random((n, 3, size, size), dtype=np.float32)
    fix = g.uniform(0.0, size, size=(n, 2)).astype(np.float32)
    return x, fix, 0.5, 0.08


STREAM_CLASSES = [  # (width, height, channels, request weight, streams)
    (84, 84, 1, 0.4, 13),
    (224, 224, 3, 0.3, 10),
    (1280, 720, 3, 0.2, 6),
    (1920, 1080, 3, 0.1, 3),
]


@dataclass
class StreamRequest:
    arrival_s: float
    stream: int
    width: int
    height: int
    channels: int
    fix_x: float
    fix_y: float


@dataclass
class ServedStream:
    requests: list = field(default_factory=list)
    stream_shapes: list = field(default_factory=list)   # (W, H, C) per stream
    sigma0: float = 0.5
    k: float = 0.02


def served_stream(seed: int = 0, rate_hz: float = 2000.0, duration_s: float = 10.0,
                  step_px: float = 30.0) -> ServedStream:
    """Poisson request stream over 32 streams with random-walk fixations.

    A request picks a stream with probability (class weight / streams in
    class), so the per-request resolution mix equals the class weights.
    """
    g = rng(seed)
    shapes, probs = [], []
    for (w, h, c, wt, ns) in STREAM_CLASSES:
        for _ in range(ns):
            shapes.append((w, h, c))
            probs.append(wt / ns)
    probs = np.asarray(probs) / np.sum(probs)
    fix = [[w / 2.0, h / 2.0] for (w, h, _) in shapes]
    t = 0.0
    reqs = []
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        s = int(g.choice(len(shapes), p=probs))
        w, h, c = shapes[s]
        step = g.normal(0.0, step_px, size=2)
        fix[s][0] = float(np.clip(fix[s][0] + step[0], 0.0, w))
        fix[s][1] = float(np.clip(fix[s][1] + step[1], 0.0, h))
        reqs.append(StreamRequest(t, s, w, h, c, float(np.float32(fix[s][0])), float(np.float32(fix[s][1]))))
    return ServedStream(reqs, shapes)
