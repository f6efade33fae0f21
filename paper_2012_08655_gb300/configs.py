"""The five measured configurations of the block-wise foveated blur, as data.

Each entry names the synthetic workload generator in ``workloads.py`` that
stands in for the paper's inputs, the frame shapes, element type and layout,
the sigma law sigma_b = sigma0 + k e_b (Section 2, Eq. 1; k drawn per frame
where it is a range), the block side, and the ``bench.py`` leg that measures
it. Nothing here computes: ``tests/test_configs_cpu.py`` checks every entry
against its generator's output, so the table and the generators cannot drift
apart.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional


@dataclass(frozen=True)
class RunConfig:
    name: str
    description: str
    generator: str                 # function in workloads.py
    shapes: tuple                  # frame shapes: (count, width, height, channels) groups
    dtype: str                     # "uint8" or "float32"
    layout: str                    # "hwc" or "chw"
    sigma0: float
    k: tuple                       # (k,) fixed, or (low, high) drawn per frame
    block: int
    bench_leg: str                 # key of the bench.py leg (the headline for "headline")
    extra: dict = field(default_factory=dict)


CONFIGS = [
    RunConfig(
        name="plain_256_f32",
        description="the plain method on a 256x256 single-channel float32 image, U[0,1), fixation at the centre",
        generator="plain_f32",
        shapes=((1, 256, 256, 1),),
        dtype="float32", layout="chw", sigma0=0.5, k=(0.02,), block=32,
        bench_leg="plain_256",
        extra={"fixation": (128.0, 128.0)}),
    RunConfig(
        name="frame_1080p_u8",
        description="the plain method at the paper's scale: one 1920x1080 RGB uint8 frame (sinusoid gratings and "
                    "rectangles), fixation at the centre",
        generator="frame_1080p",
        shapes=((1, 1920, 1080, 3),),
        dtype="uint8", layout="hwc", sigma0=0.5, k=(0.02,), block=32,
        bench_leg="headline",
        extra={"fixation": (960.0, 540.0)}),
    RunConfig(
        name="mixed_batch_64",
        description="64 RGB uint8 frames of mixed sizes, independent uniform fixations, slope per frame, "
                    "one persistent graph-captured launch with an autotuned configuration",
        generator="mixed_batch",
        shapes=((16, 640, 480, 3), (16, 1280, 720, 3), (24, 1920, 1080, 3), (8, 3840, 2160, 3)),
        dtype="uint8", layout="hwc", sigma0=0.5, k=(0.01, 0.04), block=32,
        bench_leg="batched"),
    RunConfig(
        name="served_stream",
        description="Poisson request stream at 2000 req/s for 10 s over 84x84 gray, 224x224, 1280x720 and "
                    "1920x1080 RGB frames (request weights 0.4/0.3/0.2/0.1), random-walk fixations",
        generator="served_stream",
        shapes=((1, 84, 84, 1), (1, 224, 224, 3), (1, 1280, 720, 3), (1, 1920, 1080, 3)),
        dtype="uint8", layout="hwc", sigma0=0.5, k=(0.02,), block=32,
        bench_leg="served",
        extra={"rate_hz": 2000.0, "duration_s": 10.0, "weights": (0.4, 0.3, 0.2, 0.1), "step_px": 30.0}),
    RunConfig(
        name="train_batch_f32",
        description="differentiable form: 32 float32 3x224x224 images, U[0,1), random fixations, strong "
                    "periphery law; forward and backward through torch.autograd",
        generator="train_batch",
        shapes=((32, 224, 224, 3),),
        dtype="float32", layout="chw", sigma0=0.5, k=(0.08,), block=32,
        bench_leg="train"),
]


def by_name(name: str) -> Optional[RunConfig]:
    for c in CONFIGS:
        if c.name == name:
            return c
    return None
