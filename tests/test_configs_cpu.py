"""The configuration table (paper_2012_08655_gb300/configs.py) agrees with the
workload generators it names and with the bench legs that measure it."""
import os
import re

import numpy as np

from paper_2012_08655_gb300 import configs, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_config_matches_its_generator():
    seen = set()
    for c in configs.CONFIGS:
        assert c.name not in seen
        seen.add(c.name)
        assert hasattr(wl, c.generator), c.generator
        if c.generator in ("plain_f32", "frame_1080p"):
            spec = getattr(wl, c.generator)(seed=0)
            (count, w, h, ch), = c.shapes
            assert count == 1 and spec.layout == c.layout
            assert spec.image.dtype == np.dtype(c.dtype)
            shape = (h, w, ch) if c.layout == "hwc" else (ch, h, w)
            assert spec.image.shape == shape
            assert (spec.sigma0, spec.k) == (c.sigma0, c.k[0])
            assert (spec.fix_x, spec.fix_y) == c.extra["fixation"]
        elif c.generator == "mixed_batch":
            params = wl.mixed_batch_params(seed=0)
            want = [(w, h) for (n, w, h, _) in c.shapes for _ in range(n)]
            assert [(w, h) for (w, h, _, _, _) in params] == want
            lo, hi = c.k
            assert all(lo <= k <= hi for (_, _, _, _, k) in params)
            assert all(0.0 <= fx <= w and 0.0 <= fy <= h for (w, h, fx, fy, _) in params)
        elif c.generator == "served_stream":
            stream = wl.served_stream(seed=0, duration_s=0.5)
            classes = {(w, h, ch) for (w, h, ch, _, _) in wl.STREAM_CLASSES}
            assert classes == {(w, h, ch) for (_, w, h, ch) in c.shapes}
            weights = tuple(wt for (_, _, _, wt, _) in wl.STREAM_CLASSES)
            assert weights == c.extra["weights"]
            assert (stream.requests[0].arrival_s >= 0.0) and len(stream.requests) > 0.5 * 0.5 * c.extra["rate_hz"]
        elif c.generator == "train_batch":
            x, fix, s0, k = wl.train_batch(seed=0)
            (n, w, h, ch), = c.shapes
            assert x.shape == (n, ch, h, w) and x.dtype == np.dtype(c.dtype)
            assert fix.shape == (n, 2) and (s0, k) == (c.sigma0, c.k[0])
        else:
            raise AssertionError(f"no check for generator {c.generator}")


def test_every_config_has_a_bench_leg():
    src = open(os.path.join(ROOT, "bench.py")).read()
    legs = set(re.findall(r'extras\["(\w+)"\]', src))
    for c in configs.CONFIGS:
        assert c.bench_leg == "headline" or c.bench_leg in legs, c.bench_leg
