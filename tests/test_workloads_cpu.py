"""The seeded input recipes (paper_2012_08655_gb300/workloads.py) on the CPU:
shapes, value ranges, determinism, and the statistics each recipe promises
(the served stream's class mix and Poisson rate, the mixed batch's sizes,
fixations and slopes, the training batch's fixations)."""
import math

import numpy as np

from paper_2012_08655_gb300 import workloads as wl


def test_generators_are_deterministic_and_seed_dependent():
    a, b, c = wl.grating_frame(60, 90, 3, seed=4), wl.grating_frame(60, 90, 3, seed=4), wl.grating_frame(60, 90, 3, seed=5)
    assert a.dtype == np.uint8 and a.shape == (60, 90, 3)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(wl.uniform_f32((3, 5), 1), wl.uniform_f32((3, 5), 1))
    assert np.array_equal(wl.uniform_u8((3, 5), 1), wl.uniform_u8((3, 5), 1))
    s1, s2 = wl.served_stream(seed=3, duration_s=0.5), wl.served_stream(seed=3, duration_s=0.5)
    assert s1.requests == s2.requests


def test_grating_frame_content():
    """Not flat: gratings and rectangles spread the bytes over the range, and
    rectangles leave runs of identical pixels."""
    img = wl.grating_frame(1080, 1920, 3, seed=0)
    assert img.min() < 40 and img.max() > 215
    assert len(np.unique(img)) > 200
    same_right = np.mean(np.all(img[:, 1:] == img[:, :-1], axis=2))
    assert same_right > 0.2  # rectangles are flat inside


def test_plain_and_headline_frames():
    p = wl.plain_f32()
    assert p.image.shape == (1, 256, 256) and p.image.dtype == np.float32
    assert 0.0 <= p.image.min() and p.image.max() < 1.0
    assert (p.fix_x, p.fix_y, p.sigma0, p.k, p.layout) == (128.0, 128.0, 0.5, 0.02, "chw")
    f = wl.frame_1080p()
    assert f.image.shape == (1080, 1920, 3) and f.image.dtype == np.uint8
    assert (f.fix_x, f.fix_y, f.sigma0, f.k, f.layout) == (960.0, 540.0, 0.5, 0.02, "hwc")
    assert (f.width, f.height, f.channels) == (1920, 1080, 3)


def test_mixed_batch_parameters():
    params = wl.mixed_batch_params(seed=0)
    sizes = [(w, h) for (w, h, _, _, _) in params]
    assert sizes == [(640, 480)] * 16 + [(1280, 720)] * 16 + [(1920, 1080)] * 24 + [(3840, 2160)] * 8
    mpix = sum(w * h for (w, h) in sizes) / 1e6
    assert abs(mpix - 135.7824) < 1e-9
    for (w, h, fx, fy, k) in params:
        assert 0.0 <= fx < w and 0.0 <= fy < h
        assert fx == float(np.float32(fx)) and fy == float(np.float32(fy))  # fixations are float32 values
        assert 0.01 <= k < 0.04
    ks = np.array([p[4] for p in params])
    assert ks.std() > 0.005  # drawn per frame, not one slope


def test_train_batch():
    x, fix, s0, k = wl.train_batch(seed=0)
    assert x.shape == (32, 3, 224, 224) and x.dtype == np.float32
    assert 0.0 <= x.min() and x.max() < 1.0 and abs(float(x.mean()) - 0.5) < 0.01
    assert fix.shape == (32, 2) and fix.dtype == np.float32
    assert fix.min() >= 0.0 and fix.max() < 224.0
    assert (s0, k) == (0.5, 0.08)


def test_served_stream_statistics():
    """Poisson arrivals at 2000 per second over 32 streams whose class mix is
    {0.4, 0.3, 0.2, 0.1} per request; fixations walk inside the frame."""
    s = wl.served_stream(seed=0, duration_s=10.0)
    n = len(s.requests)
    assert abs(n - 20000) < 5 * math.sqrt(20000)
    t = np.array([r.arrival_s for r in s.requests])
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < 10.0
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000) < 0.05 / 2000 and abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential
    shapes = s.stream_shapes
    assert len(shapes) == 32
    counts = {}
    for (w, h, c, _, ns) in wl.STREAM_CLASSES:
        assert sum(1 for sh in shapes if sh == (w, h, c)) == ns
    for r in s.requests:
        assert shapes[r.stream] == (r.width, r.height, r.channels)
        assert 0.0 <= r.fix_x <= r.width and 0.0 <= r.fix_y <= r.height
        counts[(r.width, r.height)] = counts.get((r.width, r.height), 0) + 1
    for (w, h, c, wt, _) in wl.STREAM_CLASSES:
        frac = counts[(w, h)] / n
        assert abs(frac - wt) < 5 * math.sqrt(wt * (1 - wt) / n), (w, h, frac)
    assert (s.sigma0, s.k) == (0.5, 0.02)
    # each stream's walk starts near its frame centre (steps of N(0, 30^2) px)
    first = {}
    for r in s.requests:
        first.setdefault(r.stream, r)
    for st, r in first.items():
        w, h, _ = shapes[st]
        assert abs(r.fix_x - w / 2) <= 6 * 30 and abs(r.fix_y - h / 2) <= 6 * 30
