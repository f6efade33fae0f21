"""Host-side logic of bench.py that the reported numbers rest on: the
algorithmic work counts (roofline numerators) and the tensor-core work model
of the per-pixel kernel, checked against brute-force counts."""
import numpy as np

import bench


def test_algorithmic_fmas_is_the_separable_count_per_block():
    # 70 x 45 frame, B = 32: blocks of 32 x 32, 6 x 32, 32 x 13, 6 x 13
    rad = np.array([[3, 5], [0, 7]], np.int32)
    C, B = 3, 32
    want = 0
    for by, bh in enumerate((32, 13)):
        for bx, bw in enumerate((32, 6)):
            r = int(rad[by, bx])
            # horizontal pass over bh + 2r rows, vertical over bh rows, 2r + 1 taps each
            want += C * (2 * r + 1) * bw * (bh + 2 * r) + C * (2 * r + 1) * bw * bh
    assert bench.algorithmic_fmas(rad, 38, 45, C, B) == want
    lb = sum(C * 2 * (2 * int(rad[by, bx]) + 1) * bw * bh
             for by, bh in enumerate((32, 13)) for bx, bw in enumerate((32, 6)))
    assert bench.lower_bound_fmas(rad, 38, 45, C, B) == lb


def test_pixel_radii_match_the_pixel_centre_law():
    r = bench.pixel_radii(5, 4, 2.5, 1.5, 0.5, 0.3)
    for y in range(4):
        for x in range(5):
            e = np.hypot(x + 0.5 - 2.5, y + 0.5 - 1.5)
            assert r[y, x] == np.ceil(3 * (0.5 + 0.3 * e))


def test_pixelwise_mma_model_counts_the_kernel_loops():
    """Brute force over tiles, columns, channel planes, k-steps and 32-pixel
    groups, as the tensor-core per-pixel kernel runs them: hi and lo m16n8k16
    MMAs (16 * 8 * 16 multiply-adds each) per k-step and 8-column n-tile."""
    W, H, C, fx, fy, s0, k = 40, 20, 3, 7.0, 3.0, 0.5, 0.1
    r = bench.pixel_radii(W, H, fx, fy, s0, k)
    macs = 0
    for y0 in range(0, H, 16):
        for x0 in range(0, W, 16):
            R = int(r[y0:y0 + 16, x0:x0 + 16].max())
            ksteps = len(range(0, 16 + 2 * R, 16))
            for lx in range(min(16, W - x0)):
                groups = len(range(0, lx + 2 * R + 1, 32))
                for _c in range(C):
                    for _ks in range(ksteps):
                        for _g in range(groups):
                            for _nt in range(4):
                                macs += 2 * 16 * 8 * 16
    assert bench.pixelwise_mma_macs(W, H, C, fx, fy, s0, k) == macs


def test_cpu_model_is_a_description():
    s = bench.cpu_model()
    assert isinstance(s, str) and "logical CPUs" in s
