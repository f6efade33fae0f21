"""Pins for the FP64 oracle: checks against things other than itself.

Each test ties the oracle to what the paper or the mathematics fixes:
scipy's textbook Gaussian filter (uniform sigma, clamp-to-edge), closed forms
of the sigma law, the paper's Eq. 7 figures, and invariants of a normalised,
clamped, symmetric linear filter (constants, identity, mirror symmetry,
linearity, the max principle, the adjoint identity). A plausible mistake in
the oracle -- a dropped tap, a wrong sign or index, a transposed operand, a
mis-centred block -- fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
from scipy import ndimage
from scipy.signal import windows

import oracle
from paper_2012_08655_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- sigma law

def test_sigma_at_fixation_block_is_sigma0():
    # Fixation exactly on the centre of block (2, 1) with B = 32: e = 0.
    sig, rad = oracle.sigma_table(200, 100, 32, 2 * 32 + 16, 1 * 32 + 16, 0.7, 0.05)
    assert sig[1, 2] == 0.7
    assert rad[1, 2] == 3  # ceil(2.1)


def test_sigma_pythagorean_distance_is_exact():
    # Block (0,0) centre (16,16); fixation (19,20): e = 5 exactly.
    sig, rad = oracle.sigma_table(64, 64, 32, 19.0, 20.0, 0.5, 0.1)
    assert sig[0, 0] == 1.0
    assert rad[0, 0] == 3
    # Block (1,0) centre (48,16): dx = 29, dy = -4 -> e = sqrt(857).
    assert sig[0, 1] == 0.5 + 0.1 * np.sqrt(857.0)


def test_sigma_symmetric_and_monotone():
    sig, rad = oracle.sigma_table(256, 256, 32, 128.0, 128.0, 0.5, 0.02)
    assert np.array_equal(sig, sig[::-1, :]) and np.array_equal(sig, sig[:, ::-1])
    assert np.array_equal(sig, sig.T)
    # Corner blocks are farthest, the four centre blocks nearest.
    assert sig[0, 0] == sig.max() and sig[3, 3] == sig.min()
    assert rad.max() == 12 and abs(sig.max() - 3.6678) < 1e-4 and abs(sig.min() - 0.95255) < 1e-4


def test_sigma_grid_counts_partial_blocks():
    sig, rad = oracle.sigma_table(1920, 1080, 32, 960.0, 540.0, 0.5, 0.02)
    assert sig.shape == (34, 60)
    # Partial last block row keeps its nominal centre (y = 33*32 + 16 = 1072).
    assert sig[33, 0] == 0.5 + 0.02 * np.hypot(16.0 - 960.0, 1072.0 - 540.0)
    assert rad.max() == 67


# ---------------------------------------------------------------- taps

@pytest.mark.parametrize("sigma", [0.3, 0.9, 1.0, 2.5, 7.3, 22.2])
def test_taps_match_scipy_window(sigma):
    r = int(np.ceil(3 * sigma))
    w = oracle.taps(sigma, r)
    ref = windows.gaussian(2 * r + 1, sigma, sym=True)
    ref = ref / ref.sum()
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.array_equal(w, w[::-1])
    assert abs(w[r + 1] / w[r] - np.exp(-1.0 / (2 * sigma * sigma))) < 1e-14


def test_taps_degenerate():
    assert np.array_equal(oracle.taps(0.0, 0), [1.0])
    w = oracle.taps(1e-3, 1)
    assert np.array_equal(w, [0.0, 1.0, 0.0])


# ---------------------------------------------------------------- uniform sigma == scipy

def _scipy_uniform(img, sigma, r, layout):
    if img.ndim == 2:
        return ndimage.gaussian_filter(img.astype(np.float64), sigma, mode="nearest", radius=r)
    if layout == "hwc":
        return ndimage.gaussian_filter(img.astype(np.float64), (sigma, sigma, 0.0), mode="nearest",
                                       radius=(r, r, 0))
    return ndimage.gaussian_filter(img.astype(np.float64), (0.0, sigma, sigma), mode="nearest",
                                   radius=(0, r, r))


@pytest.mark.parametrize("shape,layout,sigma0,B", [
    ((64, 80), "hwc", 1.3, 32),
    ((37, 29, 3), "hwc", 2.2, 8),
    ((2, 45, 50), "chw", 0.8, 16),
    ((20, 23), "hwc", 9.0, 4),       # r = 27 > W, H: clamping folds whole rows
])
def test_uniform_sigma_equals_scipy_gaussian_filter(shape, layout, sigma0, B):
    img = wl.uniform_f32(shape, seed=3).astype(np.float64)
    H, W = (shape[0], shape[1]) if layout == "hwc" else (shape[1], shape[2])
    out = oracle.forward(img, B, 0.3 * W, 0.6 * H, sigma0, 0.0, layout)
    r = int(np.ceil(3 * sigma0))
    ref = _scipy_uniform(img, sigma0, r, layout)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- block-wise selection

@pytest.mark.parametrize("W,H,C,layout,B,fx,fy,s0,k", [
    (256, 256, 1, "chw", 32, 128.0, 128.0, 0.5, 0.02),     # the 256x256 plain workload
    (100, 70, 3, "hwc", 16, 20.5, 61.25, 0.4, 0.05),       # partial edge blocks, RGB
    (57, 41, 2, "chw", 8, -10.0, 50.0, 0.0, 0.15),         # fixation outside the frame
])
def test_blockwise_equals_per_block_uniform_blur(W, H, C, layout, B, fx, fy, s0, k):
    shape = (C, H, W) if layout == "chw" else (H, W, C)
    img = wl.uniform_f32(shape, seed=11).astype(np.float64)
    out = oracle.forward(img, B, fx, fy, s0, k, layout)
    sig, rad = oracle.sigma_table(W, H, B, fx, fy, s0, k)
    for by in range(sig.shape[0]):
        for bx in range(sig.shape[1]):
            ref = _scipy_uniform(img, sig[by, bx], int(rad[by, bx]), layout)
            ys, xs = slice(by * B, min(by * B + B, H)), slice(bx * B, min(bx * B + B, W))
            if layout == "chw":
                got, exp = out[:, ys, xs], ref[:, ys, xs]
            else:
                got, exp = out[ys, xs], ref[ys, xs]
            np.testing.assert_allclose(got, exp, rtol=0, atol=1e-13)


def test_u8_frame_blockwise_matches_scipy_after_rounding():
    img = wl.grating_frame(96, 160, 3, seed=5)
    q = oracle.forward_u8(img, 32, 80.0, 48.0, 0.5, 0.04, "hwc")
    sig, rad = oracle.sigma_table(160, 96, 32, 80.0, 48.0, 0.5, 0.04)
    ref = np.zeros(img.shape, np.float64)
    for by in range(sig.shape[0]):
        for bx in range(sig.shape[1]):
            f = _scipy_uniform(img, sig[by, bx], int(rad[by, bx]), "hwc")
            ref[by * 32:by * 32 + 32, bx * 32:bx * 32 + 32] = f[by * 32:by * 32 + 32, bx * 32:bx * 32 + 32]
    refq = np.clip(np.floor(ref + 0.5), 0, 255).astype(np.uint8)
    assert np.max(np.abs(q.astype(int) - refq.astype(int))) <= 1
    assert np.mean(q == refq) > 0.999


# ---------------------------------------------------------------- invariants

def test_constant_image_stays_constant():
    img = np.full((70, 90, 3), 0.37)
    out = oracle.forward(img, 32, 10.0, 20.0, 0.5, 0.1, "hwc")
    assert np.max(np.abs(out - 0.37)) < 1e-14
    q = oracle.forward_u8(np.full((70, 90, 3), 200, np.uint8), 32, 10.0, 20.0, 0.5, 0.1)
    assert np.all(q == 200)


def test_sigma_zero_is_identity():
    img = wl.uniform_f32((3, 40, 50), seed=2).astype(np.float64)
    assert np.array_equal(oracle.forward(img, 16, 5.0, 5.0, 0.0, 0.0, "chw"), img)
    # sigma0 = 1e-3 gives r = 1 whose outer taps underflow to zero.
    assert np.array_equal(oracle.forward(img, 16, 5.0, 5.0, 1e-3, 0.0, "chw"), img)


def test_mirror_about_fixation_commutes():
    W, H, B = 128, 96, 32
    img = wl.uniform_f32((H, W, 3), seed=4).astype(np.float64)
    fx, fy = 40.25, 70.5
    out = oracle.forward(img, B, fx, fy, 0.5, 0.05, "hwc")
    flip_x = oracle.forward(img[:, ::-1], B, W - fx, fy, 0.5, 0.05, "hwc")
    np.testing.assert_allclose(flip_x, out[:, ::-1], rtol=0, atol=1e-13)
    flip_y = oracle.forward(img[::-1], B, fx, H - fy, 0.5, 0.05, "hwc")
    np.testing.assert_allclose(flip_y, out[::-1], rtol=0, atol=1e-13)


def test_transpose_commutes_on_square_image():
    img = wl.uniform_f32((96, 96), seed=8).astype(np.float64)
    out = oracle.forward(img, 32, 20.0, 61.0, 0.5, 0.04)
    tr = oracle.forward(img.T, 32, 61.0, 20.0, 0.5, 0.04)
    np.testing.assert_allclose(tr, out.T, rtol=0, atol=1e-13)


def test_linearity_and_max_principle():
    a = wl.uniform_f32((2, 50, 60), seed=5).astype(np.float64)
    b = wl.uniform_f32((2, 50, 60), seed=6).astype(np.float64)
    args = (16, 33.0, 12.0, 0.3, 0.07, "chw")
    fa, fb = oracle.forward(a, *args), oracle.forward(b, *args)
    fab = oracle.forward(2.5 * a - 1.5 * b, *args)
    np.testing.assert_allclose(fab, 2.5 * fa - 1.5 * fb, rtol=0, atol=1e-12)
    assert fa.min() >= a.min() - 1e-14 and fa.max() <= a.max() + 1e-14


def test_adjoint_identity():
    W, H, C, B = 23, 17, 2, 8
    g = wl.rng(9)
    x = g.standard_normal((C, H, W))
    y = g.standard_normal((C, H, W))
    for fx, fy, s0, k in [(5.0, 3.0, 0.5, 0.2), (30.0, -4.0, 1.0, 0.5), (11.5, 8.5, 0.0, 0.0)]:
        ax = oracle.forward(x, B, fx, fy, s0, k, "chw")
        aty = oracle.adjoint(y, B, fx, fy, s0, k, "chw")
        lhs, rhs = float(np.sum(ax * y)), float(np.sum(x * aty))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_dense_matrix_brute_force():
    """Build A and A^T column by column from unit vectors on a tiny image."""
    W, H, B = 12, 10, 4
    fx, fy, s0, k = 5.5, 3.2, 0.2, 0.3
    n = W * H
    A = np.zeros((n, n))
    AT = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        A[:, q] = oracle.forward(e.reshape(H, W), B, fx, fy, s0, k).ravel()
        AT[:, q] = oracle.adjoint(e.reshape(1, H, W), B, fx, fy, s0, k, "chw").ravel()
    np.testing.assert_allclose(AT, A.T, rtol=0, atol=1e-15)
    assert A.min() >= 0.0
    np.testing.assert_allclose(A.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    # Each output pixel's weights over the input plane form a separable
    # (rank-one) kernel: the 2D filter is a product of two 1D filters.
    for p in range(n):
        s = np.linalg.svd(A[p].reshape(H, W), compute_uv=False)
        assert s[1] <= 1e-13 * s[0]
    # The weights of an output pixel follow its block's taps with clamping:
    # column sums of its row-slice equal the 1D taps folded at the borders.
    sig, rad = oracle.sigma_table(W, H, B, fx, fy, s0, k)
    for p in [0, 17, 45, 119]:
        py, px = divmod(p, W)
        r = int(rad[py // B, px // B])
        w = oracle.taps(sig[py // B, px // B], r)
        fold = np.zeros(W)
        for i in range(-r, r + 1):
            fold[min(max(px + i, 0), W - 1)] += w[i + r]
        np.testing.assert_allclose(A[p].reshape(H, W).sum(axis=0), fold, rtol=0, atol=1e-15)


def test_sampled_blocks_match_full_frame():
    img = wl.grating_frame(70, 100, 3, seed=1)
    full = oracle.forward(img, 32, 50.0, 35.0, 0.5, 0.05, "hwc")
    part = oracle.forward(img, 32, 50.0, 35.0, 0.5, 0.05, "hwc", blocks=[0, 5, 11])
    for b in [0, 5, 11]:
        by, bx = divmod(b, 4)
        sl = (slice(by * 32, by * 32 + 32), slice(bx * 32, bx * 32 + 32))
        assert np.array_equal(part[sl], full[sl])
    assert not np.isnan(part[40, 40, 0])  # block 5 = (bx 1, by 1)
    assert np.isnan(part[10, 40, 0])      # block 1 was not listed


# ---------------------------------------------------------------- uint8 coding

def test_quantize_u8_rounding():
    v = np.array([-3.0, -0.2, 0.0, 0.49999, 0.5, 1.5, 2.5, 127.4999, 254.5, 255.0, 255.7, 300.0])
    q = oracle.quantize_u8(v)
    assert q.tolist() == [0, 0, 0, 0, 1, 2, 3, 127, 255, 255, 255, 255]


# ---------------------------------------------------------------- paper's Eq. 7 figures

def test_eq7_max_filter_sizes_pin_tile_geometry():
    """Eq. 7 with the paper's maximum filter sizes fixes two readings: the tile
    is the fragment padded by N-1 pixels in each dimension (radius (N-1)/2 on
    each side), and the 'bits' of Eq. 7 are bytes against a 48,000-byte limit."""
    with open(os.path.join(GOLDEN, "eq7_max_filter.json")) as f:
        gold = json.load(f)
    limit = gold["shared_memory_limit_bytes"]

    def usage(frag, n):
        tile = frag + n - 1
        return tile * tile + 4 * frag * tile

    for case in gold["cases"]:
        frag, nmax = case["fragment"], case["max_filter"]
        assert usage(frag, nmax) <= limit < usage(frag, nmax + 1)
        assert usage(frag, nmax) == case["bytes_at_max"]


# ---------------------------------------------------------------- other sigma laws, shifted grid

def test_geisler_perry_chain_reduces_to_the_linear_law():
    """Eqs. 2-6 taken step by step give sigma = (1 + e/e2) / pi, i.e. the
    linear law with sigma0 = 1/pi and k = e_corner / (pi e2 d_corner)."""
    g = wl.rng(5)
    for _ in range(50):
        W, H = int(g.integers(16, 4000)), int(g.integers(16, 3000))
        ec = float(g.uniform(1.0, 60.0))
        s0, k = oracle.gp_linear(W, H, ec)
        assert s0 == 1.0 / np.pi
        for d in g.uniform(0.0, 3000.0, size=8):
            np.testing.assert_allclose(oracle.gp_sigma(d, W, H, ec), s0 + k * d, rtol=1e-13)
    # at the frame corner the eccentricity is e_corner: sigma = (1 + e_corner / 2.3) / pi
    W, H, ec = 1920, 1080, 20.0
    dc = 0.5 * np.hypot(W, H)
    np.testing.assert_allclose(oracle.gp_sigma(dc, W, H, ec), (1.0 + ec / 2.3) / np.pi, rtol=1e-14)
    # the fovea keeps the finest filter: the cut-off frequency is the
    # highest there, half a cycle per pixel, so sigma = 1 / pi
    assert oracle.gp_sigma(0.0, W, H, ec) == pytest.approx(1.0 / np.pi, rel=1e-15)


@pytest.mark.parametrize("B", [8, 16, 32])
def test_centred_origin_puts_a_block_centre_on_the_fixation(B):
    g = wl.rng(6)
    for _ in range(200):
        f = float(g.uniform(-100.0, 2000.0))
        o = oracle.centred_origin(f, B)
        assert 0 <= o < B
        # the block starting at floor(f + 1/2) - floor(B/2) is on the grid
        start = int(np.floor(f + 0.5)) - B // 2
        assert (start + o) % B == 0
        if B % 2 == 0:  # its nominal centre is the nearest pixel corner to f
            assert start + B / 2 == np.floor(f + 0.5)


def test_shifted_grid_blockwise_equals_per_block_uniform_blur():
    """With a shifted grid every (clipped) block is still the uniform blur
    at its own sigma, and sigma follows the shifted block centres."""
    W, H, C, B = 90, 70, 2, 16
    img = wl.uniform_f32((H, W, C), seed=12).astype(np.float64)
    fx, fy = 41.3, 27.8
    ox, oy = oracle.centred_origin(fx, B), oracle.centred_origin(fy, B)
    assert (ox, oy) != (0, 0)
    out = oracle.forward(img, B, fx, fy, 0.4, 0.06, "hwc", origin=(ox, oy))
    sig, rad = oracle.sigma_table(W, H, B, fx, fy, 0.4, 0.06, origin=(ox, oy))
    assert sig.shape == ((H + oy + B - 1) // B, (W + ox + B - 1) // B)
    # the block holding the fixation has the smallest sigma, at most 1/sqrt(2) px off-centre
    iy, ix = np.unravel_index(np.argmin(sig), sig.shape)
    assert B * ix - ox <= fx < B * ix - ox + B and B * iy - oy <= fy < B * iy - oy + B
    assert sig[iy, ix] <= 0.4 + 0.06 * np.sqrt(0.5) + 1e-12
    for by in range(sig.shape[0]):
        for bx in range(sig.shape[1]):
            cx, cy = B * bx + B / 2 - ox, B * by + B / 2 - oy
            assert sig[by, bx] == 0.4 + 0.06 * np.sqrt((cx - fx) ** 2 + (cy - fy) ** 2)
            ref = _scipy_uniform(img, sig[by, bx], int(rad[by, bx]), "hwc")
            ys = slice(max(0, B * by - oy), min(H, B * by - oy + B))
            xs = slice(max(0, B * bx - ox), min(W, B * bx - ox + B))
            np.testing.assert_allclose(out[ys, xs], ref[ys, xs], rtol=0, atol=1e-13)


def test_mirror_commutes_with_centred_grid():
    W, H, B = 224, 160, 32
    img = wl.uniform_f32((H, W, 3), seed=13).astype(np.float64)
    fx, fy = 100.0, 37.0
    org = (oracle.centred_origin(fx, B), oracle.centred_origin(fy, B))
    out = oracle.forward(img, B, fx, fy, 0.5, 0.05, "hwc", origin=org)
    mx = W - fx
    orgx = (oracle.centred_origin(mx, B), org[1])
    flip = oracle.forward(img[:, ::-1], B, mx, fy, 0.5, 0.05, "hwc", origin=orgx)
    np.testing.assert_allclose(flip, out[:, ::-1], rtol=0, atol=1e-13)


def test_sigma_map_equal_to_the_law_reproduces_it_and_a_constant_map_is_uniform():
    W, H, B = 75, 50, 16
    img = wl.uniform_f32((2, H, W), seed=14).astype(np.float64)
    sig, rad = oracle.sigma_table(W, H, B, 30.0, 20.0, 0.5, 0.07)
    a = oracle.forward(img, B, 30.0, 20.0, 0.5, 0.07, "chw")
    b = oracle.forward(img, B, 0.0, 0.0, 0.0, 0.0, "chw", sigma_map=sig)
    assert np.array_equal(a, b)
    const = np.full(sig.shape, 1.7)
    c = oracle.forward(img, B, 0.0, 0.0, 0.0, 0.0, "chw", sigma_map=const)
    np.testing.assert_allclose(c, _scipy_uniform(img, 1.7, 6, "chw"), rtol=0, atol=1e-13)
    s2, r2 = oracle.sigma_table(W, H, B, 0.0, 0.0, 0.0, 0.0, sigma_map=const)
    assert np.all(s2 == 1.7) and np.all(r2 == 6)
    # the adjoint follows the map too
    g = wl.uniform_f32((2, H, W), seed=15).astype(np.float64)
    lhs = np.vdot(c, g)
    rhs = np.vdot(img, oracle.adjoint(g, B, 0.0, 0.0, 0.0, 0.0, "chw", sigma_map=const))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


# ---------------------------------------------------------------- per-pixel foveation

def _pixel_sigma_def(x, y, fx, fy, s0, k):
    return s0 + k * np.hypot(x + 0.5 - fx, y + 0.5 - fy)


def test_pixel_sigma_closed_form():
    # Pixel (3, 4) has centre (3.5, 4.5); from fixation (0.5, 0.5) that is a 3-4-5 triangle.
    assert oracle.pixel_sigma(3, 4, 0.5, 0.5, 0.25, 0.5) == (2.75, 9)
    # A fixation on a pixel centre gives that pixel sigma0.
    assert oracle.pixel_sigma(7, 2, 7.5, 2.5, 1.1, 3.0) == (1.1, 4)
    # Mirror pixel about the fixation has the same sigma.
    assert oracle.pixel_sigma(10, 3, 6.0, 6.0, 0.5, 0.1) == oracle.pixel_sigma(1, 8, 6.0, 6.0, 0.5, 0.1)


@pytest.mark.parametrize("W,H,C,layout,fx,fy,s0,k", [
    (24, 18, 1, "hwc", 7.3, 11.9, 0.4, 0.21),
    (19, 15, 3, "hwc", -3.0, 4.0, 0.0, 0.3),     # fixation outside the frame, sigma0 = 0
    (16, 21, 2, "chw", 8.0, 10.5, 0.7, 0.12),
])
def test_perpixel_equals_uniform_blur_at_each_pixels_sigma(W, H, C, layout, fx, fy, s0, k):
    """Every output pixel equals scipy's uniform Gaussian blur at that pixel's
    own sigma (pixel-centre distance), read at that pixel."""
    shape = (C, H, W) if layout == "chw" else (H, W, C)
    img = wl.uniform_f32(shape, seed=5).astype(np.float64)
    out = oracle.forward_pixel(img, fx, fy, s0, k, layout)
    for y in range(H):
        for x in range(W):
            sg = _pixel_sigma_def(x, y, fx, fy, s0, k)
            d = abs(3 * sg - round(3 * sg))
            assert d == 0 or d > 1e-9  # an exact integer 3 sigma is unambiguous
            r = int(np.ceil(3 * sg))
            if r == 0:
                ref = img
            else:
                ref = _scipy_uniform(img, sg, r, layout)
            if layout == "chw":
                np.testing.assert_allclose(out[:, y, x], ref[:, y, x], rtol=0, atol=1e-13)
            else:
                np.testing.assert_allclose(out[y, x], ref[y, x], rtol=0, atol=1e-13)


def test_perpixel_is_blockwise_with_one_pixel_blocks():
    """A 1x1 block's centre is its pixel's centre: per-pixel foveation is the
    block-wise map at B = 1 (a different code path of the oracle, pinned to
    scipy block by block)."""
    img = wl.uniform_f32((23, 31, 3), seed=8).astype(np.float64)
    a = oracle.forward_pixel(img, 12.25, 5.5, 0.3, 0.15, "hwc")
    b = oracle.forward(img, 1, 12.25, 5.5, 0.3, 0.15, "hwc")
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_perpixel_mirror_constant_and_sampling():
    W, H = 26, 20
    img = wl.uniform_f32((H, W), seed=9).astype(np.float64)
    fx, fy = 9.75, 6.5
    a = oracle.forward_pixel(img, fx, fy, 0.5, 0.2)
    m = oracle.forward_pixel(img[:, ::-1], W - fx, fy, 0.5, 0.2)
    np.testing.assert_allclose(a, m[:, ::-1], rtol=0, atol=1e-13)
    m = oracle.forward_pixel(img[::-1, :], fx, H - fy, 0.5, 0.2)
    np.testing.assert_allclose(a, m[::-1, :], rtol=0, atol=1e-13)
    c = oracle.forward_pixel(np.full((H, W), 0.375), fx, fy, 0.5, 0.2)
    np.testing.assert_allclose(c, 0.375, rtol=0, atol=1e-14)
    pix = [0, W - 1, 7 * W + 3, H * W - 1]
    s = oracle.forward_pixel(img, fx, fy, 0.5, 0.2, pixels=pix)
    flat_a, flat_s = a.reshape(-1), s.reshape(-1)
    assert np.array_equal(flat_s[pix], flat_a[pix])
    assert np.isnan(np.delete(flat_s, pix)).all()


# ---------------------------------------------------------------- SSIM

def _gauss_stats(img):
    f = lambda v: ndimage.gaussian_filter(v, 1.5, mode="nearest", radius=5)
    mu = f(img)
    return mu, f(img * img) - mu * mu


def test_ssim_identical_images_and_constants():
    a = wl.uniform_f32((17, 23), seed=1).astype(np.float64)
    np.testing.assert_allclose(oracle.ssim_map(a, a, 1.0), 1.0, rtol=0, atol=1e-14)
    al, be, L = 40.0, 200.0, 255.0
    C1 = (0.01 * L) ** 2
    m = oracle.ssim_map(np.full((9, 12), al), np.full((9, 12), be), L)
    np.testing.assert_allclose(m, (2 * al * be + C1) / (al * al + be * be + C1), rtol=1e-14)


@pytest.mark.parametrize("s,t", [(0.6, 0.2), (-0.7, 0.9), (1.0, 0.05)])
def test_ssim_of_an_affine_copy_matches_library_moments(s, t):
    """b = s a + t: cov = s var_a, var_b = s^2 var_a, mu_b = s mu_a + t, so
    SSIM = l * (2 s var + C2) / ((1 + s^2) var + C2) with the local moments
    taken from scipy's Gaussian filter (sigma 1.5, radius 5, nearest)."""
    a = wl.uniform_f32((21, 26), seed=4).astype(np.float64)
    b = s * a + t
    mu, var = _gauss_stats(a)
    mub = s * mu + t
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ref = (2 * mu * mub + C1) / (mu * mu + mub * mub + C1) * (2 * s * var + C2) / ((1 + s * s) * var + C2)
    np.testing.assert_allclose(oracle.ssim_map(a, b, 1.0), ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.ssim_map(b, a, 1.0), ref, rtol=0, atol=1e-12)


def test_ssim_range_scaling_and_channel_mean():
    rng = np.random.default_rng(2)
    a = rng.random((14, 19, 3))
    b = np.clip(a + 0.1 * rng.standard_normal(a.shape), 0, 1)
    m1 = oracle.ssim_map(a, b, 1.0, "hwc")
    np.testing.assert_allclose(oracle.ssim_map(255 * a, 255 * b, 255.0, "hwc"), m1, rtol=0, atol=1e-12)
    per = [oracle.ssim_map(a[:, :, c], b[:, :, c], 1.0) for c in range(3)]
    np.testing.assert_allclose(m1, np.mean(per, axis=0), rtol=0, atol=1e-14)
    chw = oracle.ssim_map(np.moveaxis(a, 2, 0).copy(), np.moveaxis(b, 2, 0).copy(), 1.0, "chw")
    np.testing.assert_allclose(chw, m1, rtol=0, atol=1e-14)
    assert (m1 < 1).all() and (m1 > -1).all()


# ---------------------------------------------------------------- Gaussian pyramid (mipmap) foveation

_W5 = np.array([1, 4, 6, 4, 1], np.float64) / 16.0


def _scipy_reduce(plane):
    blurred = ndimage.convolve1d(ndimage.convolve1d(plane, _W5, axis=0, mode="nearest"), _W5, axis=1, mode="nearest")
    return blurred[::2, ::2]


def test_pyramid_reduce_equals_library_filter_and_subsample():
    for shape in [(17, 23), (16, 16), (5, 2), (1, 7)]:
        img = wl.uniform_f32(shape, seed=sum(shape)).astype(np.float64)
        np.testing.assert_allclose(oracle.pyramid_reduce(img), _scipy_reduce(img), rtol=0, atol=1e-14)
    assert oracle.pyramid_levels(1920, 1080) == 12 and oracle.pyramid_levels(1, 1) == 1
    assert oracle.pyramid_levels(5, 3) == 4  # 5x3 -> 3x2 -> 2x1 -> 1x1


def test_pyramid_levels_have_variance_4l_minus_1_over_3():
    """The equivalent kernel of level l (response of the sample on the
    origin to an impulse at x, far from the border) sums to 1 and has
    variance (4^l - 1) / 3 per axis: the kernel has unit variance and every
    level doubles the sample spacing."""
    n = 129
    for level in (1, 2, 3):
        h = np.zeros(n)
        for x in range(n):
            img = np.zeros((1, n))
            img[0, x] = 1.0
            g = img
            for _ in range(level):
                g = oracle.pyramid_reduce(g)
            h[x] = g[0, 64 >> level]
        pos = np.arange(n) - 64
        assert abs(h.sum() - 1.0) < 1e-12
        assert abs((h * pos).sum()) < 1e-12
        assert abs((h * pos * pos).sum() - (4 ** level - 1) / 3) < 1e-10


@pytest.mark.parametrize("level_target", [1.0, 2.0, 1.5])
def test_pyramid_output_is_bilinear_interpolation_between_levels(level_target):
    """Uniform sigma with 3 sigma^2 + 1 = 4^L: the output is scipy's order-1
    interpolation of the library-reduced levels, blended by the fraction."""
    H, W = 21, 34
    img = wl.uniform_f32((H, W), seed=12).astype(np.float64)
    sigma = np.sqrt((4.0 ** level_target - 1.0) / 3.0)
    out = oracle.forward_pyramid(img, 3.0, 4.0, sigma, 0.0)
    levels = [img]
    for _ in range(3):
        levels.append(_scipy_reduce(levels[-1]))
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)

    def up(l):
        return ndimage.map_coordinates(levels[l], [yy / 2 ** l, xx / 2 ** l], order=1, mode="nearest")

    l0 = int(np.floor(level_target + 1e-12))
    f = level_target - l0
    ref = up(l0) if f == 0 else (1 - f) * up(l0) + f * up(l0 + 1)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9)


def test_pyramid_identity_constants_linearity_and_sampling():
    img = wl.uniform_f32((18, 27, 3), seed=13).astype(np.float64)
    np.testing.assert_allclose(oracle.forward_pyramid(img, 9.0, 9.0, 0.0, 0.0), img, rtol=0, atol=0)
    c = oracle.forward_pyramid(np.full((18, 27, 3), 0.625), 9.0, 9.0, 0.5, 0.3)
    np.testing.assert_allclose(c, 0.625, rtol=0, atol=1e-14)
    b = wl.uniform_f32((18, 27, 3), seed=14).astype(np.float64)
    lhs = oracle.forward_pyramid(2.0 * img - 0.5 * b, 4.5, 11.0, 0.5, 0.3)
    rhs = 2.0 * oracle.forward_pyramid(img, 4.5, 11.0, 0.5, 0.3) - 0.5 * oracle.forward_pyramid(b, 4.5, 11.0, 0.5, 0.3)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13)
    full = oracle.forward_pyramid(img, 4.5, 11.0, 0.5, 0.3)
    pix = [0, 26, 5 * 27 + 7, 18 * 27 - 1]
    s = oracle.forward_pyramid(img, 4.5, 11.0, 0.5, 0.3, pixels=pix)
    assert np.array_equal(s.reshape(-1, 3)[pix], full.reshape(-1, 3)[pix])
