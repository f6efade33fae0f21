"""FP64 CPU oracle for block-wise foveated Gaussian blur (ctypes binding).

TEST INFRASTRUCTURE ONLY: the slow, plain restatement of the method that the
CUDA library is checked against. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package. It shares no
code with the CUDA path and never imports it.

What the functions compute is stated in ``fovea_oracle.c`` (paper Section 2,
Algorithm 1, Eq. 1 and the truncation/normalisation paragraph after it, and
the sigma law of Appendix "Choosing the Standard Deviation"). In short:

    sigma_b = sigma0 + k * |centre_b - fixation|      (binary64, no FMA)
    r_b     = ceil(3 * sigma_b)
    out(p)  = sum_{|i|,|j| <= r_b} w_i w_j / S^2 * in(clamp(p + (i, j)))

written as a direct 2D sum per output pixel, and its adjoint as a scatter.
Per-pixel foveation (Section 3.1's quality reference) is the same sum with
sigma taken at every pixel's own centre; ``ssim_map`` is the SSIM of Wang et
al. (2004) with its standard 11x11, sigma 1.5 Gaussian window;
``forward_pyramid`` is the Gaussian-pyramid (mipmap) foveation the paper
compares against: a Burt-Adelson pyramid sampled at level log4(3 sigma^2 + 1).

Parity status: every function here is pinned by tests under ``tests/``
(scipy's uniform Gaussian filter, brute-force unit-vector matrices, closed
forms and invariants; for SSIM, closed forms of constant and affine pairs
with local moments from scipy; for the pyramid, scipy's filter-and-subsample
and order-1 interpolation and the closed-form level variance); none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fovea_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, binary64, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
            lib.oracle_sigma_table.argtypes = [i, i, i, d, d, d, d, p, p]
            lib.oracle_sigma_table.restype = None
            lib.oracle_taps.argtypes = [d, i, p]
            lib.oracle_taps.restype = None
            lib.oracle_forward.argtypes = [p, p, i, i, i, l, l, l, i, d, d, d, d, p, i, i]
            lib.oracle_forward.restype = None
            lib.oracle_adjoint.argtypes = [p, p, i, i, i, l, l, l, i, d, d, d, d, i]
            lib.oracle_adjoint.restype = None
            lib.oracle_quantize_u8.argtypes = [p, p, l]
            lib.oracle_quantize_u8.restype = None
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = i
            lib.oracle_sigma_table_ex.argtypes = [i, i, i, i, i, d, d, d, d, p, p, p]
            lib.oracle_sigma_table_ex.restype = None
            lib.oracle_forward_ex.argtypes = [p, p, i, i, i, l, l, l, i, i, i, d, d, d, d, p, p, i, i]
            lib.oracle_forward_ex.restype = None
            lib.oracle_adjoint_ex.argtypes = [p, p, i, i, i, l, l, l, i, i, i, d, d, d, d, p, i]
            lib.oracle_adjoint_ex.restype = None
            lib.oracle_gp_sigma.argtypes = [d, i, i, d]
            lib.oracle_gp_sigma.restype = d
            lib.oracle_gp_linear.argtypes = [i, i, d, ctypes.POINTER(d), ctypes.POINTER(d)]
            lib.oracle_gp_linear.restype = None
            lib.oracle_centred_origin.argtypes = [d, i]
            lib.oracle_centred_origin.restype = i
            lib.oracle_pixel_sigma.argtypes = [i, i, d, d, d, d, ctypes.POINTER(d), ctypes.POINTER(i)]
            lib.oracle_pixel_sigma.restype = None
            lib.oracle_forward_pixel.argtypes = [p, p, i, i, i, l, l, l, d, d, d, d, p, l, i]
            lib.oracle_forward_pixel.restype = None
            lib.oracle_ssim_map.argtypes = [p, p, i, i, i, l, l, l, d, p, i]
            lib.oracle_ssim_map.restype = None
            lib.oracle_pyramid_levels.argtypes = [i, i]
            lib.oracle_pyramid_levels.restype = i
            lib.oracle_pyramid_reduce.argtypes = [p, i, i, p]
            lib.oracle_pyramid_reduce.restype = None
            lib.oracle_forward_pyramid.argtypes = [p, p, i, i, i, l, l, l, d, d, d, d, p, l]
            lib.oracle_forward_pyramid.restype = None
            _lib = lib
    return _lib


def max_threads() -> int:
    """Number of OpenMP threads the oracle uses by default."""
    return int(_load().oracle_max_threads())


def grid_shape(width: int, height: int, block: int, origin=(0, 0)) -> tuple[int, int]:
    """(blocks along y, blocks along x) for grid origin offsets (ox, oy)."""
    ox, oy = origin
    return (height + oy + block - 1) // block, (width + ox + block - 1) // block


def _map_arg(sigma_map, shape):
    if sigma_map is None:
        return None, None
    m = np.ascontiguousarray(np.asarray(sigma_map, dtype=np.float64))
    if m.shape != shape:
        raise ValueError(f"sigma map of shape {m.shape}, expected {shape}")
    return m, m.ctypes.data


def sigma_table(width, height, block, fix_x, fix_y, sigma0, k, origin=(0, 0), sigma_map=None):
    """Per-block sigma (float64) and radius (int32), shape (nby, nbx).

    ``origin`` = (ox, oy): grid origin offsets; ``sigma_map``: per-block
    sigma replacing the law."""
    nby, nbx = grid_shape(width, height, block, origin)
    sig = np.zeros((nby, nbx), np.float64)
    rad = np.zeros((nby, nbx), np.int32)
    keep, mp = _map_arg(sigma_map, (nby, nbx))
    _load().oracle_sigma_table_ex(width, height, block, int(origin[0]), int(origin[1]), float(fix_x), float(fix_y),
                                  float(sigma0), float(k), mp, sig.ctypes.data, rad.ctypes.data)
    return sig, rad


def gp_sigma(d, width, height, e_corner):
    """Geisler-Perry sigma at pixel distance d, by the literal chain of Eqs. 2-6."""
    return float(_load().oracle_gp_sigma(float(d), int(width), int(height), float(e_corner)))


def gp_linear(width, height, e_corner):
    """(sigma0, k) of the Geisler-Perry law written as sigma = sigma0 + k d."""
    s0, k = ctypes.c_double(), ctypes.c_double()
    _load().oracle_gp_linear(int(width), int(height), float(e_corner), ctypes.byref(s0), ctypes.byref(k))
    return s0.value, k.value


def centred_origin(fix, block):
    """Grid origin offset that centres a fragment on fixation coordinate ``fix``."""
    return int(_load().oracle_centred_origin(float(fix), int(block)))


def taps(sigma: float, r: int) -> np.ndarray:
    """Normalised taps for offsets -r..r (float64, length 2r+1)."""
    w = np.zeros(2 * max(r, 0) + 1, np.float64)
    _load().oracle_taps(float(sigma), int(r), w.ctypes.data)
    return w


def _geometry(img: np.ndarray, layout: str):
    """Return (H, W, C, sy, sx, sc) in elements for a C-contiguous array."""
    if img.ndim == 2:
        H, W = img.shape
        return H, W, 1, W, 1, 0
    if layout == "hwc":
        H, W, C = img.shape
        return H, W, C, W * C, C, 1
    if layout == "chw":
        C, H, W = img.shape
        return H, W, C, W, 1, H * W
    raise ValueError(f"unknown layout {layout!r}")


def forward(img, block, fix_x, fix_y, sigma0, k, layout="hwc", blocks=None, nthreads=0, origin=(0, 0),
            sigma_map=None):
    """Foveated blur of one image in binary64.

    ``img`` is (H, W), (H, W, C) for layout 'hwc' or (C, H, W) for 'chw'; any
    real dtype (converted exactly to float64). ``blocks`` optionally lists
    row-major block indices to compute; other pixels of the result are NaN.
    ``origin`` / ``sigma_map`` as in :func:`sigma_table`.
    """
    x = np.ascontiguousarray(img, dtype=np.float64)
    H, W, C, sy, sx, sc = _geometry(x, layout)
    out = np.full_like(x, np.nan)
    if blocks is None:
        bl, nl = None, 0
    else:
        barr = np.ascontiguousarray(np.asarray(blocks, dtype=np.int32))
        bl, nl = barr.ctypes.data, int(barr.size)
    keep, mp = _map_arg(sigma_map, grid_shape(W, H, block, origin))
    _load().oracle_forward_ex(x.ctypes.data, out.ctypes.data, W, H, C, sy, sx, sc, int(block), int(origin[0]),
                              int(origin[1]), float(fix_x), float(fix_y), float(sigma0), float(k), mp, bl, nl,
                              int(nthreads))
    return out


def adjoint(g_out, block, fix_x, fix_y, sigma0, k, layout="chw", nthreads=0, origin=(0, 0), sigma_map=None):
    """Transpose of :func:`forward` applied to ``g_out`` (binary64)."""
    g = np.ascontiguousarray(g_out, dtype=np.float64)
    H, W, C, sy, sx, sc = _geometry(g, layout)
    out = np.zeros_like(g)
    keep, mp = _map_arg(sigma_map, grid_shape(W, H, block, origin))
    _load().oracle_adjoint_ex(g.ctypes.data, out.ctypes.data, W, H, C, sy, sx, sc, int(block), int(origin[0]),
                              int(origin[1]), float(fix_x), float(fix_y), float(sigma0), float(k), mp, int(nthreads))
    return out


def quantize_u8(v) -> np.ndarray:
    """Nearest integer (halves up), clamped to [0, 255], as uint8."""
    x = np.ascontiguousarray(v, dtype=np.float64)
    q = np.zeros(x.shape, np.uint8)
    _load().oracle_quantize_u8(x.ctypes.data, q.ctypes.data, int(x.size))
    return q


def forward_u8(img_u8, block, fix_x, fix_y, sigma0, k, layout="hwc", blocks=None, nthreads=0, origin=(0, 0),
               sigma_map=None):
    """Foveated blur of a uint8 image, coded back to uint8.

    With ``blocks`` given, pixels outside the listed blocks come back as 0.
    """
    v = forward(img_u8, block, fix_x, fix_y, sigma0, k, layout, blocks, nthreads, origin, sigma_map)
    return quantize_u8(np.nan_to_num(v, nan=0.0))


def pixel_sigma(x, y, fix_x, fix_y, sigma0, k):
    """(sigma, radius) of pixel (x, y) under per-pixel foveation."""
    sg, r = ctypes.c_double(), ctypes.c_int()
    _load().oracle_pixel_sigma(int(x), int(y), float(fix_x), float(fix_y), float(sigma0), float(k),
                               ctypes.byref(sg), ctypes.byref(r))
    return sg.value, r.value


def forward_pixel(img, fix_x, fix_y, sigma0, k, layout="hwc", pixels=None, nthreads=0):
    """Per-pixel ("perfect") foveation in binary64: every pixel blurred with
    the sigma of its own centre. ``pixels`` optionally lists row-major pixel
    indices y * W + x to compute; other pixels of the result are NaN."""
    x = np.ascontiguousarray(img, dtype=np.float64)
    H, W, C, sy, sx, sc = _geometry(x, layout)
    out = np.full_like(x, np.nan)
    if pixels is None:
        pl, nl = None, 0
    else:
        parr = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        pl, nl = parr.ctypes.data, int(parr.size)
    _load().oracle_forward_pixel(x.ctypes.data, out.ctypes.data, W, H, C, sy, sx, sc, float(fix_x), float(fix_y),
                                 float(sigma0), float(k), pl, nl, int(nthreads))
    return out


def forward_pixel_u8(img_u8, fix_x, fix_y, sigma0, k, layout="hwc", pixels=None, nthreads=0):
    """Per-pixel foveation of a uint8 image, coded back to uint8 (unlisted
    pixels come back as 0)."""
    v = forward_pixel(img_u8, fix_x, fix_y, sigma0, k, layout, pixels, nthreads)
    return quantize_u8(np.nan_to_num(v, nan=0.0))


def ssim_map(a, b, data_range, layout="hwc", nthreads=0):
    """SSIM map (H, W) of two images of equal shape, binary64: 11x11 Gaussian
    window (sigma 1.5), C1 = (0.01 L)^2, C2 = (0.03 L)^2, clamp-to-edge
    border, mean over channels."""
    x = np.ascontiguousarray(a, dtype=np.float64)
    y = np.ascontiguousarray(b, dtype=np.float64)
    if x.shape != y.shape:
        raise ValueError("images differ in shape")
    H, W, C, sy, sx, sc = _geometry(x, layout)
    m = np.zeros((H, W), np.float64)
    _load().oracle_ssim_map(x.ctypes.data, y.ctypes.data, W, H, C, sy, sx, sc, float(data_range), m.ctypes.data,
                            int(nthreads))
    return m


def pyramid_levels(width, height):
    """Levels of a width x height Gaussian pyramid down to 1 x 1 (level 0 included)."""
    return int(_load().oracle_pyramid_levels(int(width), int(height)))


def pyramid_reduce(plane):
    """One REDUCE (5-tap (1,4,6,4,1)/16 kernel, clamp, subsample by two) of a 2-D plane."""
    x = np.ascontiguousarray(plane, dtype=np.float64)
    H, W = x.shape
    out = np.zeros(((H + 1) // 2, (W + 1) // 2), np.float64)
    _load().oracle_pyramid_reduce(x.ctypes.data, W, H, out.ctypes.data)
    return out


def forward_pyramid(img, fix_x, fix_y, sigma0, k, layout="hwc", pixels=None):
    """Gaussian-pyramid (mipmap) foveation in binary64: each pixel
    interpolated from the pyramid at level log4(3 sigma_p^2 + 1). ``pixels``
    optionally lists row-major pixel indices; others come back NaN."""
    x = np.ascontiguousarray(img, dtype=np.float64)
    H, W, C, sy, sx, sc = _geometry(x, layout)
    out = np.full_like(x, np.nan)
    if pixels is None:
        pl, nl = None, 0
    else:
        parr = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        pl, nl = parr.ctypes.data, int(parr.size)
    _load().oracle_forward_pyramid(x.ctypes.data, out.ctypes.data, W, H, C, sy, sx, sc, float(fix_x), float(fix_y),
                                   float(sigma0), float(k), pl, nl)
    return out


def forward_pyramid_u8(img_u8, fix_x, fix_y, sigma0, k, layout="hwc", pixels=None):
    """Pyramid foveation of a uint8 image, coded back to uint8 (unlisted pixels 0)."""
    v = forward_pyramid(img_u8, fix_x, fix_y, sigma0, k, layout, pixels)
    return quantize_u8(np.nan_to_num(v, nan=0.0))
