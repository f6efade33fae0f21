"""Thin ctypes binding of libfovea (``include/fovea.h``) plus autograd glue.

Every step of the foveation path runs in the library's CUDA kernels; this
module only marshals arguments (device pointers of torch tensors, the
current CUDA stream) and raises on error. There is no CPU fallback: if
``libfovea.so`` has not been built, importing this module raises.

Paper: "CUDA-Optimized real-time rendering of a Foveated Visual System"
(arXiv 2012.08655), Section 2 and Algorithm 1 (block-wise foveation), Eq. 1
(the Gaussian filter) and Appendix "Choosing the Standard Deviation" (sigma
law, here sigma = sigma0 + k * eccentricity in pixels).
"""
from __future__ import annotations

import ctypes
import json
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# FOVEA_LIBRARY may name another build of the library (the bounds-checked
# libfovea_bounds.so); by default the package's own libfovea.so.
LIB_PATH = os.environ.get("FOVEA_LIBRARY") or os.path.join(_HERE, "libfovea.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libfovea.so is missing at {LIB_PATH}; build it with "
        "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")

_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
U8_HWC, F32_CHW = 0, 1
MAX_RADIUS = 1023
MAX_BLOCK = 256
# device fault bits (FOVEA_FAULT_* of include/fovea.h), reported by Context.check()
FAULT_SIGMA_RANGE, FAULT_RADIUS_BOUND, FAULT_ADJ_BOUND, FAULT_ORDER = 0x01, 0x02, 0x04, 0x08
FAULT_WORKLIST, FAULT_BUCKETS, FAULT_WAIT, FAULT_PIXEL_RADIUS = 0x10, 0x20, 0x40, 0x80
FAULT_BOUNDS, FAULT_VALUE_RANGE = 0x100, 0x200


LAW_LINEAR, LAW_GEISLER_PERRY, LAW_MAP = 0, 1, 2
GRID_ANCHORED, GRID_CENTRED = 0, 1


class SigmaLaw(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma0", ctypes.c_double), ("k", ctypes.c_double),
                ("e_corner_deg", ctypes.c_double), ("sigma_map", ctypes.c_void_p),
                ("sigma_map_max", ctypes.c_double), ("grid", ctypes.c_int)]


class Frame(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("channels", ctypes.c_int),
                ("format", ctypes.c_int), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("fix_x", ctypes.c_float), ("fix_y", ctypes.c_float),
                ("sigma0", ctypes.c_double), ("k", ctypes.c_double),
                ("grid", ctypes.c_int), ("sigma_map", ctypes.c_void_p), ("sigma_map_max", ctypes.c_double)]


class Config(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("rows_per_chunk", ctypes.c_int),
                ("tensor_cores", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int),
                ("block", ctypes.c_int), ("max_inflight", ctypes.c_int)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("arrival_us", ctypes.c_double), ("admit_us", ctypes.c_double),
                ("start_us", ctypes.c_double), ("done_us", ctypes.c_double),
                ("batch_size", ctypes.c_int), ("status", ctypes.c_int)]


_vp, _i, _f, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
_sig = {
    "fovea_create": (_i, [_i, _i, _i, _i, ctypes.POINTER(SigmaLaw), _i, ctypes.POINTER(_vp)]),
    "fovea_render": (_i, [_vp, _vp, _vp, _f, _f, _vp]),
    "fovea_render_batch": (_i, [_vp, ctypes.POINTER(Frame), _i, _vp]),
    "fovea_reserve": (_i, [_vp, _i, ctypes.c_longlong]),
    "fovea_render_host": (_i, [_vp, _vp, _vp, _f, _f, _vp]),
    "fovea_render_pixelwise": (_i, [_vp, _vp, _vp, _f, _f, _vp]),
    "fovea_render_pyramid": (_i, [_vp, _vp, _vp, _f, _f, _vp]),
    "fovea_ssim": (_i, [_i, _i, _i, _i, _vp, _vp, _d, _vp, _vp, _vp]),
    "fovea_backward": (_i, [_vp, _vp, _vp, _f, _f, _vp]),
    "fovea_backward_batch": (_i, [_vp, ctypes.POINTER(Frame), _i, _vp]),
    "fovea_sigma_table": (_i, [_vp, _f, _f, _vp, _vp, _vp]),
    "fovea_get_config": (_i, [_vp, ctypes.POINTER(Config)]),
    "fovea_set_config": (_i, [_vp, ctypes.POINTER(Config)]),
    "fovea_autotune": (_i, [_vp, _i, ctypes.c_char_p]),
    "fovea_autotune_batch": (_i, [_vp, ctypes.POINTER(Frame), _i, _i, ctypes.c_char_p, ctypes.POINTER(Config)]),
    "fovea_set_kernel_events": (_i, [_vp, _vp, _vp]),
    "fovea_destroy": (None, [_vp]),
    "fovea_render_noalloc": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _d, _d, _f, _f, _vp]),
    "fovea_check": (_i, [_vp, _vp, ctypes.POINTER(ctypes.c_uint)]),
    "fovea_check_async": (_i, [_vp, _vp, ctypes.POINTER(ctypes.c_uint)]),
    "fovea_noalloc_check": (_i, [_vp, ctypes.POINTER(ctypes.c_uint)]),
    "fovea_strerror": (ctypes.c_char_p, [_i]),
    "fovea_last_cuda_error": (_i, []),
    "fovea_build_flags": (_i, []),
    "fovea_measure_fma_rate": (_i, [ctypes.POINTER(_d), _vp]),
    "fovea_gp_law": (_i, [_i, _i, _d, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "fovea_grid": (_i, [_vp, _f, _f, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                        ctypes.POINTER(_i)]),
    "fovea_server_create": (_i, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]),
    "fovea_server_submit": (ctypes.c_longlong, [_vp, ctypes.POINTER(Frame), _d]),
    "fovea_server_wait": (_i, [_vp, ctypes.c_longlong, _i, ctypes.POINTER(RequestTimes)]),
    "fovea_server_now_us": (_d, []),
    "fovea_server_destroy": (None, [_vp]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

# The bounds-checked build (FOVEA_LIBRARY naming libfovea_bounds.so): every
# Context reads its fault word when it closes, and bounds faults are kept in
# BOUNDS_FAULTS for a test harness to report.
BOUNDS_BUILD = bool(_lib.fovea_build_flags() & 1)
BOUNDS_FAULTS: list = []


class FoveaError(RuntimeError):
    def __init__(self, status: int, what: str, faults: int = 0):
        msg = _lib.fovea_strerror(status).decode()
        if faults:
            msg += f" (device faults 0x{faults:02x})"
        elif status == ECUDA:
            msg += f" (cudaError {_lib.fovea_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{status}]")
        self.status = status
        self.faults = faults


def _check(status: int, what: str) -> int:
    if status < 0:
        raise FoveaError(status, what)
    return status


def _check_faults(fn, what: str, *args) -> int:
    """Call a fault-reporting entry point (fovea_check and its forms): raise
    FoveaError carrying the fault word unless it returns OK; return the word."""
    w = ctypes.c_uint(0)
    st = fn(*args, ctypes.byref(w))
    if st < 0:
        raise FoveaError(st, what, int(w.value))
    return int(w.value)


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _fmt_of(t: torch.Tensor) -> int:
    if t.dtype == torch.uint8:
        return U8_HWC
    if t.dtype == torch.float32:
        return F32_CHW
    raise TypeError(f"unsupported dtype {t.dtype}: uint8 (HWC) or float32 (CHW)")


def _shape_of(t: torch.Tensor, fmt: int):
    """(W, H, C) of one frame tensor: uint8 (H, W[, C]) or float32 ([C,] H, W)."""
    if t.dim() == 2:
        h, w = t.shape
        return w, h, 1
    if t.dim() != 3:
        raise ValueError(f"one frame must be 2-D or 3-D, got shape {tuple(t.shape)}")
    if fmt == U8_HWC:
        h, w, c = t.shape
    else:
        c, h, w = t.shape
    return w, h, c


def _require_device_frame(t: torch.Tensor, name: str, device: Optional[int] = None):
    """A contiguous CUDA tensor on `device` (default: the current device),
    the one the library's kernels run on: a pointer into another GPU's memory
    would be an illegal address there."""
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    want = torch.cuda.current_device() if device is None else int(device)
    if t.device.index != want:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the call runs on cuda:{want}")


def _require_host_frame(t: torch.Tensor, name: str):
    if t.is_cuda:
        raise ValueError(f"{name} must be a host (preferably pinned) tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _require_frame_size(t: torch.Tensor, name: str, width: int, height: int, channels: int, fmt: int):
    """The library reads and writes width x height x channels elements of the
    format's type through the tensor's pointer: anything smaller would be
    accessed out of bounds, so the dtype and element count must match."""
    want = torch.uint8 if fmt == U8_HWC else torch.float32
    if t.dtype != want:
        raise TypeError(f"{name} is {t.dtype}, the frame format needs {want}")
    n = int(width) * int(height) * int(channels)
    if t.numel() != n:
        raise ValueError(f"{name} holds {t.numel()} elements; the frame ({width}x{height}x{channels}) has {n}")


def _require_like(t: torch.Tensor, ref: torch.Tensor, name: str):
    """An output (or second operand) that matches the input frame's dtype and size."""
    if t.dtype != ref.dtype or t.numel() != ref.numel():
        raise ValueError(f"{name} ({t.dtype}, {t.numel()} elements) does not match the input "
                         f"({ref.dtype}, {ref.numel()} elements)")


class Context:
    """One fovea context (``fovea_create``): frame shape, format, block side,
    sigma law and grid mode.

    ``law``: LAW_LINEAR (sigma0 + k e), LAW_GEISLER_PERRY (``e_corner`` degrees
    at the frame corner) or LAW_MAP (``sigma_map``: a float32 CUDA tensor of
    per-block sigma on this context's grid, kept alive by the caller;
    ``sigma_map_max`` bounds its values). ``grid``: GRID_ANCHORED or
    GRID_CENTRED (a block centred on the fixation)."""

    def __init__(self, width: int, height: int, channels: int, block: int = 32,
                 sigma0: float = 0.5, k: float = 0.02, fmt: int = U8_HWC, *, law: int = LAW_LINEAR,
                 e_corner: float = 0.0, sigma_map: Optional[torch.Tensor] = None,
                 sigma_map_max: Optional[float] = None, grid: int = GRID_ANCHORED):
        mp, mmax = 0, 0.0
        self.device = torch.cuda.current_device()
        if law == LAW_MAP:
            if sigma_map is None or not sigma_map.is_cuda or sigma_map.dtype != torch.float32:
                raise ValueError("LAW_MAP needs a float32 CUDA sigma_map")
            _require_device_frame(sigma_map, "sigma_map", self.device)
            mp = sigma_map.data_ptr()
            mmax = float(sigma_map.max().item()) if sigma_map_max is None else float(sigma_map_max)
        sl = SigmaLaw(int(law), float(sigma0), float(k), float(e_corner), mp, mmax, int(grid))
        h = _vp()
        _check(_lib.fovea_create(int(width), int(height), int(channels), int(block), ctypes.byref(sl),
                                 int(fmt), ctypes.byref(h)), "fovea_create")
        self._h = h
        self._map = sigma_map
        self.width, self.height, self.channels, self.block = int(width), int(height), int(channels), int(block)
        self.sigma0, self.k, self.fmt = float(sigma0), float(k), int(fmt)
        self.law, self.grid = int(law), int(grid)

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if BOUNDS_BUILD:
                self.record_bounds_faults()
            _lib.fovea_destroy(self._h)
            self._h = _vp()

    def record_bounds_faults(self):
        """Bounds-checked build only: read (and clear) the fault word and keep
        a FOVEA_FAULT_BOUNDS in BOUNDS_FAULTS (other bits are left to check())."""
        w = ctypes.c_uint(0)
        _lib.fovea_check(self._h, None, ctypes.byref(w))
        if w.value & FAULT_BOUNDS:
            BOUNDS_FAULTS.append((self.width, self.height, self.channels, int(w.value)))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- calls
    def _frames(self, pairs, device: bool = True, fmt: Optional[int] = None):
        """Check (tensor, name) pairs against this context's frame (and, for
        device tensors, against the context's device)."""
        for t, name in pairs:
            if device:
                _require_device_frame(t, name, self.device)
            else:
                _require_host_frame(t, name)
            _require_frame_size(t, name, self.width, self.height, self.channels, self.fmt if fmt is None else fmt)

    def check(self, stream=None) -> int:
        """Wait for the stream and read and clear the context's device fault
        word (``fovea_check``). Raises FoveaError (with ``.faults``) when a
        kernel recorded a fault since the last check; returns 0 otherwise."""
        return _check_faults(_lib.fovea_check, "fovea_check", self._h, _stream_handle(stream))

    def check_async(self, stream=None) -> int:
        """Non-blocking form of :meth:`check` (``fovea_check_async``): raises
        for a fault that an earlier call saw land, never waits otherwise."""
        return _check_faults(_lib.fovea_check_async, "fovea_check_async", self._h, _stream_handle(stream))

    def render(self, inp: torch.Tensor, out: torch.Tensor, fix_x: float, fix_y: float, stream=None):
        self._frames([(inp, "input"), (out, "output")])
        _check(_lib.fovea_render(self._h, inp.data_ptr(), out.data_ptr(), float(fix_x), float(fix_y),
                                 _stream_handle(stream)), "fovea_render")
        return out

    def render_pixelwise(self, inp: torch.Tensor, out: torch.Tensor, fix_x: float, fix_y: float, stream=None):
        """Per-pixel ("perfect") foveation of one device frame with this
        context's shape, format and law (``fovea_render_pixelwise``)."""
        self._frames([(inp, "input"), (out, "output")])
        _check(_lib.fovea_render_pixelwise(self._h, inp.data_ptr(), out.data_ptr(), float(fix_x), float(fix_y),
                                           _stream_handle(stream)), "fovea_render_pixelwise")
        return out

    def render_pyramid(self, inp: torch.Tensor, out: torch.Tensor, fix_x: float, fix_y: float, stream=None):
        """Gaussian-pyramid (mipmap) foveation of one device frame with this
        context's shape, format and law (``fovea_render_pyramid``)."""
        self._frames([(inp, "input"), (out, "output")])
        _check(_lib.fovea_render_pyramid(self._h, inp.data_ptr(), out.data_ptr(), float(fix_x), float(fix_y),
                                         _stream_handle(stream)), "fovea_render_pyramid")
        return out

    def render_host(self, inp: torch.Tensor, out: torch.Tensor, fix_x: float, fix_y: float, stream=None):
        self._frames([(inp, "input"), (out, "output")], device=False)
        _check(_lib.fovea_render_host(self._h, inp.data_ptr(), out.data_ptr(), float(fix_x), float(fix_y),
                                      _stream_handle(stream)), "fovea_render_host")
        return out

    def backward(self, grad_out: torch.Tensor, grad_in: torch.Tensor, fix_x: float, fix_y: float, stream=None):
        self._frames([(grad_out, "grad_out"), (grad_in, "grad_in")], fmt=F32_CHW)
        _check(_lib.fovea_backward(self._h, grad_out.data_ptr(), grad_in.data_ptr(), float(fix_x), float(fix_y),
                                   _stream_handle(stream)), "fovea_backward")
        return grad_in

    def grid_shape(self, fix_x: float, fix_y: float):
        """(nby, nbx, oy, ox): block grid for this fixation (``fovea_grid``)."""
        nbx, nby, ox, oy = _i(), _i(), _i(), _i()
        _check(_lib.fovea_grid(self._h, float(fix_x), float(fix_y), ctypes.byref(nbx), ctypes.byref(nby),
                               ctypes.byref(ox), ctypes.byref(oy)), "fovea_grid")
        return nby.value, nbx.value, oy.value, ox.value

    def sigma_table(self, fix_x: float, fix_y: float, stream=None):
        nby, nbx, _, _ = self.grid_shape(fix_x, fix_y)
        sig = torch.empty((nby, nbx), dtype=torch.float32, device="cuda")
        rad = torch.empty((nby, nbx), dtype=torch.int32, device="cuda")
        _check(_lib.fovea_sigma_table(self._h, float(fix_x), float(fix_y), sig.data_ptr(), rad.data_ptr(),
                                      _stream_handle(stream)), "fovea_sigma_table")
        return sig, rad

    def render_batch(self, frames: Sequence["BatchFrame"], stream=None):
        arr = _frames_array(frames, self.device)
        _check(_lib.fovea_render_batch(self._h, arr, len(frames), _stream_handle(stream)), "fovea_render_batch")

    def reserve(self, max_frames: int, max_items: int):
        """Pre-size the batch buffers (frames per batch, (frame, block) items in all)."""
        _check(_lib.fovea_reserve(self._h, int(max_frames), int(max_items)), "fovea_reserve")

    def backward_batch(self, frames: Sequence["BatchFrame"], stream=None):
        arr = _frames_array(frames, self.device)
        _check(_lib.fovea_backward_batch(self._h, arr, len(frames), _stream_handle(stream)), "fovea_backward_batch")

    def set_kernel_events(self, start: Optional[torch.cuda.Event], stop: Optional[torch.cuda.Event]):
        """Bracket the persistent blur kernel of later renders with these events."""
        a = start.cuda_event if start is not None else None
        b = stop.cuda_event if stop is not None else None
        _check(_lib.fovea_set_kernel_events(self._h, a, b), "fovea_set_kernel_events")

    def get_config(self) -> dict:
        c = Config()
        _check(_lib.fovea_get_config(self._h, ctypes.byref(c)), "fovea_get_config")
        return {"threads": c.threads, "ctas_per_sm": c.ctas_per_sm, "rows_per_chunk": c.rows_per_chunk,
                "tensor_cores": c.tensor_cores}

    def set_config(self, threads=256, ctas_per_sm=0, rows_per_chunk=32, tensor_cores=1):
        c = Config(int(threads), int(ctas_per_sm), int(rows_per_chunk), int(tensor_cores))
        _check(_lib.fovea_set_config(self._h, ctypes.byref(c)), "fovea_set_config")

    def autotune(self, iters: int = 20, cache_path: Optional[str] = None) -> dict:
        p = cache_path.encode() if cache_path else None
        _check(_lib.fovea_autotune(self._h, int(iters), p), "fovea_autotune")
        return self.get_config()

    def autotune_batch(self, frames: Sequence["BatchFrame"], iters: int = 3, cache_path: Optional[str] = None) -> dict:
        """Time the configurations on this batch (``fovea_autotune_batch``);
        later batches like it render with the fastest. Returns it."""
        arr = _frames_array(frames, self.device)
        c = Config()
        p = cache_path.encode() if cache_path else None
        _check(_lib.fovea_autotune_batch(self._h, arr, len(frames), int(iters), p, ctypes.byref(c)),
               "fovea_autotune_batch")
        return {"threads": c.threads, "ctas_per_sm": c.ctas_per_sm, "rows_per_chunk": c.rows_per_chunk,
                "tensor_cores": c.tensor_cores}


def batch_context(block: int = 32) -> Context:
    """A batch-only context (``fovea_create`` with width = height = 0)."""
    return Context(0, 0, 3, block)


@dataclass
class BatchFrame:
    inp: torch.Tensor
    out: torch.Tensor
    fix_x: float
    fix_y: float
    sigma0: float
    k: float
    grid: int = GRID_ANCHORED
    sigma_map: Optional[torch.Tensor] = None
    sigma_map_max: float = 0.0


def _frames_array(frames: Sequence[BatchFrame], device: Optional[int] = None):
    if len(frames) == 0:
        raise ValueError("empty batch")
    arr = (Frame * len(frames))()
    keep = []
    for i, fr in enumerate(frames):
        _require_device_frame(fr.inp, f"frame {i} input", device)
        _require_device_frame(fr.out, f"frame {i} output", device)
        _require_like(fr.out, fr.inp, f"frame {i} output")
        if fr.sigma_map is not None:
            _require_device_frame(fr.sigma_map, f"frame {i} sigma map", device)
        fmt = _fmt_of(fr.inp)
        w, h, c = _shape_of(fr.inp, fmt)
        mp = fr.sigma_map.data_ptr() if fr.sigma_map is not None else None
        arr[i] = Frame(w, h, c, fmt, fr.inp.data_ptr(), fr.out.data_ptr(), float(fr.fix_x), float(fr.fix_y),
                       float(fr.sigma0), float(fr.k), int(fr.grid), mp, float(fr.sigma_map_max))
        keep.append(fr)
    return arr


# numpy mirror of the Frame struct (same field offsets and size), so a batch's
# frame records are filled by vectorised assignments instead of one ctypes
# constructor per frame
_FRAME_NP = np.dtype({
    "names": [name for name, _ in Frame._fields_],
    "formats": [{ctypes.c_int: np.int32, ctypes.c_void_p: np.uint64, ctypes.c_float: np.float32,
                 ctypes.c_double: np.float64}[typ] for _, typ in Frame._fields_],
    "offsets": [getattr(Frame, name).offset for name, _ in Frame._fields_],
    "itemsize": ctypes.sizeof(Frame)})


class _FrameRecords:
    """Frame records in a numpy array, passed to the C calls as Frame*."""

    def __init__(self, recs: np.ndarray):
        self.recs = recs
        self.ptr = recs.ctypes.data_as(ctypes.POINTER(Frame))

    def __len__(self):
        return len(self.recs)


def _frames_of_nchw(x: torch.Tensor, y: torch.Tensor, fixes: np.ndarray, sigma0: float, k: float):
    """Frame records of a contiguous float32 [N, C, H, W] batch (input x,
    output y) from the base pointers, without a tensor view per image;
    fixes: float32 [N, 2] (x, y)."""
    n, c, h, w = x.shape
    step = np.uint64(c * h * w * 4)
    idx = np.arange(n, dtype=np.uint64)
    recs = np.zeros(n, dtype=_FRAME_NP)
    recs["width"], recs["height"], recs["channels"], recs["format"] = w, h, c, F32_CHW
    recs["in_"] = np.uint64(x.data_ptr()) + idx * step
    recs["out"] = np.uint64(y.data_ptr()) + idx * step
    recs["fix_x"], recs["fix_y"] = fixes[:, 0], fixes[:, 1]
    recs["sigma0"], recs["k"], recs["grid"] = sigma0, k, GRID_ANCHORED
    return _FrameRecords(recs)


# ------------------------------------------------------------------ functional API
_ctx_cache: dict = {}


def _ctx_for(w, h, c, block, sigma0, k, fmt, grid=GRID_ANCHORED, e_corner=None) -> Context:
    key = (torch.cuda.current_device(), w, h, c, block, float(sigma0), float(k), fmt, int(grid), e_corner)
    ctx = _ctx_cache.get(key)
    if ctx is None:
        if e_corner is None:
            ctx = Context(w, h, c, block, sigma0, k, fmt, grid=grid)
        else:
            ctx = Context(w, h, c, block, 0.0, 0.0, fmt, law=LAW_GEISLER_PERRY, e_corner=e_corner, grid=grid)
        _ctx_cache[key] = ctx
    return ctx


def gp_law(width: int, height: int, e_corner: float):
    """(sigma0, k) of the Geisler-Perry law for this frame size (``fovea_gp_law``)."""
    s0, k = _d(), _d()
    _check(_lib.fovea_gp_law(int(width), int(height), float(e_corner), ctypes.byref(s0), ctypes.byref(k)),
           "fovea_gp_law")
    return s0.value, k.value


def foveate(x: torch.Tensor, fix_x: float, fix_y: float, sigma0: float = 0.5, k: float = 0.02,
            block: int = 32, out: Optional[torch.Tensor] = None, *, grid: int = GRID_ANCHORED,
            e_corner: Optional[float] = None) -> torch.Tensor:
    """Foveate one frame: uint8 (H, W[, C]) or float32 ([C,] H, W), on the GPU.

    ``e_corner`` (degrees at the frame corner) selects the Geisler-Perry law
    instead of (sigma0, k); ``grid`` = GRID_CENTRED centres a block on the
    fixation."""
    _require_device_frame(x, "input")
    fmt = _fmt_of(x)
    w, h, c = _shape_of(x, fmt)
    ctx = _ctx_for(w, h, c, block, sigma0, k, fmt, grid, e_corner)
    if out is None:
        out = torch.empty_like(x)
    return ctx.render(x, out, fix_x, fix_y)


def foveate_pixelwise(x: torch.Tensor, fix_x: float, fix_y: float, sigma0: float = 0.5, k: float = 0.02,
                      out: Optional[torch.Tensor] = None, *, e_corner: Optional[float] = None) -> torch.Tensor:
    """Per-pixel ("perfect") foveation of one frame on the GPU: every pixel
    blurred with the sigma of its own centre (the block-wise map's quality
    reference)."""
    _require_device_frame(x, "input")
    fmt = _fmt_of(x)
    w, h, c = _shape_of(x, fmt)
    ctx = _ctx_for(w, h, c, 32, sigma0, k, fmt, GRID_ANCHORED, e_corner)
    if out is None:
        out = torch.empty_like(x)
    return ctx.render_pixelwise(x, out, fix_x, fix_y)


def foveate_pyramid(x: torch.Tensor, fix_x: float, fix_y: float, sigma0: float = 0.5, k: float = 0.02,
                    out: Optional[torch.Tensor] = None, *, e_corner: Optional[float] = None) -> torch.Tensor:
    """Gaussian-pyramid (mipmap) foveation of one frame on the GPU."""
    _require_device_frame(x, "input")
    fmt = _fmt_of(x)
    w, h, c = _shape_of(x, fmt)
    ctx = _ctx_for(w, h, c, 32, sigma0, k, fmt, GRID_ANCHORED, e_corner)
    if out is None:
        out = torch.empty_like(x)
    return ctx.render_pyramid(x, out, fix_x, fix_y)


def ssim(a: torch.Tensor, b: torch.Tensor, data_range: float = 0.0, want_map: bool = True, stream=None):
    """SSIM of two device frames of one shape and format (``fovea_ssim``):
    returns (map, mean) with the (H, W) float32 map (None unless
    ``want_map``) and the mean over the map as a Python float."""
    _require_device_frame(a, "a")
    _require_device_frame(b, "b")
    _require_like(b, a, "b")
    if a.shape != b.shape or a.dtype != b.dtype:
        raise ValueError("SSIM needs two frames of one shape and dtype")
    fmt = _fmt_of(a)
    w, h, c = _shape_of(a, fmt)
    m = torch.empty((h, w), dtype=torch.float32, device=a.device) if want_map else None
    total = torch.empty(1, dtype=torch.float64, device=a.device)
    _check(_lib.fovea_ssim(w, h, c, fmt, a.data_ptr(), b.data_ptr(), float(data_range),
                           m.data_ptr() if m is not None else None, total.data_ptr(), _stream_handle(stream)),
           "fovea_ssim")
    return m, float(total.item()) / (w * h)


def render_noalloc(x: torch.Tensor, out: torch.Tensor, fix_x: float, fix_y: float, sigma0: float = 0.5,
                   k: float = 0.02, block: int = 32, stream=None) -> torch.Tensor:
    """Foveate one device frame through ``fovea_render_noalloc``: same kernels
    as :func:`foveate`, no memory allocated by the library (its scratch is a
    fixed array inside the library; calls that overlap on the GPU race)."""
    _require_device_frame(x, "input")
    _require_device_frame(out, "output")
    _require_like(out, x, "output")
    fmt = _fmt_of(x)
    w, h, c = _shape_of(x, fmt)
    _check(_lib.fovea_render_noalloc(x.data_ptr(), out.data_ptr(), w, h, c, fmt, int(block), float(sigma0),
                                     float(k), float(fix_x), float(fix_y), _stream_handle(stream)),
           "fovea_render_noalloc")
    return out


def noalloc_check(stream=None) -> int:
    """Wait for the stream and read the device fault word of the latest
    :func:`render_noalloc` call on the current device
    (``fovea_noalloc_check``); raises FoveaError on a fault."""
    return _check_faults(_lib.fovea_noalloc_check, "fovea_noalloc_check", _stream_handle(stream))


def measure_fma_rate(stream=None) -> float:
    """Measured FP32 FMA lane-operations per second of the current GPU
    (``fovea_measure_fma_rate``): the roof of the blur kernels' arithmetic."""
    v = ctypes.c_double(0.0)
    _check(_lib.fovea_measure_fma_rate(ctypes.byref(v), _stream_handle(stream)), "fovea_measure_fma_rate")
    return v.value


def sigma_table(width: int, height: int, fix_x: float, fix_y: float, sigma0: float = 0.5, k: float = 0.02,
                block: int = 32, *, grid: int = GRID_ANCHORED, e_corner: Optional[float] = None):
    """Per-block (sigma float32, radius int32) computed by the sigma-table kernel."""
    return _ctx_for(width, height, 1, block, sigma0, k, F32_CHW, grid, e_corner).sigma_table(fix_x, fix_y)


def take_bounds_faults() -> list:
    """Bounds-checked build: the bounds faults recorded so far (closed
    contexts, and the module's cached contexts, read now), cleared on return.
    Always empty for the regular build."""
    if BOUNDS_BUILD:
        for ctx in list(_ctx_cache.values()):
            if ctx._h.value:
                ctx.record_bounds_faults()
    out = list(BOUNDS_FAULTS)
    BOUNDS_FAULTS.clear()
    return out


def _batch_ctx(block: int) -> Context:
    key = ("batch", torch.cuda.current_device(), block)
    ctx = _ctx_cache.get(key)
    if ctx is None:
        ctx = batch_context(block)
        _ctx_cache[key] = ctx
    return ctx


def foveate_batch(frames: Sequence[BatchFrame], block: int = 32, stream=None):
    """Render frames of mixed sizes in one batched launch sequence."""
    _batch_ctx(block).render_batch(frames, stream)


def autotune_batch(frames: Sequence[BatchFrame], block: int = 32, iters: int = 3) -> dict:
    """Autotune :func:`foveate_batch` for batches like this one."""
    return _batch_ctx(block).autotune_batch(frames, iters)


class FoveaFunction(torch.autograd.Function):
    """Differentiable foveation of a float32 batch [N, C, H, W] with per-image fixations.

    Forward: ``fovea_render_batch``; backward: ``fovea_backward_batch`` (the
    adjoint kernel). Gradients flow to the images only (the fixation and the
    sigma law are constants).
    """

    @staticmethod
    def forward(ctx, x: torch.Tensor, fix: torch.Tensor, sigma0: float, k: float, block: int):
        if x.dtype != torch.float32 or x.dim() != 4:
            raise ValueError("FoveaFunction takes float32 [N, C, H, W]")
        x = x.contiguous()
        _require_device_frame(x, "x")
        fixes = np.ascontiguousarray(fix.detach().cpu().numpy(), dtype=np.float32).reshape(-1, 2)
        if len(fixes) != x.shape[0]:
            raise ValueError("one fixation per image")
        y = torch.empty_like(x)
        bctx = _batch_ctx(block)
        arr = _frames_of_nchw(x, y, fixes, float(sigma0), float(k))
        st = _stream_handle(None)
        _check(_lib.fovea_render_batch(bctx._h, arr.ptr, len(arr), st), "fovea_render_batch")
        bctx.check_async()  # faults of earlier launches surface here without a wait
        ctx.fixes, ctx.sigma0, ctx.k, ctx.block = fixes, sigma0, k, block
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        gy = gy.contiguous()
        _require_device_frame(gy, "grad_output")
        gx = torch.empty_like(gy)
        bctx = _batch_ctx(ctx.block)
        arr = _frames_of_nchw(gy, gx, ctx.fixes, float(ctx.sigma0), float(ctx.k))
        _check(_lib.fovea_backward_batch(bctx._h, arr.ptr, len(arr), _stream_handle(None)), "fovea_backward_batch")
        bctx.check_async()
        return gx, None, None, None, None


def foveate_train(x: torch.Tensor, fix: torch.Tensor, sigma0: float = 0.5, k: float = 0.08,
                  block: int = 32) -> torch.Tensor:
    """Differentiable foveation of x [N, C, H, W] float32 at fixations fix [N, 2] (x, y)."""
    return FoveaFunction.apply(x, fix, sigma0, k, block)


def check_train(block: int = 32, stream=None) -> int:
    """Blocking fault check of the context :func:`foveate_train` uses
    (its forward and backward check without waiting)."""
    return _batch_ctx(block).check(stream)


# ------------------------------------------------------------------ serving
class RequestLog:
    """Append-only JSON-lines file of served requests (one object per line,
    keys in insertion order); flushed after every line."""

    def __init__(self, path: str):
        self._f = open(path, "a", encoding="utf-8")

    def append(self, record: dict):
        if self._f is None:
            raise ValueError("request log is closed")
        self._f.write(json.dumps(record, separators=(",", ":")) + "\n")
        self._f.flush()

    def close(self):
        if self._f is not None:
            self._f.close()
            self._f = None


class Server:
    """Continuous-batching request loop (``fovea_server_*``).

    The host tensors of a request are held by this object from ``submit``
    until ``wait`` reports the request done (or until ``close``), so the
    library's copies never outlive them. With ``log_path`` every request
    that ``wait`` sees finish is appended to that file as one JSON line (its
    id, frame shape, fixation and the library's timestamps and status)."""

    def __init__(self, device_budget_bytes: int = 1 << 30, max_batch: int = 64, block: int = 32,
                 max_inflight: int = 256, log_path: Optional[str] = None):
        self._held = {}
        self._log = RequestLog(log_path) if log_path else None
        self._meta = {}
        cfg = ServerConfig(int(device_budget_bytes), int(max_batch), int(block), int(max_inflight))
        h = _vp()
        _check(_lib.fovea_server_create(ctypes.byref(cfg), ctypes.byref(h)), "fovea_server_create")
        self._h = h

    @staticmethod
    def now_us() -> float:
        return float(_lib.fovea_server_now_us())

    def submit(self, inp: torch.Tensor, out: torch.Tensor, fix_x: float, fix_y: float, sigma0: float,
               k: float, arrival_us: Optional[float] = None, grid: int = GRID_ANCHORED,
               sigma_map: Optional[torch.Tensor] = None, sigma_map_max: float = 0.0) -> int:
        """Submit one host frame; ``sigma_map`` (a float32 device tensor of
        per-block sigma, bounded by ``sigma_map_max``) replaces the linear law."""
        _require_host_frame(inp, "input")
        _require_host_frame(out, "output")
        _require_like(out, inp, "output")
        if sigma_map is not None:
            _require_device_frame(sigma_map, "sigma_map")
        fmt = _fmt_of(inp)
        w, h, c = _shape_of(inp, fmt)
        mp = sigma_map.data_ptr() if sigma_map is not None else None
        fr = Frame(w, h, c, fmt, inp.data_ptr(), out.data_ptr(), float(fix_x), float(fix_y), float(sigma0), float(k),
                   int(grid), mp, float(sigma_map_max))
        t = self.now_us() if arrival_us is None else float(arrival_us)
        rid = _check(int(_lib.fovea_server_submit(self._h, ctypes.byref(fr), t)), "fovea_server_submit")
        self._held[rid] = (inp, out, sigma_map)
        if self._log:
            self._meta[rid] = {"width": w, "height": h, "channels": c, "format": int(fmt),
                               "fix_x": float(fix_x), "fix_y": float(fix_y)}
        return rid

    def wait(self, rid: int, timeout_ms: int = 10000) -> dict:
        t = RequestTimes()
        _check(_lib.fovea_server_wait(self._h, int(rid), int(timeout_ms), ctypes.byref(t)), "fovea_server_wait")
        self._held.pop(int(rid), None)
        times = {"arrival_us": t.arrival_us, "admit_us": t.admit_us, "start_us": t.start_us,
                 "done_us": t.done_us, "batch_size": t.batch_size, "status": t.status}
        if self._log:
            self._log.append({"id": int(rid), **self._meta.pop(int(rid), {}), **times})
        return times

    def close(self):
        if getattr(self, "_log", None):
            self._log.close()
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.fovea_server_destroy(self._h)  # finishes every admitted request first
            self._h = _vp()
        if hasattr(self, "_held"):
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
