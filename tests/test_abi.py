"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/fovea.h declares. Only argument checks that return
before touching CUDA are exercised here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fovea.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2012_08655_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(fovea_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fovea_create", "fovea_render", "fovea_render_batch", "fovea_backward",
                     "fovea_destroy", "fovea_strerror", "fovea_sigma_table", "fovea_render_host",
                     "fovea_render_pixelwise", "fovea_render_pyramid", "fovea_ssim"]:
        assert required in names


def test_every_declaration_is_documented():
    """Each entry point in the header sits directly under its own comment
    (meaning, layout, ownership and errors of its arguments)."""
    lines = open(HEADER).read().split("\n")
    undocumented = []
    for i, line in enumerate(lines):
        m = re.match(r"^[A-Za-z_][\w \*]*?\b(fovea_\w+)\s*\(", line)
        if not m or line.strip().startswith(("*", "/*")):
            continue
        j = i - 1
        while j >= 0 and not lines[j].strip():
            j -= 1
        if not lines[j].strip().endswith("*/"):
            undocumented.append(m.group(1))
    assert not undocumented, f"declared without a comment: {undocumented}"


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"libfovea.so lacks {missing}"


def test_strerror_and_invalid_arguments(lib):
    lib.fovea_strerror.restype = ctypes.c_char_p
    assert lib.fovea_strerror(0) == b"ok"
    assert lib.fovea_strerror(-1) == b"invalid argument"
    assert lib.fovea_strerror(-6) == b"unsupported"

    class Law(ctypes.Structure):
        _fields_ = [("kind", ctypes.c_int), ("sigma0", ctypes.c_double), ("k", ctypes.c_double),
                    ("e_corner_deg", ctypes.c_double), ("sigma_map", ctypes.c_void_p),
                    ("sigma_map_max", ctypes.c_double), ("grid", ctypes.c_int)]

    h = ctypes.c_void_p()
    create = lib.fovea_create
    create.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(Law), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    good = Law(0, 0.5, 0.02)
    assert create(64, 64, 3, 32, None, 0, ctypes.byref(h)) == -1           # null law
    assert create(64, 64, 3, 0, ctypes.byref(good), 0, ctypes.byref(h)) == -1   # block <= 0
    assert create(64, 64, 3, 48, ctypes.byref(good), 0, ctypes.byref(h)) == -6  # block > 32, not a multiple of 32
    assert create(64, 64, 3, 288, ctypes.byref(good), 0, ctypes.byref(h)) == -6  # block > 256
    assert create(64, 64, 5, 32, ctypes.byref(good), 0, ctypes.byref(h)) == -1  # channels
    assert create(64, 64, 3, 32, ctypes.byref(good), 7, ctypes.byref(h)) == -1  # format
    assert create(64, 64, 3, 32, ctypes.byref(Law(0, -1.0, 0.02)), 0, ctypes.byref(h)) == -1
    assert create(64, 64, 3, 32, ctypes.byref(Law(0, 0.5, float("nan"))), 0, ctypes.byref(h)) == -1
    assert create(64, 64, 3, 32, ctypes.byref(Law(3, 0.5, 0.02)), 0, ctypes.byref(h)) == -1   # unknown law
    assert create(64, 64, 3, 32, ctypes.byref(Law(0, 0.5, 0.02, 0.0, None, 0.0, 5)), 0, ctypes.byref(h)) == -1
    assert create(0, 0, 3, 32, ctypes.byref(Law(1, 0.0, 0.0, 20.0)), 0, ctypes.byref(h)) == -1  # GP needs a size
    assert create(64, 64, 3, 32, ctypes.byref(Law(1, 0.0, 0.0, -2.0)), 0, ctypes.byref(h)) == -1
    assert create(64, 64, 3, 32, ctypes.byref(Law(2, 0.0, 0.0, 0.0, None, 3.0)), 0, ctypes.byref(h)) == -1
    s0, k = ctypes.c_double(), ctypes.c_double()
    lib.fovea_gp_law.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
    assert lib.fovea_gp_law(1920, 1080, 20.0, ctypes.byref(s0), ctypes.byref(k)) == 0
    import oracle
    assert (s0.value, k.value) == oracle.gp_linear(1920, 1080, 20.0)  # bit for bit
    assert lib.fovea_gp_law(0, 1080, 20.0, ctypes.byref(s0), ctypes.byref(k)) == -1
    assert create(-4, 64, 3, 32, ctypes.byref(good), 0, ctypes.byref(h)) == -1
    assert h.value is None
    lib.fovea_render.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_float] * 2 + [ctypes.c_void_p]
    assert lib.fovea_render(None, None, None, 1.0, 1.0, None) == -1
    lib.fovea_render_pixelwise.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_float] * 2 + [ctypes.c_void_p]
    assert lib.fovea_render_pixelwise(None, None, None, 1.0, 1.0, None) == -1
    lib.fovea_render_pyramid.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_float] * 2 + [ctypes.c_void_p]
    assert lib.fovea_render_pyramid(None, None, None, 1.0, 1.0, None) == -1
    lib.fovea_reserve.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong]
    assert lib.fovea_reserve(None, 4, 1024) == -1
    lib.fovea_ssim.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 2 + [ctypes.c_double] + [ctypes.c_void_p] * 3
    fake = ctypes.c_void_p(16)  # never dereferenced: every call below is refused on the host
    assert lib.fovea_ssim(8, 8, 3, 0, None, fake, 0.0, fake, None, None) == -1      # null image
    assert lib.fovea_ssim(8, 8, 5, 0, fake, fake, 0.0, fake, None, None) == -1      # channels
    assert lib.fovea_ssim(8, 8, 3, 9, fake, fake, 0.0, fake, None, None) == -1      # format
    assert lib.fovea_ssim(8, 8, 3, 0, fake, fake, 0.0, None, None, None) == -1      # no output
    assert lib.fovea_ssim(0, 8, 3, 0, fake, fake, 0.0, fake, None, None) == -1      # empty


def test_fault_bits_and_checks(lib):
    """The FOVEA_FAULT_* bits of the header are distinct single bits, the
    binding's constants equal them, and the checks refuse a null context on
    the host (the status mapping itself needs a device: tests/test_gpu_faults.py)."""
    text = open(HEADER).read()
    bits = {n: int(v, 16) for n, v in re.findall(r"#define FOVEA_FAULT_(\w+)\s+(0x[0-9a-fA-F]+)u", text)}
    assert len(bits) == 10 and len(set(bits.values())) == 10
    assert all(v & (v - 1) == 0 for v in bits.values())
    from paper_2012_08655_gb300 import fovea
    for n, v in bits.items():
        assert getattr(fovea, "FAULT_" + n) == v
    w = ctypes.c_uint(7)
    lib.fovea_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint)]
    assert lib.fovea_check(None, None, ctypes.byref(w)) == -1 and w.value == 0
    w.value = 7
    lib.fovea_check_async.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint)]
    assert lib.fovea_check_async(None, None, ctypes.byref(w)) == -1 and w.value == 0


def test_python_binding_imports_without_gpu():
    from paper_2012_08655_gb300 import fovea
    assert fovea.MAX_RADIUS == 1023


def test_regular_build_reports_no_bounds_checks():
    """fovea_build_flags tells the bounds-checked build (FOVEA_BOUNDS) from the
    regular one; the binding keys its bounds-fault bookkeeping on it."""
    from paper_2012_08655_gb300 import fovea
    expect = 1 if "bounds" in os.path.basename(fovea.LIB_PATH) else 0
    assert fovea._lib.fovea_build_flags() == expect
    assert fovea.BOUNDS_BUILD == bool(expect)
    assert fovea.take_bounds_faults() == []
