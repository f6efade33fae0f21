"""Out-of-bounds evidence without compute-sanitizer: every output the library
writes sits between guard bands that must come back untouched (ragged and
misaligned frames, every forward kernel and thread count, batches, adjoint,
per-pixel, pyramid, SSIM, the no-allocation entry point, host buffers), with
no device fault recorded. The same cases then run against the bounds-checked
build (-DFOVEA_BOUNDS), whose kernels check each global store and the
tensor-core kernels' shared-memory stores and record FOVEA_FAULT_BOUNDS
instead of writing out of range."""
import os
import subprocess
import sys

import pytest
import torch

import _canary

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fv():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_08655_gb300 import fovea
    return fovea


def test_guard_bands_intact_and_no_device_fault(fv):
    fails = _canary.run_cases(fv, torch)
    assert not fails, "\n".join(fails)


def test_bounds_checked_build_reports_nothing(fv):
    from paper_2012_08655_gb300 import build
    lib = build.build(bounds=True)
    env = dict(os.environ, FOVEA_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_canary.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "libfovea_bounds.so: 0 failures" in r.stdout
