"""Argument checks of the Python binding, on the CPU: the library reads and
writes as many elements as the frame has through the tensors' pointers, so
the binding refuses tensors of the wrong dtype, size, device or layout before
any library call."""
import pytest
import torch

from paper_2012_08655_gb300 import fovea as fv


def test_frame_size_check():
    fv._require_frame_size(torch.zeros((10, 12, 3), dtype=torch.uint8), "x", 12, 10, 3, fv.U8_HWC)
    fv._require_frame_size(torch.zeros((10, 12), dtype=torch.uint8), "x", 12, 10, 1, fv.U8_HWC)
    fv._require_frame_size(torch.zeros((3, 10, 12), dtype=torch.float32), "x", 12, 10, 3, fv.F32_CHW)
    fv._require_frame_size(torch.zeros((1, 10, 12), dtype=torch.float32), "x", 12, 10, 1, fv.F32_CHW)
    with pytest.raises(ValueError):
        fv._require_frame_size(torch.zeros((10, 11, 3), dtype=torch.uint8), "x", 12, 10, 3, fv.U8_HWC)
    with pytest.raises(TypeError):
        fv._require_frame_size(torch.zeros((10, 12, 3), dtype=torch.float32), "x", 12, 10, 3, fv.U8_HWC)
    with pytest.raises(TypeError):
        fv._require_frame_size(torch.zeros((3, 10, 12), dtype=torch.float64), "x", 12, 10, 3, fv.F32_CHW)


def test_host_frame_and_like_checks():
    a = torch.zeros((8, 6, 3), dtype=torch.uint8)
    fv._require_host_frame(a, "a")
    with pytest.raises(ValueError):
        fv._require_host_frame(a.transpose(0, 1), "a")  # not contiguous
    fv._require_like(torch.empty_like(a), a, "b")
    with pytest.raises(ValueError):
        fv._require_like(torch.zeros((8, 6, 2), dtype=torch.uint8), a, "b")
    with pytest.raises(ValueError):
        fv._require_like(torch.zeros((8, 6, 3), dtype=torch.float32), a, "b")
    with pytest.raises(ValueError):
        fv._require_device_frame(a, "a")  # a host tensor where a device one is needed


def _bare(cls, **attrs):
    obj = cls.__new__(cls)  # no library handle: every check below must fire first
    for k, v in attrs.items():
        setattr(obj, k, v)
    return obj


def test_context_refuses_mismatched_frames_before_the_library():
    ctx = _bare(fv.Context, width=12, height=10, channels=3, fmt=fv.U8_HWC, device=0)
    good = torch.zeros((10, 12, 3), dtype=torch.uint8)
    ctx._frames([(good, "input"), (torch.empty_like(good), "output")], device=False)
    with pytest.raises(ValueError):
        ctx.render_host(good, torch.zeros((10, 12, 1), dtype=torch.uint8), 1.0, 1.0)
    with pytest.raises(ValueError):
        ctx.render_host(torch.zeros((9, 12, 3), dtype=torch.uint8), good, 1.0, 1.0)
    with pytest.raises(ValueError):
        ctx.render(good, torch.empty_like(good), 1.0, 1.0)  # host tensors for a device call
    f32 = _bare(fv.Context, width=12, height=10, channels=3, fmt=fv.F32_CHW, device=0)
    with pytest.raises(TypeError):
        f32._frames([(good, "grad_out")], device=False, fmt=fv.F32_CHW)


def test_server_refuses_mismatched_output_before_the_library():
    srv = _bare(fv.Server, _held={})
    inp = torch.zeros((10, 12, 3), dtype=torch.uint8)
    with pytest.raises(ValueError):
        srv.submit(inp, torch.zeros((10, 12), dtype=torch.uint8), 1.0, 1.0, 0.5, 0.02)
    with pytest.raises(ValueError):
        srv.submit(inp.transpose(0, 1), torch.empty_like(inp), 1.0, 1.0, 0.5, 0.02)
    assert srv._held == {}


class _FakeDeviceTensor:
    """Stands in for a contiguous CUDA tensor on a given device index (no GPU
    is needed: the device check must fire before anything else)."""

    is_cuda = True

    def __init__(self, index):
        self.device = torch.device("cuda", index)

    def is_contiguous(self):
        return True


def test_device_tensors_must_be_on_the_call_device(monkeypatch):
    fv._require_device_frame(_FakeDeviceTensor(1), "x", 1)
    with pytest.raises(ValueError, match="cuda:1"):
        fv._require_device_frame(_FakeDeviceTensor(1), "x", 0)
    # default: the current device
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 2)
    fv._require_device_frame(_FakeDeviceTensor(2), "x")
    with pytest.raises(ValueError):
        fv._require_device_frame(_FakeDeviceTensor(0), "x")


def test_context_refuses_tensors_of_another_device():
    ctx = _bare(fv.Context, width=12, height=10, channels=3, fmt=fv.U8_HWC, device=0)
    other = _FakeDeviceTensor(1)
    with pytest.raises(ValueError, match="cuda:1"):
        ctx._frames([(other, "input")])


def test_fault_error_carries_the_word():
    e = fv.FoveaError(fv.EINVAL, "fovea_check", fv.FAULT_SIGMA_RANGE)
    assert e.status == fv.EINVAL and e.faults == fv.FAULT_SIGMA_RANGE
    assert "0x01" in str(e)


def test_request_log_writes_one_json_object_per_line(tmp_path):
    """The serving loop's optional request log (Server(log_path=...)):
    append-only JSON lines, readable back record for record."""
    import json
    from paper_2012_08655_gb300.fovea import RequestLog
    path = tmp_path / "requests.jsonl"
    log = RequestLog(str(path))
    recs = [{"id": 0, "width": 84, "height": 84, "channels": 1, "arrival_us": 1.5, "done_us": 90.25, "status": 0},
            {"id": 1, "width": 1920, "height": 1080, "channels": 3, "arrival_us": 2.0, "done_us": 310.0, "status": 0}]
    for r in recs:
        log.append(r)
    log.close()
    lines = path.read_text().splitlines()
    assert [json.loads(l) for l in lines] == recs
    log2 = RequestLog(str(path))      # appends, never truncates
    log2.append({"id": 2})
    log2.close()
    assert len(path.read_text().splitlines()) == 3


def test_frame_records_match_the_ctypes_struct():
    """The numpy frame records of the autograd path have the C struct's
    layout: each record's bytes equal a ctypes Frame built field by field."""
    import ctypes
    import numpy as np
    import torch
    from paper_2012_08655_gb300 import fovea as fv
    x = torch.zeros((3, 2, 5, 8), dtype=torch.float32)
    y = torch.zeros_like(x)
    fixes = np.array([[1.5, 2.25], [-3.0, 7.125], [100.0, 0.5]], np.float32)
    recs = fv._frames_of_nchw(x, y, fixes, 0.5, 0.08)
    assert len(recs) == 3 and recs.recs.itemsize == ctypes.sizeof(fv.Frame)
    step = 2 * 5 * 8 * 4
    for i in range(3):
        want = fv.Frame(8, 5, 2, fv.F32_CHW, x.data_ptr() + i * step, y.data_ptr() + i * step,
                        float(fixes[i, 0]), float(fixes[i, 1]), 0.5, 0.08, fv.GRID_ANCHORED, None, 0.0)
        assert recs.recs[i].tobytes() == bytes(want)
    # and the pointer handed to the C calls is the array's first record
    assert ctypes.addressof(recs.ptr.contents) == recs.recs.ctypes.data
