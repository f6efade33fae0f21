"""Faults the kernels detect on the device reach the caller as a status.

A render call only enqueues work, so a condition found while the kernels run
(here: a per-block sigma map value outside the bound the caller declared)
is recorded in the context's fault word; fovea_check (blocking) and
fovea_check_async (non-blocking) turn it into FOVEA_EINVAL and clear it, the
serving loop gives it to the requests of the batch, and the next clean call
on the same context reports FOVEA_OK again. The out-of-range values are
clamped on the device, so the output equals the oracle's blur with the
clamped map."""
import numpy as np
import pytest
import torch

import oracle
from paper_2012_08655_gb300 import workloads as wl
from _helpers import assert_u8_close

pytestmark = pytest.mark.gpu

W, H, C, B = 96, 64, 3, 32   # a 3 x 2 block grid
BAD = np.array([[1.0, 2.0, 3.0], [2.5, 40.0, -1.0]], np.float32)   # 40 above the bound, -1 negative
BOUND = 4.0
CLAMPED = np.array([[1.0, 2.0, 3.0], [2.5, 4.0, 0.0]], np.float64)
GOOD = np.array([[1.0, 2.0, 3.0], [2.5, 3.5, 0.5]], np.float32)


@pytest.fixture(scope="module")
def fv():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_08655_gb300 import fovea
    return fovea


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_sigma_map_out_of_range_is_reported_then_cleared(fv, tc):
    img = wl.grating_frame(H, W, C, seed=81)
    m = to_dev(BAD)
    ctx = fv.Context(W, H, C, B, fmt=fv.U8_HWC, law=fv.LAW_MAP, sigma_map=m, sigma_map_max=BOUND)
    ctx.set_config(256, 0, 16 if tc == 3 else 32, tensor_cores=tc)
    assert ctx.check() == 0                      # a fresh context holds no fault
    x = to_dev(img)
    y = torch.empty_like(x)
    ctx.render(x, y, 10.0, 10.0)                 # returns OK: the fault is found on the device
    with pytest.raises(fv.FoveaError) as e:
        ctx.check()
    assert e.value.status == fv.EINVAL
    assert e.value.faults == fv.FAULT_SIGMA_RANGE
    # the blocks were blurred with the clamped values
    assert_u8_close(y.cpu().numpy(), oracle.forward_u8(img, B, 0.0, 0.0, 0.0, 0.0, "hwc", sigma_map=CLAMPED),
                    min_equal=0.99)
    assert np.array_equal(y.cpu().numpy()[32:, 64:], img[32:, 64:])   # clamped to sigma 0: the identity
    sig, rad = ctx.sigma_table(10.0, 10.0)
    with pytest.raises(fv.FoveaError):
        ctx.check()
    assert np.array_equal(sig.cpu().numpy(), CLAMPED.astype(np.float32))
    assert np.array_equal(rad.cpu().numpy(), np.ceil(3.0 * CLAMPED).astype(np.int32))
    # the word was cleared: a valid map on the same context checks clean
    m.copy_(to_dev(GOOD))
    ctx.render(x, y, 10.0, 10.0)
    assert ctx.check() == 0
    assert_u8_close(y.cpu().numpy(), oracle.forward_u8(img, B, 0.0, 0.0, 0.0, 0.0, "hwc",
                                                       sigma_map=GOOD.astype(np.float64)), min_equal=0.99)


def test_non_blocking_check_reports_after_the_work_lands(fv):
    img = wl.grating_frame(H, W, C, seed=82)
    m = to_dev(BAD)
    ctx = fv.Context(W, H, C, B, fmt=fv.U8_HWC, law=fv.LAW_MAP, sigma_map=m, sigma_map_max=BOUND)
    x = to_dev(img)
    y = torch.empty_like(x)
    ctx.render(x, y, 10.0, 10.0)
    assert ctx.check_async() == 0                # enqueues a copy of the word, does not wait
    torch.cuda.synchronize()
    with pytest.raises(fv.FoveaError) as e:
        ctx.check_async()                        # the copy has landed and holds the fault
    assert e.value.status == fv.EINVAL and e.value.faults == fv.FAULT_SIGMA_RANGE
    assert ctx.check() == 0                      # cleared by the report
    m.copy_(to_dev(GOOD))
    ctx.render(x, y, 10.0, 10.0)
    assert ctx.check_async() == 0
    torch.cuda.synchronize()
    assert ctx.check_async() == 0


def test_batch_fault_is_reported_then_cleared(fv):
    img = wl.grating_frame(H, W, C, seed=83)
    x = to_dev(img)
    bad = fv.BatchFrame(x, torch.empty_like(x), 10.0, 10.0, 0.0, 0.0, fv.GRID_ANCHORED, to_dev(BAD), BOUND)
    plain = fv.BatchFrame(x, torch.empty_like(x), 40.0, 30.0, 0.5, 0.04)
    fv.foveate_batch([plain, bad])
    with pytest.raises(fv.FoveaError) as e:
        fv._batch_ctx(32).check()
    assert e.value.status == fv.EINVAL and e.value.faults == fv.FAULT_SIGMA_RANGE
    assert_u8_close(bad.out.cpu().numpy(), oracle.forward_u8(img, B, 0.0, 0.0, 0.0, 0.0, "hwc", sigma_map=CLAMPED),
                    min_equal=0.99)
    assert_u8_close(plain.out.cpu().numpy(), oracle.forward_u8(img, B, 40.0, 30.0, 0.5, 0.04, "hwc"), min_equal=0.99)
    fv.foveate_batch([plain])
    assert fv._batch_ctx(32).check() == 0


def test_served_request_gets_its_batch_fault(fv):
    img = wl.grating_frame(H, W, C, seed=84)
    xin = torch.from_numpy(img).pin_memory()
    outs = [torch.empty_like(xin).pin_memory() for _ in range(2)]
    m = to_dev(BAD)
    with fv.Server(device_budget_bytes=64 << 20, max_batch=8) as srv:
        rid = srv.submit(xin, outs[0], 10.0, 10.0, 0.0, 0.0, sigma_map=m, sigma_map_max=BOUND)
        res = srv.wait(rid)
        assert res["status"] == fv.EINVAL
        rid = srv.submit(xin, outs[1], 40.0, 30.0, 0.5, 0.04)   # the next batch is clean again
        res = srv.wait(rid)
        assert res["status"] == fv.OK
    assert_u8_close(outs[1].numpy(), oracle.forward_u8(img, B, 40.0, 30.0, 0.5, 0.04, "hwc"), min_equal=0.99)
