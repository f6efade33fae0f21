"""GPU parity of the other sigma laws and of the fixation-centred block grid
(the Geisler-Perry law of Eqs. 2-6, per-block sigma maps, Algorithm 1's
grid shifted to centre a fragment on the fixation) against the FP64 oracle,
through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2012_08655_gb300 import workloads as wl
from _helpers import assert_f32_close, assert_u8_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_08655_gb300 import fovea
    return fovea


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_centred_grid_sigma_table_bit_exact(fv):
    g = wl.rng(21)
    for _ in range(30):
        W, H = int(g.integers(8, 1500)), int(g.integers(8, 1500))
        B = int(g.choice([8, 16, 32]))
        fx, fy = np.float32(g.uniform(-50, W + 50)), np.float32(g.uniform(-50, H + 50))
        ctx = fv.Context(W, H, 1, B, 0.5, 0.03, fv.F32_CHW, grid=fv.GRID_CENTRED)
        nby, nbx, oy, ox = ctx.grid_shape(float(fx), float(fy))
        assert (ox, oy) == (oracle.centred_origin(fx, B), oracle.centred_origin(fy, B))
        sig, rad = ctx.sigma_table(float(fx), float(fy))
        osig, orad = oracle.sigma_table(W, H, B, fx, fy, 0.5, 0.03, origin=(ox, oy))
        assert sig.shape == osig.shape == (nby, nbx)
        assert np.array_equal(rad.cpu().numpy(), orad)
        assert np.array_equal(sig.cpu().numpy(), osig.astype(np.float32))


def test_geisler_perry_sigma_table_bit_exact(fv):
    for (W, H, ec, fx, fy) in [(1920, 1080, 20.0, 960.0, 540.0), (640, 480, 60.0, 10.5, 400.25),
                               (224, 224, 5.0, 112.0, 30.0)]:
        s0, k = oracle.gp_linear(W, H, ec)
        assert fv.gp_law(W, H, ec) == (s0, k)
        sig, rad = fv.sigma_table(W, H, fx, fy, block=32, e_corner=ec)
        osig, orad = oracle.sigma_table(W, H, 32, np.float32(fx), np.float32(fy), s0, k)
        assert np.array_equal(rad.cpu().numpy(), orad)
        assert np.array_equal(sig.cpu().numpy(), osig.astype(np.float32))


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
@pytest.mark.parametrize("W,H,C,B,fx,fy,k", [
    (640, 360, 3, 32, 300.4, 170.6, 0.03),
    (129, 77, 1, 16, 64.0, 38.0, 0.05),
    (200, 150, 4, 8, -20.0, 10.0, 0.08),
])
def test_centred_grid_u8_matches_oracle(fv, tc, W, H, C, B, fx, fy, k):
    img = wl.grating_frame(H, W, C, seed=W + B)
    ctx = fv.Context(W, H, C, B, 0.5, k, fv.U8_HWC, grid=fv.GRID_CENTRED)
    ctx.set_config(256, 0, 16 if tc == 3 else 32, tensor_cores=tc)
    x = to_dev(img)
    y = torch.empty_like(x)
    ctx.render(x, y, fx, fy)
    torch.cuda.synchronize()
    org = (oracle.centred_origin(np.float32(fx), B), oracle.centred_origin(np.float32(fy), B))
    ref = oracle.forward_u8(img, B, fx, fy, 0.5, k, "hwc", origin=org)
    assert_u8_close(y.cpu().numpy(), ref, min_equal=0.99)


def test_centred_grid_f32_forward_and_backward(fv):
    W, H, C, B = 96, 80, 3, 16
    img = wl.uniform_f32((C, H, W), seed=31)
    gout = wl.uniform_f32((C, H, W), seed=32)
    fx, fy = 37.3, 51.9
    ctx = fv.Context(W, H, C, B, 0.4, 0.06, fv.F32_CHW, grid=fv.GRID_CENTRED)
    y = torch.empty(C, H, W, device="cuda")
    ctx.render(to_dev(img), y, fx, fy)
    gin = torch.empty(C, H, W, device="cuda")
    ctx.backward(to_dev(gout), gin, fx, fy)
    torch.cuda.synchronize()
    org = (oracle.centred_origin(np.float32(fx), B), oracle.centred_origin(np.float32(fy), B))
    assert_f32_close(y.cpu().numpy(), oracle.forward(img, B, fx, fy, 0.4, 0.06, "chw", origin=org))
    ref = oracle.adjoint(gout, B, fx, fy, 0.4, 0.06, "chw", origin=org)
    np.testing.assert_allclose(gin.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_geisler_perry_frame_matches_oracle(fv, tc):
    W, H, ec = 640, 480, 30.0
    img = wl.grating_frame(H, W, 3, seed=41)
    ctx = fv.Context(W, H, 3, 32, fmt=fv.U8_HWC, law=fv.LAW_GEISLER_PERRY, e_corner=ec)
    ctx.set_config(256, 0, 16 if tc == 3 else 32, tensor_cores=tc)
    x = to_dev(img)
    y = torch.empty_like(x)
    ctx.render(x, y, 500.0, 100.0)
    torch.cuda.synchronize()
    s0, k = oracle.gp_linear(W, H, ec)
    assert_u8_close(y.cpu().numpy(), oracle.forward_u8(img, 32, 500.0, 100.0, s0, k, "hwc"), min_equal=0.99)


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_sigma_map_matches_oracle(fv, tc):
    W, H, C, B = 300, 200, 3, 32
    g = wl.rng(51)
    nby, nbx = (H + B - 1) // B, (W + B - 1) // B
    smap = g.uniform(0.0, 9.0, size=(nby, nbx)).astype(np.float32)
    smap[0, 0] = 0.0                      # identity block
    img = wl.grating_frame(H, W, C, seed=52)
    ctx = fv.Context(W, H, C, B, fmt=fv.U8_HWC, law=fv.LAW_MAP, sigma_map=to_dev(smap))
    ctx.set_config(256, 0, 16 if tc == 3 else 32, tensor_cores=tc)
    x = to_dev(img)
    y = torch.empty_like(x)
    ctx.render(x, y, 0.0, 0.0)
    sig, rad = ctx.sigma_table(0.0, 0.0)
    torch.cuda.synchronize()
    osig, orad = oracle.sigma_table(W, H, B, 0.0, 0.0, 0.0, 0.0, sigma_map=smap.astype(np.float64))
    assert np.array_equal(rad.cpu().numpy(), orad)
    assert np.array_equal(sig.cpu().numpy(), smap)
    ref = oracle.forward_u8(img, B, 0.0, 0.0, 0.0, 0.0, "hwc", sigma_map=smap.astype(np.float64))
    assert_u8_close(y.cpu().numpy(), ref, min_equal=0.99)
    assert np.array_equal(y.cpu().numpy()[:B, :B], img[:B, :B])  # sigma 0: identity


def test_batch_mixes_grids_laws_and_maps(fv):
    B = 32
    specs = [(224, 224, fv.GRID_CENTRED, None), (300, 170, fv.GRID_ANCHORED, None),
             (256, 128, fv.GRID_CENTRED, "map")]
    frames, refs = [], []
    g = wl.rng(61)
    for i, (W, H, grid, kind) in enumerate(specs):
        img = wl.grating_frame(H, W, 3, seed=70 + i)
        fx, fy = float(g.uniform(0, W)), float(g.uniform(0, H))
        org = (oracle.centred_origin(np.float32(fx), B), oracle.centred_origin(np.float32(fy), B)) \
            if grid == fv.GRID_CENTRED else (0, 0)
        x = to_dev(img)
        if kind == "map":
            nby, nbx = (H + org[1] + B - 1) // B, (W + org[0] + B - 1) // B
            smap = g.uniform(0.3, 6.0, size=(nby, nbx)).astype(np.float32)
            m = to_dev(smap)
            frames.append(fv.BatchFrame(x, torch.empty_like(x), fx, fy, 0.0, 0.0, grid, m, float(smap.max())))
            refs.append(oracle.forward_u8(img, B, fx, fy, 0.0, 0.0, "hwc", origin=org,
                                          sigma_map=smap.astype(np.float64)))
        else:
            frames.append(fv.BatchFrame(x, torch.empty_like(x), fx, fy, 0.5, 0.04, grid))
            refs.append(oracle.forward_u8(img, B, fx, fy, 0.5, 0.04, "hwc", origin=org))
    fv.foveate_batch(frames)
    torch.cuda.synchronize()
    for fr, ref in zip(frames, refs):
        assert_u8_close(fr.out.cpu().numpy(), ref, min_equal=0.99)


# ---------------------------------------------------------------- blocks larger than 32 (32 x 32 tiles sharing sigma)

@pytest.mark.parametrize("tc", [0, 1, 2, 3])
@pytest.mark.parametrize("grid", [0, 1])
def test_block_64_u8_matches_oracle(fv, tc, grid):
    W, H, C, B = 500, 300, 3, 64
    img = wl.grating_frame(H, W, C, seed=81)
    fx, fy = 210.7, 140.2
    ctx = fv.Context(W, H, C, B, 0.5, 0.02, fv.U8_HWC, grid=grid)
    ctx.set_config(256, 0, 16 if tc == 3 else 32, tensor_cores=tc)
    x = to_dev(img)
    y = torch.empty_like(x)
    ctx.render(x, y, fx, fy)
    sig, rad = ctx.sigma_table(fx, fy)
    torch.cuda.synchronize()
    org = (oracle.centred_origin(np.float32(fx), B), oracle.centred_origin(np.float32(fy), B)) if grid else (0, 0)
    osig, orad = oracle.sigma_table(W, H, B, np.float32(fx), np.float32(fy), 0.5, 0.02, origin=org)
    assert np.array_equal(rad.cpu().numpy(), orad)
    ref = oracle.forward_u8(img, B, fx, fy, 0.5, 0.02, "hwc", origin=org)
    assert_u8_close(y.cpu().numpy(), ref, min_equal=0.99)


def test_block_64_f32_forward_and_backward(fv):
    W, H, C, B = 150, 100, 2, 64
    img = wl.uniform_f32((C, H, W), seed=82)
    gout = wl.uniform_f32((C, H, W), seed=83)
    ctx = fv.Context(W, H, C, B, 0.4, 0.05, fv.F32_CHW)
    y = torch.empty(C, H, W, device="cuda")
    gin = torch.empty(C, H, W, device="cuda")
    ctx.render(to_dev(img), y, 60.0, 20.0)
    ctx.backward(to_dev(gout), gin, 60.0, 20.0)
    torch.cuda.synchronize()
    assert_f32_close(y.cpu().numpy(), oracle.forward(img, B, 60.0, 20.0, 0.4, 0.05, "chw"))
    np.testing.assert_allclose(gin.cpu().numpy(), oracle.adjoint(gout, B, 60.0, 20.0, 0.4, 0.05, "chw"),
                               rtol=1e-5, atol=1e-5)
