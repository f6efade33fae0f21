"""Shared helpers of the GPU parity tests (block sampling, comparisons)."""
import numpy as np


def sample_blocks(width, height, block, fix_x, fix_y, n_random=64, seed=0, all_edges=False):
    """Row-major block indices to check against the oracle at large sizes:
    the fixation block, the four corners, the partial edge blocks, and
    ``n_random`` random blocks (with ``all_edges`` every border block)."""
    nbx, nby = (width + block - 1) // block, (height + block - 1) // block
    sel = {0, nbx - 1, (nby - 1) * nbx, nby * nbx - 1}
    fbx = min(max(int(fix_x // block), 0), nbx - 1)
    fby = min(max(int(fix_y // block), 0), nby - 1)
    sel.add(fby * nbx + fbx)
    if width % block:
        sel.update(by * nbx + nbx - 1 for by in range(nby))
    if height % block:
        sel.update((nby - 1) * nbx + bx for bx in range(nbx))
    if all_edges:
        sel.update(bx for bx in range(nbx))
        sel.update((nby - 1) * nbx + bx for bx in range(nbx))
        sel.update(by * nbx for by in range(nby))
        sel.update(by * nbx + nbx - 1 for by in range(nby))
    g = np.random.Generator(np.random.PCG64(seed))
    k = min(n_random, nbx * nby)
    sel.update(int(b) for b in g.choice(nbx * nby, size=k, replace=False))
    return sorted(sel)


def block_mask(width, height, block, blocks, layout, channels):
    """Boolean mask of the pixels of `blocks` in an image of the given layout."""
    nbx = (width + block - 1) // block
    m = np.zeros((height, width), bool)
    for b in blocks:
        by, bx = divmod(b, nbx)
        m[by * block:(by + 1) * block, bx * block:(bx + 1) * block] = True
    if channels is None:
        return m
    if layout == "hwc":
        return np.repeat(m[:, :, None], channels, axis=2)
    return np.repeat(m[None], channels, axis=0)


def assert_u8_close(got, ref, mask=None, max_lsb=1, min_equal=0.99):
    got = np.asarray(got).astype(np.int32)
    ref = np.asarray(ref).astype(np.int32)
    if mask is not None:
        got, ref = got[mask], ref[mask]
    d = np.abs(got - ref)
    assert d.size > 0
    assert d.max() <= max_lsb, f"uint8 max difference {d.max()} LSB > {max_lsb}"
    eq = float(np.mean(d == 0))
    assert eq >= min_equal, f"only {eq:.4f} of uint8 outputs equal the oracle"


def assert_f32_close(got, ref, mask=None, atol=1e-5):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if mask is not None:
        got, ref = got[mask], ref[mask]
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    worst = float(err.max())
    assert worst <= atol, f"float32 max abs error {worst:.3e} > {atol:.0e}"
