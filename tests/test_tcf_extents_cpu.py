"""CPU check of the float32 tensor-core kernel's per-item geometry
(csrc/tcf_forward.cu) against its TMA and shared-memory constraints.

For random items (widths a multiple of 4, as the float32 tensor maps need;
heights from 1 row; 1 to 4 planes; radii up to the library's bound of 1023;
shifted block grids; block sides 4 to 64) the geometry is worked out as
item_geometry does (csrc/fwd_common.cuh, 16-row chunks, full slabs of the
kernel's slab width), with the host's rule for planes per pass (all C = 2..4
planes together when the launch's radius bound is at most 128, else one).
For every slab pass and chunk the kernel would issue:

* each 3D box starts at an x coordinate that is a multiple of 4 floats (the
  16-byte rule of tiled TMA copies; a misaligned x is an illegal instruction);
* a plane's boxes (ceil((ph + slab width) / 32)) fit the plane's warps, so
  box p * wpp + b stays inside the stage of 8 boxes;
* the slab's V row, rounded up to whole k-steps, fits the V pitch, and every
  V write and zero-fill lies inside the V array of 32 x CP rows.
The kernel's constants are restated and checked against its source.
"""
import os
import random
import re

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2012_08655_gb300", "csrc")


def tc_vp(C, NW):
    """V pitch (halves) of tc_common.cuh's tc_vp."""
    w = ((32 * NW - 16) // C + 15) // 16 * 16
    return w if (w // 8) % 2 else w + 8


def slab_cols(cp):
    """TcfDims<CP>::SLAB."""
    wpp = 8 // cp
    return min(32 * wpp - 3, tc_vp(cp, 8) // 16 * 16)


def test_constants_match_the_source():
    k = open(os.path.join(CSRC, "tcf_forward.cu")).read()
    assert re.search(r"constexpr int kNWF = 8;", k)
    assert re.search(r"constexpr int kRBF = 16;", k)
    assert re.search(r"constexpr int kTcfPackedRadius = 128;", k)
    assert "static constexpr int SLAB = tcf_min(32 * WPP - 3, VP / 16 * 16);" in k
    c = open(os.path.join(CSRC, "tc_common.cuh")).read()
    assert "((((32 * NW - 16) / C + 15) / 16 * 16) / 8) % 2" in c
    assert [tc_vp(cp, 8) for cp in (1, 2, 3, 4)] == [248, 136, 88, 72]
    assert [slab_cols(cp) for cp in (1, 2, 3, 4)] == [240, 125, 61, 61]


def test_boxes_and_v_stay_inside_their_limits():
    rng = random.Random(11)
    worst = {"boxes": 0, "vcols": 0}
    for _ in range(30000):
        W = 4 * rng.choice([1, 2, 8, 9, 16, 56, 75, 480, 960, rng.randint(1, 1000)])
        H = rng.choice([1, 2, 16, 33, 224, 1080, rng.randint(1, 2000)])
        C = rng.randint(1, 4)
        B = rng.choice([4, 8, 16, 32, 64])
        T = min(B, 32)
        rbound = rng.choice([64, 128, 192, 512, 1024])
        r = rng.randint(0, min(rbound, 1023))
        cp = C if 2 <= C <= 4 and rbound <= 128 else 1
        wpp, vp = 8 // cp, tc_vp(cp, 8)
        ox = rng.randint(0, T - 1) if rng.random() < 0.3 else 0
        oy = rng.randint(0, T - 1) if rng.random() < 0.3 else 0
        nbx, nby = (W + ox + T - 1) // T, (H + oy + T - 1) // T
        xs, ys = rng.randrange(nbx) * T - ox, rng.randrange(nby) * T - oy
        x0, y0 = max(0, xs), max(0, ys)
        bw, bh = min(xs + T, W) - x0, min(ys + T, H) - y0
        if bw <= 0 or bh <= 0:
            continue
        # item_geometry (float32: elements are pixels; full slabs)
        gx0 = max(0, x0 - r)
        EW = min(W - 1, x0 + bw - 1 + r) - gx0 + 1
        gy0 = max(0, y0 - r)
        EH = min(H - 1, y0 + bh - 1 + r) - gy0 + 1
        offy = gy0 - (y0 - r)
        ph_y = offy & 15
        vrows = (EH + ph_y + 15) & ~15
        cap = slab_cols(cp)
        nsl = (EW + cap - 1) // cap
        sw = cap if nsl > 1 else EW
        nchunks = (vrows + 15) // 16
        assert vrows % 16 == 0 and nchunks * 16 == vrows
        for s in range(nsl):
            e0 = s * sw
            sws = min(sw, EW - e0)
            assert sws >= 1
            ph = (gx0 + e0) & 3  # base 16-byte aligned and W a multiple of 4
            x = gx0 + e0 - ph
            assert x % 4 == 0 and x >= 0, (W, gx0, e0)
            nbox = (ph + sws + 31) >> 5
            assert nbox <= wpp, (cp, ph, sws)
            for p in range(cp):
                for bx in range(nbox):
                    assert 0 <= p * wpp + bx < 8
                    assert (x + 32 * bx) % 4 == 0
            npx16 = (sws + 15) & ~15
            assert npx16 <= vp, (cp, sws, vp)
            # V writes: rows 32 p + 0..31, columns e in [0, sws); zero-fill
            # columns [sws, npx16); the array holds 32 CP rows of vp halves
            last = (32 * (cp - 1) + 31) * vp + npx16 - 1
            assert last < 32 * cp * vp
            worst["boxes"] = max(worst["boxes"], nbox)
            worst["vcols"] = max(worst["vcols"], npx16)
    # the sampled items reach the limits the kernel is sized for
    assert worst["boxes"] == 8 and worst["vcols"] == 240
