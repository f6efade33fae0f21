"""CPU check of the two-pass tcgen05 kernel's operand reads against its
shared-memory buffers (csrc/tc05_forward.cu, csrc/tc05_common.cuh).

For random items (frame sizes from 1 pixel to 4K, radii up to the kernel's
bound, shifted block grids, partial blocks) the item geometry is worked out
as item_geometry does (csrc/fwd_common.cuh), and every MMA's B descriptor is
followed to the tap-strip entries it reads: pass 1 (entry D0/8 + 4 + 2 kidx
plus the K and N core offsets) and pass 2 (entry (offx + P0 + p0 - 31 -
delta2)/8 + kXOff plus the same offsets). All of them must lie inside the
strip of strip_entries(rmax) entries, and each slab's staged bytes inside one
staged row. The kernel's constants are read from its source.
"""
import os
import random
import re

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2012_08655_gb300", "csrc")


def _const(text, name):
    m = re.search(rf"constexpr int {name} = ([^;]+);", text)
    assert m, name
    return m.group(1)


def _constants():
    k = open(os.path.join(CSRC, "tc05_forward.cu")).read()
    c = open(os.path.join(CSRC, "tc05_common.cuh")).read()
    tiles = int(_const(k, "kTiles"))
    pxt = int(_const(k, "kPxT"))
    boxes = int(_const(k, "kBoxes5"))
    rmax_bound = int(_const(k, "kMaxRadius5"))
    rb = int(_const(k, "kRB5"))
    xoff = int(_const(c, "kXOff"))
    m = re.search(r"int strip_entries\(int rmax\) \{ return rmax / (\d+) \+ (\d+); \}", c)
    assert m
    div, add = int(m.group(1)), int(m.group(2))
    return tiles, pxt, boxes, rmax_bound, rb, xoff, (lambda r: r // div + add)


def test_strip_and_staged_reads_stay_inside_their_buffers():
    tiles, pxt, boxes, rmax_bound, rb, xoff, strip_entries = _constants()
    slab_cap = tiles * pxt * 3
    row_bytes = boxes * 128
    rng = random.Random(7)
    worst = {"p1": -10 ** 9, "p2": -10 ** 9, "lo": 10 ** 9}
    for _ in range(40000):
        W = rng.choice([1, 2, 31, 65, 256, 300, 1920, 3840, rng.randint(1, 4000)])
        H = rng.choice([1, 2, 33, 256, 1080, 2160, rng.randint(1, 3000)])
        rmax = rng.choice([r for r in (64, 128, 192, 256) if r <= rmax_bound] + [rmax_bound])
        r = rng.randint(0, rmax)
        T = 32
        ox = rng.randint(0, T - 1) if rng.random() < 0.3 else 0
        oy = rng.randint(0, T - 1) if rng.random() < 0.3 else 0
        nbx, nby = (W + ox + T - 1) // T, (H + oy + T - 1) // T
        xs, ys = rng.randrange(nbx) * T - ox, rng.randrange(nby) * T - oy
        x0, y0 = max(0, xs), max(0, ys)
        bw, bh = min(xs + T, W) - x0, min(ys + T, H) - y0
        if bw <= 0 or bh <= 0:
            continue
        gx0 = max(0, x0 - r)
        EW = min(W - 1, x0 + bw - 1 + r) - gx0 + 1
        offx = gx0 - (x0 - r)
        gy0 = max(0, y0 - r)
        EH = min(H - 1, y0 + bh - 1 + r) - gy0 + 1
        offy = gy0 - (y0 - r)
        ph = offy & 15
        vrows = (EH + ph + 15) & ~15
        nent = strip_entries(rmax)
        # pass 1
        D0 = offy - ph
        assert D0 % 16 == 0 and D0 >= 0
        k_end = min(vrows, 32 - D0 + 2 * r)
        for k0 in range(0, k_end, rb):
            first = D0 // 8 + 4 + 2 * (k0 // 16)
            last = first + 1 + 3          # K groups +0, +1; N core pairs +0 .. +3
            worst["p1"] = max(worst["p1"], last - (nent - 1))
            worst["lo"] = min(worst["lo"], first)
            assert 0 <= first and last <= nent - 1, (W, H, r, rmax, k0)
        # pass 2, slab by slab
        E = EW * 3
        nsl = (E + slab_cap - 1) // slab_cap
        sw = slab_cap if nsl > 1 else E
        delta2 = (offx + 1) & 7
        for s in range(nsl):
            e0 = s * sw
            sws = min(sw, E - e0)
            npx, P0 = sws // 3, e0 // 3
            num = offx + P0 - 31 - delta2
            assert num % 8 == 0
            base = num // 8 + xoff
            assert (npx + pxt - 1) // pxt <= tiles
            for p0 in range(0, npx, 16):
                first = base + 2 * (p0 // 16)
                last = first + 1 + 3
                worst["p2"] = max(worst["p2"], last - (nent - 1))
                worst["lo"] = min(worst["lo"], first)
                assert 0 <= first and last <= nent - 1, (W, H, r, rmax, s, p0)
            # a slab's bytes, after up to 15 bytes of alignment padding, fit one staged row
            assert 15 + sws <= row_bytes
    assert worst["p1"] < 0 and worst["p2"] < 0 and worst["lo"] >= 0
