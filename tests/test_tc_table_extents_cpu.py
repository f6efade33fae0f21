"""Extents of the tap-pair table reads of the mma.sync kernels, checked on the
CPU over radii up to the library's bound.

The kernels read each fragment's pair of consecutive taps (u(i), u(i + 1))
from shared-memory tables without a bounds check: table p (the parity of i)
holds, at entry j, the pair starting at tap 2j + p - 32, for j in
[0, npair), npair = rmax + 56 (csrc/tc_common.cuh: make_pairs, kPairPad = 32).
Every read below must (a) use the table of i's parity, (b) land on the
entry of i, and (c) stay inside [0, npair), for every lane (g, t), every
k-step a pass issues and every geometry an item can have. The index formulas
are restated from the kernels:

* forward pass 1 (csrc/tcf_forward.cu, as csrc/tc_forward.cu): lane (g, t)
  of the k-step at staged row k0 reads entries j0 + {-12, -8, -4, 0, 4},
  j0 = (k0 + D0 + 2t - g + 32) >> 1, table g mod 2, D0 = offy - (offy mod 16),
  in every k-step where the band meets one of the two m-tiles;
* forward pass 2 (tc_pass2_slab and tcf_pass2's form): entries jb and jb + 4,
  jb = (offx + P0 + kk + 2t - 8 nt - g + 32) >> 1, table (offx + P0 + g) mod 2,
  every k-step kk of the slab;
* adjoint pass A (csrc/tca_adjoint.cu): entries jb and jb + 4,
  jb = (Dx + 16 ks - n0 + 2t - g + 32) >> 1, table (Dx + g) mod 2,
  Dx = 2r - offx, where the band meets the k-step;
* adjoint pass B: entries j0 + {-4, 0, 4}, j0 = (Dy + 16 ks - m0 + 2t - g + 32) >> 1,
  table (Dy + g) mod 2, Dy = 2r - offy, where the band meets the k-step.
"""
import numpy as np

PAD = 32
R_BOUND = 1023
RADII = sorted(set(range(0, 40)) | set(range(40, R_BOUND + 1, 71)) | {R_BOUND})
LANE_G, LANE_T = np.meshgrid(np.arange(8), np.arange(4), indexing="ij")
G, T = LANE_G.ravel(), LANE_T.ravel()


def npair(rmax):
    return rmax + 56


def offsets(r):
    """Fold offsets an item can have (0 when the halo is inside the frame,
    r - x0 when it is clipped): all small ones and the largest ones."""
    return sorted({o for o in list(range(0, min(r, 20) + 1)) + list(range(max(0, r - 20), r + 1))})


def check_reads(tap, table, entry, r, what):
    """tap: the fragment's first tap index; table: parity table used; entry:
    table entry read for it (all arrays of one shape)."""
    assert np.all(table == (tap & 1)), f"{what}: wrong parity table at r={r}"
    assert np.all(2 * entry + table - PAD == tap), f"{what}: entry does not hold tap i at r={r}"
    assert np.all((entry >= 0) & (entry < npair(r))), \
        f"{what}: entry outside [0, {npair(r)}) at r={r}: {entry.min()}..{entry.max()}"


def test_forward_pass1_reads_stay_in_the_tables():
    for r in RADII:
        for offy in offsets(r):
            ph = offy & 15
            D0 = offy - ph
            EH = 32 + 2 * r - offy  # largest folded halo for this offset (offy rows clipped above)
            vrows = (EH + ph + 15) & ~15
            for k0 in range(0, vrows, 16):
                on0 = k0 + 15 >= -D0 and k0 <= 15 - D0 + 2 * r
                on1 = k0 + 15 >= 16 - D0 and k0 <= 31 - D0 + 2 * r
                if not (on0 or on1):
                    continue
                i0 = k0 + D0 + 2 * T - G  # tap of a[0] of m-tile 0 (row g, column 2t)
                j0 = (i0 + PAD) >> 1
                table = G & 1
                for d in (-12, -8, -4, 0, 4):  # both m-tiles' four registers
                    check_reads(i0 + 2 * d, table, j0 + d, r, "forward pass 1")


def test_forward_pass2_reads_stay_in_the_tables():
    for r in RADII:
        for offx in offsets(r):
            EW = 32 + 2 * r - offx  # largest folded halo for this offset
            for slab in (240, 125, 61):  # one plane per pass; two; three or four (packed)
                for P0 in range(0, EW, slab):
                    npx = min(slab, EW - P0)
                    npx16 = (npx + 15) & ~15
                    table = (offx + P0 + G) & 1
                    for nt in range(4):
                        for kk in range(0, npx16, 16):
                            i = offx + P0 + kk + 2 * T - 8 * nt - G
                            jb = (i + PAD) >> 1
                            check_reads(i, table, jb, r, "forward pass 2")
                            check_reads(i + 8, table, jb + 4, r, "forward pass 2")


def test_adjoint_pass_a_reads_stay_in_the_tables():
    for r in RADII:
        for offx in offsets(r):
            Dx = 2 * r - offx
            EW = 32 + 2 * r - offx
            table = (Dx + G) & 1
            for n0 in range(0, EW + 8, 8):
                for ks in (0, 1):
                    i0 = Dx + 16 * ks - n0
                    if i0 + 15 < 0 or i0 - 7 > 2 * r:
                        continue
                    i = i0 + 2 * T - G
                    jb = (i + PAD) >> 1
                    check_reads(i, table, jb, r, "adjoint pass A")
                    check_reads(i + 8, table, jb + 4, r, "adjoint pass A")


def test_adjoint_pass_b_reads_stay_in_the_tables():
    for r in RADII:
        for offy in offsets(r):
            Dy = 2 * r - offy
            EH = 32 + 2 * r - offy
            table = (Dy + G) & 1
            for m0 in range(0, EH + 16, 16):
                for ks in (0, 1):
                    i0 = Dy + 16 * ks - m0
                    if i0 + 15 < 0 or i0 - 15 > 2 * r:
                        continue
                    i = i0 + 2 * T - G
                    j0 = (i + PAD) >> 1
                    for d in (-4, 0, 4):  # rows + 8 (-4), columns + 8 (+4)
                        check_reads(i + 2 * d, table, j0 + d, r, "adjoint pass B")


def test_the_check_catches_a_parity_slip():
    """The check is live: reading the forward pass-2 table of the wrong
    parity (g instead of offx + P0 + g) is caught."""
    r, offx, P0 = 5, 3, 0
    i = offx + P0 + 2 * T - G
    try:
        check_reads(i, G & 1, (i + PAD) >> 1, r, "slip")
    except AssertionError:
        return
    raise AssertionError("a wrong parity table went unnoticed")


def test_the_check_catches_a_short_table(monkeypatch):
    """The check is live on extents too: the forward passes read up to entry
    r + 38 (and down to entry 0), so a table of r + 37 entries fails."""
    import sys
    mod = sys.modules[__name__]
    monkeypatch.setattr(mod, "npair", lambda rmax: rmax + 37)
    try:
        test_forward_pass1_reads_stay_in_the_tables()
    except AssertionError:
        return
    raise AssertionError("a table too short for the reads went unnoticed")
