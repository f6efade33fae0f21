"""Host model of the float32 tensor-core kernel's ring protocol
(csrc/tcf_forward.cu), run under random schedules on the CPU.

Eight warps consume 16-row chunks from a four-stage ring. Thread 0 (in warp
0) issues a chunk into stage c mod 4 once that stage's empty barrier has
seen all eight warps release chunk c - 4; the chunk's bytes land on the
stage's full barrier after a random delay. Every warp waits for each chunk's
full barrier, reads it, and arrives once on its empty barrier; block-wide
barriers sit at slab ends (two) and at item boundaries. The model fails on a
parity wait whose barrier has run two phases ahead, a wait that passes on
an older phase, an arrival counted into another chunk's phase, a stage
overwritten while a warp still reads it, or no role able to move.
"""
import random

import pytest

from test_tc05_protocol_cpu import Bar

WARPS, STAGES = 8, 4


def simulate(items, seed, idle_warps_wait=True):
    rng = random.Random(seed)
    full = [Bar(f"full{s}", 1) for s in range(STAGES)]
    empty = [Bar(f"empty{s}", WARPS) for s in range(STAGES)]
    landed = {}            # chunk -> True once its bytes are in the stage
    readers = {}           # stage -> set of warps reading its current chunk
    stage_chunk = {}       # stage -> chunk it holds (or is receiving)
    events, clock = [], [0]

    class Barrier:         # __syncthreads: generation counter
        def __init__(self):
            self.count, self.gen = 0, 0

    bar = Barrier()

    def sync():
        g = bar.gen
        bar.count += 1
        if bar.count == WARPS:
            bar.count, bar.gen = 0, bar.gen + 1
        while bar.gen == g:
            yield

    def issue(c):
        s = c % STAGES
        if c >= STAGES:
            while not empty[s].test((c - STAGES) // STAGES):
                yield
        if readers.get(s):
            raise RuntimeError(f"chunk {c} overwrites stage {s} while warps {sorted(readers[s])} read it")
        stage_chunk[s] = c
        ph = full[s].next_phase()
        full[s].arrive(ph, tx=1)
        landed[c] = False

        def land(s=s, ph=ph, c=c):
            landed[c] = True
            full[s].land_tx(ph, 1)
        events.append((clock[0] + rng.randint(1, 50), land))

    def warp(w):
        gq0 = 0
        for it in items:
            Q, nch, active = it["Q"], it["nch"], it["active"]
            if w == 0:
                for q in range(min(STAGES - 1, Q)):
                    yield from issue(gq0 + q)
            yield from sync()                       # tables ready
            for q in range(Q):
                c = gq0 + q
                s = c % STAGES
                if w == 0 and q + STAGES - 1 < Q:
                    yield from issue(c + STAGES - 1)
                act = w in active[q // nch]
                if act or idle_warps_wait:
                    while not full[s].test(c // STAGES):
                        yield
                if act:
                    if stage_chunk.get(s) != c or not landed.get(c):
                        raise RuntimeError(f"warp {w} reads chunk {c} from stage {s} before it landed")
                    readers.setdefault(s, set()).add(w)
                    for _ in range(rng.randint(0, 3)):
                        yield                       # pass 1 on the chunk
                    readers[s].discard(w)
                empty[s].arrive(c // STAGES)
                yield
                if q % nch == nch - 1:
                    yield from sync()               # previous slab's V free
                    yield                           # V written
                    yield from sync()               # V complete
                    yield                           # pass 2
            gq0 += Q
            yield from sync()                       # item end (fault vote)
            yield from sync()                       # value-range vote
            yield from sync()                       # next item's start

    roles = [warp(w) for w in range(WARPS)]
    live = list(roles)
    while live:
        events.sort(key=lambda e: e[0])
        while events and events[0][0] <= clock[0]:
            events.pop(0)[1]()
        role = rng.choice(live)
        try:
            next(role)
        except StopIteration:
            live.remove(role)
        clock[0] += 1
        if clock[0] > 400_000:
            raise RuntimeError("no role can move")


def random_items(rng):
    items = []
    for _ in range(rng.randint(0, 6)):
        C = rng.randint(1, 3)
        nsl = rng.choice([1, 1, 2, 3])
        nch = rng.randint(1, 9)
        # warps holding slab elements per slab pass: any set that contains
        # warp 0 (one plane per pass: a prefix; planes side by side: the
        # first warps of each plane)
        active = []
        for _c in range(C):
            for _s in range(nsl):
                active.append({0} | {w for w in range(1, WARPS) if rng.random() < 0.6})
        items.append({"Q": C * nsl * nch, "nch": nch, "active": active})
    return items


@pytest.mark.parametrize("seed_base", [0, 1000, 2000])
def test_ring_protocol_never_hangs_or_aliases(seed_base):
    for seed in range(seed_base, seed_base + 40):
        simulate(random_items(random.Random(seed)), seed)


def test_model_catches_idle_warps_skipping_the_wait():
    """The model's check is live: warps without slab elements that arrive on
    the empty barrier without waiting for the chunk run ahead and count
    their arrivals into an earlier chunk's phase."""
    failures = 0
    for seed in range(60):
        try:
            simulate(random_items(random.Random(seed)), seed, idle_warps_wait=False)
        except RuntimeError:
            failures += 1
    assert failures > 10
