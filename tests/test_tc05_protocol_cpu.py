"""Host model of the two-pass tcgen05 kernel's mbarrier protocol
(csrc/tc05_forward.cu), run under random schedules on the CPU.

Every role of the kernel is a generator that performs, in the kernel's
order, the same waits (phase-parity tests), arrivals and commits on the same
barriers with the same phase arithmetic:

* control: TMA producer (ring stages, released by the five tile warps) and
  pass-2 issuer (A2 buffers, D2 slots, item slots);
* five tile warps: ring wait, A1-buffer wait, release of the stage, wait for
  the read-back of the tile's previous slab, MMA commit per chunk, slab commit
  plus arrive;
* four read-back warps: slab commits of every tile, D1 release, A2 hand-off,
  per-item arrival for the output;
* the table warps: items published kSlots - 1 ahead, output of each item
  after its V columns and D2 are done, D2 release.

Asynchronous completions (TMA bytes, tcgen05.commit) land after random
delays, in issue order per issuing thread. The model fails on what would
hang or corrupt the kernel: a parity wait whose barrier has already run two
phases ahead (it would never see its phase), a wait that passes on an older
phase, an arrival counted into the wrong phase, or no role able to move.
"""
import random

import pytest

TILES, SLOTS = 5, 3


class Bar:
    def __init__(self, name, count):
        self.name, self.count = name, count
        self.done = 0          # completed phases
        self.pending = count   # arrivals still expected in the current phase
        self.tx = 0            # transaction bytes still expected
        self.issued = 0        # arrivals handed out so far (fixes each arrival's phase)

    def next_phase(self):
        k = self.issued
        self.issued += 1
        return k // self.count

    def arrive(self, phase, tx=0):
        if phase != self.done:
            raise RuntimeError(f"{self.name}: arrival meant for phase {phase} lands in phase {self.done}")
        self.pending -= 1
        self.tx += tx
        self._complete()

    def land_tx(self, phase, tx):
        if phase != self.done:
            raise RuntimeError(f"{self.name}: bytes meant for phase {phase} land in phase {self.done}")
        self.tx -= tx
        self._complete()

    def _complete(self):
        if self.pending == 0 and self.tx == 0:
            self.done += 1
            self.pending = self.count

    def test(self, phase):
        """mbarrier.test_wait.parity for the given phase."""
        if self.done > phase + 1:
            raise RuntimeError(f"{self.name}: waits for phase {phase}, {self.done} already done: never seen")
        passed = (self.done & 1) != (phase & 1)
        if passed and self.done != phase + 1:
            raise RuntimeError(f"{self.name}: wait for phase {phase} passes at {self.done}")
        return passed


def simulate(items, seed, stages, nbuf, idle_tile_waits_readback=True):
    rng = random.Random(seed)
    bars = {}

    def bar(name, count):
        bars[name] = Bar(name, count)

    for i in range(stages):
        bar(f"ring{i}", 1)
        bar(f"ringfree{i}", TILES)
    for t in range(TILES):
        for b in range(nbuf):
            bar(f"a1free{t}.{b}", 1)
        bar(f"tdone{t}", 2)
        bar(f"d1free{t}", 4)
    for i in range(2):
        bar(f"a2full{i}", 4)
        bar(f"a2free{i}", 1)
        bar(f"d2full{i}", 1)
        bar(f"d2free{i}", 4)
    for i in range(SLOTS):
        bar(f"itemfull{i}", 1)
        bar(f"vready{i}", 4)
    slots = [None] * SLOTS
    events, clock, last_commit = [], [0], {}

    def later(fn):
        events.append((clock[0] + rng.randint(1, 40), fn))

    def commit(thread, name):
        phase = bars[name].next_phase()
        t = max(last_commit.get(thread, 0), clock[0]) + rng.randint(1, 60)
        last_commit[thread] = t
        events.append((t, lambda: bars[name].arrive(phase)))

    def arrive(name):
        bars[name].arrive(bars[name].next_phase())

    def control():
        pj = gq = issued = 0
        p_item = None
        p_end = False
        ij = gtl = done = 0
        i_item = None
        i_end = i_d2ok = False
        while not (p_end and i_end):
            if not p_end:
                if p_item is None and bars[f"itemfull{pj % SLOTS}"].test(pj // SLOTS):
                    if slots[pj % SLOTS] is None:
                        p_end = True
                    else:
                        p_item, issued = slots[pj % SLOTS], 0
                if p_item is not None and (gq < stages or bars[f"ringfree{gq % stages}"].test(gq // stages - 1)):
                    stg = gq % stages
                    ph = bars[f"ring{stg}"].next_phase()
                    bars[f"ring{stg}"].arrive(ph, tx=1)
                    later(lambda stg=stg, ph=ph: bars[f"ring{stg}"].land_tx(ph, 1))
                    gq += 1
                    issued += 1
                    if issued == p_item["nsl"] * p_item["nch"]:
                        p_item, pj = None, pj + 1
            if not i_end:
                if i_item is None and bars[f"itemfull{ij % SLOTS}"].test(ij // SLOTS):
                    if slots[ij % SLOTS] is None:
                        i_end = True
                    else:
                        i_item, done, i_d2ok = slots[ij % SLOTS], 0, ij < 2
                if i_item is not None and not i_d2ok and bars[f"d2free{ij & 1}"].test((ij >> 1) - 1):
                    i_d2ok = True
                if i_item is not None and i_d2ok and bars[f"a2full{gtl & 1}"].test(gtl >> 1):
                    commit("control", f"a2free{gtl & 1}")
                    gtl += 1
                    done += 1
                    if done == sum(i_item["tiles"]):
                        commit("control", f"d2full{ij & 1}")
                        i_item, ij = None, ij + 1
            yield

    def tile(t):
        g = gs = j = 0
        while True:
            while not bars[f"itemfull{j % SLOTS}"].test(j // SLOTS):
                yield
            it = slots[j % SLOTS]
            if it is None:
                return
            for s in range(it["nsl"]):
                active = t < it["tiles"][s]
                for kq in range(it["nch"]):
                    while not bars[f"ring{g % stages}"].test(g // stages):
                        yield
                    if g >= nbuf:
                        while not bars[f"a1free{t}.{g % nbuf}"].test(g // nbuf - 1):
                            yield
                    yield  # conversion
                    arrive(f"ringfree{g % stages}")
                    if kq == 0 and gs > 0 and (active or idle_tile_waits_readback):
                        while not bars[f"d1free{t}"].test(gs - 1):
                            yield
                    commit(f"tile{t}", f"a1free{t}.{g % nbuf}")
                    g += 1
                commit(f"tile{t}", f"tdone{t}")
                arrive(f"tdone{t}")
                gs += 1
                yield
            j += 1

    def readback(q):
        gs = gtl = j = 0
        while True:
            while not bars[f"itemfull{j % SLOTS}"].test(j // SLOTS):
                yield
            it = slots[j % SLOTS]
            if it is None:
                return
            for s in range(it["nsl"]):
                for t in range(TILES):
                    while not bars[f"tdone{t}"].test(gs):
                        yield
                    if t >= it["tiles"][s]:
                        arrive(f"d1free{t}")
                        continue
                    if gtl >= 2:
                        while not bars[f"a2free{gtl & 1}"].test((gtl >> 1) - 1):
                            yield
                    yield  # TMEM read
                    arrive(f"d1free{t}")
                    yield  # V to A2
                    arrive(f"a2full{gtl & 1}")
                    gtl += 1
                gs += 1
            arrive(f"vready{j % SLOTS}")
            j += 1

    def tables():
        def publish(j):
            slots[j % SLOTS] = items[j] if j < len(items) else None
            arrive(f"itemfull{j % SLOTS}")
            return j < len(items)

        pub, ended = 0, False
        while pub < SLOTS - 1 and not ended:
            ended = not publish(pub)
            pub += 1
            yield
        j = 0
        while not ended or j < pub - 1:
            if not ended:
                ended = not publish(pub)
                pub += 1
            yield
            while not bars[f"vready{j % SLOTS}"].test(j // SLOTS):
                yield
            while not bars[f"d2full{j & 1}"].test(j >> 1):
                yield
            for _ in range(4):
                arrive(f"d2free{j & 1}")
            yield
            j += 1

    roles = [control()] + [tile(t) for t in range(TILES)] + [readback(q) for q in range(4)] + [tables()]
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
    while events:
        events.sort(key=lambda e: e[0])
        events.pop(0)[1]()


def random_items(rng):
    items = []
    for _ in range(rng.randint(0, 7)):
        nsl = rng.choice([1, 1, 1, 2, 3])
        tiles = [TILES] * (nsl - 1) + [rng.randint(1, TILES)]
        items.append({"nsl": nsl, "tiles": tiles, "nch": rng.randint(1, 9)})
    return items


@pytest.mark.parametrize("stages,nbuf", [(6, 3), (5, 3), (5, 2), (4, 2)])
def test_protocol_never_hangs_or_aliases(stages, nbuf):
    for seed in range(60):
        simulate(random_items(random.Random(seed)), seed, stages, nbuf)


def test_model_catches_an_idle_tile_running_ahead():
    """The model's check is live: with an empty tile's warp not waiting for
    the read-back of its previous slab (the fault the kernel once had), its
    slab commits run ahead of the read-back warps' parity waits."""
    failures = 0
    for seed in range(60):
        try:
            simulate(random_items(random.Random(seed)), seed, 6, 3, idle_tile_waits_readback=False)
        except RuntimeError:
            failures += 1
    assert failures > 10
