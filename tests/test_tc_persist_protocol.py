"""The persistent tensor-core kernels' barrier protocol, replayed on the CPU.

k_expand_tcp (csrc/k_tc_persist.cuh) runs four roles in each CTA that pass
stage slots, the Z block buffer and two tensor-memory accumulators to each
other through mbarriers:

* producer (one thread): per chunk, waits for the slot's previous use to be
  released (empty barrier), then arms the slot's full barrier with the bytes
  of the A tiles and requests them; a chunk of X that tensor copies can bring
  comes with them (and the producer gives the full barrier's second arrival),
  any other chunk is handed to the stagers by an arrival on the slot's
  "B is yours" barrier;
* MMA issuer (one thread): per item, waits for the accumulator set to be
  drained (acce), per chunk for the slot to be full, issues the MMAs and
  commits them to the slot's empty barrier, then the item to accf;
* stagers (64 threads behind one named barrier, one role here): for every
  chunk they fill, wait on the slot's "B is yours" barrier with a phase they
  count themselves, write B (X rows, or Z rows converted from the Z block in
  shared memory, which a bulk copy on its own barrier brings a whole item
  ahead), then give the full barrier's second arrival;
* epilogue: per item, waits for accf, reads the accumulators, arrives on acce.

The model keeps the mbarrier semantics (arrival count, transaction bytes,
phase; a parity wait returns once the barrier's current phase has the other
parity, so it cannot tell a phase from the one two before it), runs the roles
and the copies and MMAs in flight in random interleavings, and checks every
write and read window: no copy or stager write into a slot the MMAs still
read, the MMAs read the chunk they wait for, the Z block is not overwritten
while converted, an accumulator set is not overwritten while the epilogue
reads it, and no interleaving deadlocks.  The stagers' earlier protocol (a
parity wait on the empty barrier for the chunks they fill, skipping the ones
TMA fills) is planted as a mistake and must be caught: it let the stagers run
two phases ahead of that barrier and overwrite B under running MMAs.
"""

import random

import pytest


class MBar:
    """An mbarrier: expected arrivals per phase, pending transaction bytes, and
    the index of the phase in progress."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0

    def arrive(self, tx=0):
        self.tx += tx
        self.pending -= 1
        _check(self.pending >= 0, "more arrivals than the barrier's count")
        self._advance()

    def complete_tx(self, n):
        self.tx -= n
        self._advance()

    def _advance(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def parity_done(self, parity):
        return (self.phase & 1) != parity


class Violation(AssertionError):
    pass


def _check(cond, what):
    if not cond:
        raise Violation(what)


def run_protocol(seed, nst, items, nK, nX, stager_mode="producer_signal", max_steps=200000):
    """One random interleaving of one CTA's roles over `items` (a list of nXt
    values, the chunks of X that tensor copies bring for that item: 0 or nX).
    Chunks c < nX hold X rows, the others Z rows from the Z block."""
    rnd = random.Random(seed)
    full = [MBar(2) for _ in range(nst)]
    empty = [MBar(1) for _ in range(nst)]
    bfree = [MBar(1) for _ in range(nst)]
    accf = [MBar(1) for _ in range(2)]
    acce = [MBar(1) for _ in range(2)]
    zbar = MBar(1)
    # contents and windows
    slotA = [None] * nst
    slotB = [None] * nst
    readers = [0] * nst            # MMAs in flight on the slot
    b_writing = [False] * nst      # stagers inside their write of the slot's B
    x_inflight = [0] * nst         # tensor copies of X in flight into the slot's B
    acc_item = [None, None]        # (item, chunks accumulated) of each accumulator set
    acc_inflight = [0, 0]
    epi_reading = [None, None]
    zr = {"item": None, "reading": False, "inflight": 0}
    events = []                    # copies in flight: any order
    mma_fifo = []                  # MMAs and commits: in issue order

    def producer():
        g = 0
        for it, nXt in enumerate(items):
            for c in range(nK):
                s, u = g % nst, g // nst
                if u > 0:
                    yield ("wait", empty[s], (u - 1) & 1)
                tma_x = c < nXt
                full[s].arrive(tx=2 if tma_x else 1)          # arrival 1 with the copies' bytes

                def land_a(s=s, g=g):
                    _check(readers[s] == 0, "A copy lands in a slot the MMAs read")
                    slotA[s] = g
                    full[s].complete_tx(1)
                events.append(land_a)
                if tma_x:
                    x_inflight[s] += 1

                    def land_x(s=s, g=g):
                        _check(readers[s] == 0, "X copy lands in a slot the MMAs read")
                        _check(not b_writing[s], "X copy lands while the stagers write the slot")
                        slotB[s] = g
                        x_inflight[s] -= 1
                        full[s].complete_tx(1)
                    events.append(land_x)
                    full[s].arrive()                           # arrival 2: B comes with the copies
                elif stager_mode == "producer_signal":
                    bfree[s].arrive()
                g += 1
                yield ("step",)

    def mma():
        g = 0
        for kk in range(len(items)):
            b, ub = kk & 1, kk >> 1
            if ub > 0:
                yield ("wait", acce[b], (ub - 1) & 1)
            for c in range(nK):
                s = g % nst
                yield ("wait", full[s], (g // nst) & 1)
                _check(slotA[s] == g and slotB[s] == g,
                       "MMA reads a stale stage (A %s, B %s, chunk %d)" % (slotA[s], slotB[s], g))
                _check(not b_writing[s] and x_inflight[s] == 0, "MMA reads B while it is written")
                _check(epi_reading[b] is None, "MMA writes accumulators the epilogue reads")
                readers[s] += 1
                acc_inflight[b] += 1

                def done(s=s, b=b, kk=kk, c=c):
                    _check(epi_reading[b] is None, "MMA writes accumulators the epilogue reads")
                    readers[s] -= 1
                    acc_inflight[b] -= 1
                    acc_item[b] = (kk, c + 1)
                mma_fifo.append(done)
                mma_fifo.append(lambda s=s: empty[s].arrive())    # commit: after the MMAs before it
                g += 1
                yield ("step",)
            mma_fifo.append(lambda b=b: accf[b].arrive())

    def stagers():
        g = 0
        uses = [0] * nst
        zitem, zpend, zphase = None, False, 0

        def fetch(item):
            zbar.arrive(tx=1)
            zr["inflight"] += 1

            def land(item=item):
                _check(not zr["reading"], "Z block copy lands while it is converted")
                zr["item"] = item
                zr["inflight"] -= 1
                zbar.complete_tx(1)
            events.append(land)

        for it, nXt in enumerate(items):
            zready = False
            for c in range(nK):
                s, u = g % nst, g // nst
                if stager_mode == "producer_signal":
                    if c < nXt:
                        g += 1
                        continue
                    yield ("wait", bfree[s], uses[s] & 1)
                    uses[s] += 1
                else:                                       # the planted mistake
                    if c < nXt:
                        g += 1
                        continue
                    if u > 0:
                        yield ("wait", empty[s], (u - 1) & 1)
                zchunk = c >= nX
                if zchunk and not zready:
                    if zitem != it:
                        fetch(it)
                        zpend = True
                    if zpend:
                        yield ("wait", zbar, zphase & 1)
                        zphase += 1
                        zpend = False
                    _check(zr["item"] == it, "Z block of item %s converted for item %d" % (zr["item"], it))
                    zready = True
                    zitem = it
                _check(readers[s] == 0, "stagers write B of a slot the MMAs read")
                _check(x_inflight[s] == 0, "stagers write B while an X copy is in flight into it")
                b_writing[s] = True
                if zchunk:
                    zr["reading"] = True
                yield ("step",)
                _check(readers[s] == 0, "stagers write B of a slot the MMAs read")
                slotB[s] = g
                b_writing[s] = False
                zr["reading"] = False
                full[s].arrive()                            # arrival 2: B is in place
                g += 1
            if nK > nX and it + 1 < len(items):
                fetch(it + 1)                               # the next item's Z block, an item ahead
                zpend = True
                zitem = it + 1
        if zpend:
            yield ("wait", zbar, zphase & 1)

    def epilogue():
        for kk in range(len(items)):
            b, ub = kk & 1, kk >> 1
            yield ("wait", accf[b], ub & 1)
            _check(acc_inflight[b] == 0 and acc_item[b] == (kk, nK),
                   "epilogue reads accumulators %s for item %d" % (acc_item[b], kk))
            epi_reading[b] = kk
            yield ("step",)
            epi_reading[b] = None
            acce[b].arrive()

    roles = [producer(), mma(), stagers(), epilogue()]
    state = [None] * len(roles)
    alive = [True] * len(roles)
    for _ in range(max_steps):
        choices = []
        for i in range(len(roles)):
            if not alive[i]:
                continue
            w = state[i]
            if w is None or w[0] == "step" or w[1].parity_done(w[2]):
                choices.append(i)
        if events:
            choices.append("copy")
        if mma_fifo:
            choices.append("mma")
        if not choices:
            if not any(alive):
                return
            raise Violation("deadlock")
        pick = rnd.choice(choices)
        if pick == "copy":
            events.pop(rnd.randrange(len(events)))()
        elif pick == "mma":
            mma_fifo.pop(0)()
        else:
            try:
                state[pick] = next(roles[pick])
            except StopIteration:
                alive[pick] = False
    raise Violation("no end after %d steps" % max_steps)


def _items(rnd, n, nX):
    return [rnd.choice((0, nX)) for _ in range(n)]


CONFIGS = [(nst, nK, nX) for nst in (2, 3, 4, 6) for nK, nX in ((6, 4), (5, 1), (3, 2), (4, 0))]


@pytest.mark.parametrize("nst,nK,nX", CONFIGS)
def test_protocol_has_no_race_or_deadlock(nst, nK, nX):
    for seed in range(150):
        rnd = random.Random(1000 * seed + 7 * nst + nK)
        items = _items(rnd, rnd.randint(1, 7), nX)
        run_protocol(seed, nst, items, nK, nX)
    # every item fed by tensor copies of X, and none
    for seed in range(20):
        run_protocol(seed, nst, [nX] * 5, nK, nX)
        run_protocol(seed, nst, [0] * 5, nK, nX)


@pytest.mark.parametrize("nst", [2, 3])
def test_planted_stager_wait_on_empty_barrier_is_caught(nst):
    """The stagers' earlier wait (the empty barrier's parity for the chunks
    they fill) must fail: items whose X comes by tensor copies advance the
    slots without them, so their parity wait could be two phases ahead."""
    caught = 0
    for seed in range(300):
        rnd = random.Random(seed)
        items = _items(rnd, 6, 4)
        try:
            run_protocol(seed, nst, items, 6, 4, stager_mode="empty_parity")
        except Violation:
            caught += 1
    assert caught > 0


def test_model_barrier_parity_semantics():
    """The MBar model: a phase completes on its last arrival once its bytes
    have landed, and a parity wait is satisfied by the phase two later too."""
    b = MBar(2)
    b.arrive(tx=3)
    assert not b.parity_done(0)
    b.arrive()
    assert not b.parity_done(0)                 # bytes still in flight
    b.complete_tx(3)
    assert b.parity_done(0) and not b.parity_done(1)
    b.arrive()
    b.arrive()
    b.arrive()
    b.arrive()                                  # phases 1 and 2 complete
    assert b.phase == 3
    assert b.parity_done(0)                     # phase 0, 2: indistinguishable
