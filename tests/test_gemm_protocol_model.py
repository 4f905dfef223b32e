"""CPU model of the persistent digit GEMM's pipeline protocol (gemm_oz.cu).

The kernel's three roles keep running counters across the output tiles a CTA walks: the
TMA producer (stage full / empty barriers), the MMA issuer (per 512-deep chunk: the lower
levels into H buffer gch & 1 once that buffer's previous use is drained, the exact levels
once the previous chunk's exact levels are drained, a commit per stage and per chunk) and
the drain warps (exact levels, then H, each signalled on its own barrier).  This model
replays those waits and arrivals with mbarrier phase-parity semantics under random
interleavings, with tensor-core products that complete in issue order and TMA loads that
land in any order, and checks that every schedule finishes (no deadlock) and that no
stage is overwritten before its products ran and no accumulator is read before its
chunk's products completed or after the next chunk's started.  The split-BF16 kernel's
protocol (one accumulator per tile, two alternating, released by the drain warps) is
modelled the same way.  A planted parity mistake makes each model fail.
"""
import random

import pytest

CHUNK_KS = 32


class Bar:
    def __init__(self, count):
        self.count, self.arr, self.ph = count, 0, 0

    def arrive(self):
        self.arr += 1
        assert self.arr <= self.count
        if self.arr == self.count:
            self.arr = 0
            self.ph += 1

    def test(self, parity):  # try_wait.parity: true once the phase with this parity is done
        return (self.ph & 1) != parity


def simulate(tiles_nk, nst, NL=2, NS=5, ndrain=2, seed=0, h_parity_flip=0):
    rng = random.Random(seed)
    full = [Bar(1) for _ in range(nst)]
    empty = [Bar(1) for _ in range(nst)]
    chunk_done, exact_drained, all_done = Bar(1), Bar(ndrain), Bar(1)
    hbuf = [Bar(ndrain), Bar(ndrain)]
    stage_ver = [None] * nst        # iteration whose data the stage holds
    pending_tma = []                # (stage, it) loads in flight
    fifo = []                       # tensor-core queue: ('mma', buf, chunk, stage, it) / ('commit', bar)
    last_written = {}               # accumulator -> chunk of the last executed product

    def producer():
        it = 0
        for nk in tiles_nk:
            for i in range(nk):
                st = it % nst
                while not empty[st].test(((it // nst) & 1) ^ 1):
                    yield
                pending_tma.append((st, it))
                it += 1
        for j in range(max(it - nst, 0), it):
            while not full[j % nst].test((j // nst) & 1):
                yield

    def issuer():
        it = gch = 0
        issued = False
        for nk in tiles_nk:
            nch = (nk + CHUNK_KS - 1) // CHUNK_KS
            for ch in range(nch):
                kbeg, kend = ch * CHUNK_KS, min((ch + 1) * CHUNK_KS, nk)
                for ks in range(kbeg, kend):
                    st = it % nst
                    while not full[st].test((it // nst) & 1):
                        yield
                    if ks == kbeg and gch >= 2:
                        while not hbuf[gch & 1].test((((gch - 2) >> 1) & 1) ^ h_parity_flip):
                            yield
                    for _ in range(NS * (NS + 1) // 2 - NL * (NL + 1) // 2):
                        fifo.append(('mma', 'H%d' % (gch & 1), gch, st, it))
                    if ks == kbeg and gch > 0:
                        while not exact_drained.test((gch - 1) & 1):
                            yield
                    for l in range(NL):
                        fifo.append(('mma', 'L%d' % l, gch, st, it))
                    fifo.append(('commit', empty[st]))
                    issued = True
                    it += 1
                    yield
                fifo.append(('commit', chunk_done))
                gch += 1
        if issued:
            fifo.append(('commit', all_done))
            while not all_done.test(0):
                yield

    def drain(w):
        gch = 0
        for nk in tiles_nk:
            nch = (nk + CHUNK_KS - 1) // CHUNK_KS
            for ch in range(nch):
                while not chunk_done.test(gch & 1):
                    yield
                for l in range(NL):
                    assert last_written.get('L%d' % l) == gch, ('exact', l, gch, last_written)
                exact_drained.arrive()
                yield
                assert last_written.get('H%d' % (gch & 1)) == gch, ('H', gch, last_written)
                hbuf[gch & 1].arrive()
                gch += 1
                yield
            for _ in range(rng.randint(0, 6)):   # epilogue from registers
                yield

    roles = [producer(), issuer()] + [drain(w) for w in range(ndrain)]
    alive = list(range(len(roles)))
    steps = 0
    while alive or pending_tma or fifo:
        steps += 1
        assert steps < 10 ** 7, "no progress"
        ev = rng.random()
        if pending_tma and ev < 0.2:
            st, it = pending_tma.pop(rng.randrange(len(pending_tma)))   # any order
            assert stage_ver[st] is None or stage_ver[st] == it - nst, ('overwrite', st, it)
            stage_ver[st] = it
            full[st].arrive()
            continue
        if fifo and ev < 0.5:
            op = fifo.pop(0)
            if op[0] == 'mma':
                _, buf, g, st, it = op
                assert stage_ver[st] == it, ('stage data', st, it, stage_ver[st])
                last_written[buf] = g
            else:
                op[1].arrive()
            continue
        if not alive:
            if not pending_tma and not fifo:
                break
            continue
        r = rng.choice(alive)
        try:
            next(roles[r])
        except StopIteration:
            alive.remove(r)
        # deadlock check: nothing in flight and every live role blocked for long
    assert not pending_tma and not fifo
    return steps


CFGS = [([4], 4), ([4] * 9, 4), ([64, 100, 33, 5], 3), ([32] * 7, 5), ([1] * 20, 2),
        ([144] * 3, 4), ([97, 3, 200, 31, 64], 7), ([144, 144, 1296], 4)]


@pytest.mark.parametrize("tiles,nst", CFGS)
def test_protocol_finishes_without_hazards(tiles, nst):
    for seed in range(12):
        simulate(tiles, nst, seed=seed)                       # five-digit form
        simulate(tiles, nst, NL=4, NS=7, seed=seed + 100)    # seven-digit form


def test_planted_parity_mistake_is_caught():
    with pytest.raises(AssertionError):
        for seed in range(12):
            simulate([64] * 4, 4, seed=seed, h_parity_flip=1)


def simulate_split(tiles_nk, nst, ndrain=2, seed=0, acc_parity_flip=0):
    """The split-BF16 kernel: every product of a tile into accumulator lt & 1 over the
    tile's whole K, one commit per tile, the drain warps read the tile out and release the
    accumulator for tile lt + 2."""
    rng = random.Random(seed)
    full = [Bar(1) for _ in range(nst)]
    empty = [Bar(1) for _ in range(nst)]
    acc_full = [Bar(1), Bar(1)]
    acc_empty = [Bar(ndrain), Bar(ndrain)]
    all_done = Bar(1)
    stage_ver = [None] * nst
    pending_tma, fifo = [], []
    acc_tile = {0: None, 1: None}    # tile whose products the accumulator holds
    read_out = set()

    def producer():
        it = 0
        for nk in tiles_nk:
            for i in range(nk):
                st = it % nst
                while not empty[st].test(((it // nst) & 1) ^ 1):
                    yield
                pending_tma.append((st, it))
                it += 1
        for j in range(max(it - nst, 0), it):
            while not full[j % nst].test((j // nst) & 1):
                yield

    def issuer():
        it = 0
        for lt, nk in enumerate(tiles_nk):
            j = lt & 1
            if lt >= 2:
                while not acc_empty[j].test((((lt - 2) >> 1) & 1) ^ acc_parity_flip):
                    yield
            for i in range(nk):
                st = it % nst
                while not full[st].test((it // nst) & 1):
                    yield
                fifo.append(('mma', j, lt, st, it))
                fifo.append(('commit', empty[st]))
                it += 1
                yield
            fifo.append(('commit', acc_full[j]))
        fifo.append(('commit', all_done))
        while not all_done.test(0):
            yield

    def drain(w):
        for lt in range(len(tiles_nk)):
            j = lt & 1
            while not acc_full[j].test((lt >> 1) & 1):
                yield
            assert acc_tile[j] == lt, ('acc', lt, acc_tile)
            read_out.add((w, lt))
            acc_empty[j].arrive()
            for _ in range(rng.randint(0, 6)):   # the stores of the tile
                yield

    roles = [producer(), issuer()] + [drain(w) for w in range(ndrain)]
    alive = list(range(len(roles)))
    steps = 0
    while alive or pending_tma or fifo:
        steps += 1
        assert steps < 10 ** 7, "no progress"
        ev = rng.random()
        if pending_tma and ev < 0.2:
            st, it = pending_tma.pop(rng.randrange(len(pending_tma)))
            assert stage_ver[st] is None or stage_ver[st] == it - nst, ('overwrite', st, it)
            stage_ver[st] = it
            full[st].arrive()
            continue
        if fifo and ev < 0.5:
            op = fifo.pop(0)
            if op[0] == 'mma':
                _, j, lt, st, it = op
                assert stage_ver[st] == it, ('stage data', st, it)
                # the accumulator must have been read out before a new tile writes it
                assert acc_tile[j] in (None, lt) or all((w, acc_tile[j]) in read_out
                                                         for w in range(ndrain)), ('reuse', j)
                acc_tile[j] = lt
            else:
                op[1].arrive()
            continue
        if not alive:
            continue
        r = rng.choice(alive)
        try:
            next(roles[r])
        except StopIteration:
            alive.remove(r)
    assert len(read_out) == ndrain * len(tiles_nk)


@pytest.mark.parametrize("tiles,nst", CFGS)
def test_split_protocol_finishes_without_hazards(tiles, nst):
    for seed in range(12):
        simulate_split(tiles, nst, seed=seed)


def test_split_planted_parity_mistake_is_caught():
    with pytest.raises(AssertionError):
        for seed in range(12):
            simulate_split([8] * 6, 4, seed=seed, acc_parity_flip=1)
