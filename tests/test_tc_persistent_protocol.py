"""Barrier protocol of the persistent tensor-core mode product, simulated on the host.

`tc_gemm_persistent_kernel` (kernels_fd_tc.cu) runs three roles per CTA over the CTA's tiles
(tile = blockIdx.x + i * gridDim.x):

* the TMA producer fills ring stage g % nstage with chunk g of the CTA's (tile, chunk)
  sequence after waiting for phase g / nstage - 1 of that stage's `empty` barrier;
* the MMA issuer waits for `full` phase g / nstage, accumulates into TMEM accumulator
  i & 1 (after waiting for phase i / 2 - 1 of `acce[i & 1]`), commits each stage to
  `empty` and the finished accumulator to `accf[i & 1]`;
* four epilogue warps wait for `accf[i & 1]` phase i / 2, drain the accumulator and
  arrive on `acce[i & 1]` (count 4).

Here each role is a generator over mbarriers with phase / parity semantics (a parity wait
succeeds once the phase of that parity has completed), run in random interleavings: every
tile must be summed over all its chunks from the right ring stages, drained once, in
order, and no interleaving may deadlock.
"""

import random


class Bar:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):
        return (self.phase & 1) != parity


def simulate_cta(tiles, nchunks, nstage, rnd):
    full = [Bar(1) for _ in range(nstage)]
    empty = [Bar(1) for _ in range(nstage)]
    accf, acce = [Bar(1), Bar(1)], [Bar(4), Bar(4)]
    ring = [None] * nstage      # (tile, chunk) a stage holds, None when free
    acc = [None, None]          # accumulator: (tile, chunks summed)
    drained = []

    def producer():
        g = 0
        for t in tiles:
            for c in range(nchunks):
                s, use = g % nstage, g // nstage
                if use > 0:
                    while not empty[s].done((use - 1) & 1):
                        yield
                assert ring[s] is None, "stage overwritten before it was consumed"
                ring[s] = (t, c)
                full[s].arrive()  # the copy lands (expect_tx + complete_tx)
                g += 1
                yield

    def mma():
        g = 0
        for i, t in enumerate(tiles):
            b, ub = i & 1, i >> 1
            if ub > 0:
                while not acce[b].done((ub - 1) & 1):
                    yield
            assert acc[b] is None, "accumulator reused before it was drained"
            acc[b] = (t, 0)
            for c in range(nchunks):
                s, use = g % nstage, g // nstage
                while not full[s].done(use & 1):
                    yield
                assert ring[s] == (t, c)
                acc[b] = (t, acc[b][1] + 1)
                ring[s] = None
                empty[s].arrive()
                g += 1
                yield
            accf[b].arrive()

    def epilogue(w):
        for i, t in enumerate(tiles):
            b, ub = i & 1, i >> 1
            while not accf[b].done(ub & 1):
                yield
            assert acc[b] == (t, nchunks)
            yield
            if w == 0:
                drained.append(t)
            acce[b].arrive()
            if acce[b].phase == ub + 1 and acce[b].pending == acce[b].count:
                acc[b] = None  # all four warps have drained it

    live = [producer(), mma()] + [epilogue(w) for w in range(4)]
    steps = 0
    while live:
        gen = rnd.choice(live)
        try:
            next(gen)
        except StopIteration:
            live.remove(gen)
        steps += 1
        assert steps < 10 ** 6, "deadlock"
    assert drained == list(tiles)


def test_protocol_over_random_shapes_and_interleavings():
    for seed in range(150):
        rnd = random.Random(seed)
        ntiles = rnd.randint(1, 40)
        grid = rnd.randint(1, ntiles)
        nchunks, nstage = rnd.randint(1, 9), rnd.randint(2, 8)
        for cta in range(grid):
            simulate_cta(range(cta, ntiles, grid), nchunks, nstage, rnd)


def test_a_broken_protocol_is_caught():
    """Plant a mistake in the model: the MMA issuer no longer waits for the epilogue before
    it reuses an accumulator.  With two or more tiles per CTA some interleaving must trip."""
    tripped = False
    orig = Bar.done
    try:
        def done(self, parity):  # acce (count 4) always reads as drained
            return True if self.count == 4 else orig(self, parity)
        Bar.done = done
        for seed in range(50):
            try:
                simulate_cta(range(0, 6), 3, 2, random.Random(seed))
            except AssertionError:
                tripped = True
                break
    finally:
        Bar.done = orig
    assert tripped
