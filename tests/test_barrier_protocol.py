"""The grid barrier's ring protocol, modelled on the CPU and checked under many
interleavings of the blocks' steps.  Device code: `grid_barrier` and
`ring_word` in paper_2512_21967_gb300/csrc/device_common.cuh.

Protocol (sequentially consistent model; the device's release/acquire ordering
is what makes each step below visible in this order): barrier number b uses
ring word b mod 4, whose high half counts arrivals and whose low half is the
queue size that the phase before the barrier appends to.  In each phase a block
first adds its appends to the low half of the word of the barrier that ends the
phase, then arrives (+1 in the high half), then polls until all blocks have
arrived; the poll that completes returns the low half.  Block 0, on completing
barrier b, clears word (b + 2) mod 4.

Checked in every interleaving: every block completes every barrier, and the
value it returns is exactly the sum of that phase's appends (no arrival or
append of another barrier mixed in, no clear lost or premature).  Planted
mutants of the clear distance must fail the check."""
import random

import pytest

RING = 4


def run(nblocks, nbarriers, appends, seed, clear_ahead=2):
    """One random interleaving.  appends[i][b]: what block i appends before
    barrier b.  Returns the values each block read at each barrier, or raises
    AssertionError when the protocol lets a block complete a barrier wrongly."""
    rng = random.Random(seed)
    arr = [0] * RING
    low = [0] * RING
    # per block: next barrier, phase (0 append, 1 arrive, 2 poll)
    bar = [0] * nblocks
    phase = [0] * nblocks
    seen = [[None] * nbarriers for _ in range(nblocks)]
    steps = 0
    while any(b < nbarriers for b in bar):
        steps += 1
        assert steps < 100000, "no progress: a barrier can never complete"
        i = rng.choice([j for j in range(nblocks) if bar[j] < nbarriers])
        b = bar[i]
        w = b % RING
        if phase[i] == 0:
            low[w] += appends[i][b]
            phase[i] = 1
        elif phase[i] == 1:
            arr[w] += 1
            phase[i] = 2
        else:
            if arr[w] >= nblocks:
                seen[i][b] = (arr[w], low[w])
                if i == 0:
                    c = (b + clear_ahead) % RING
                    arr[c] = 0
                    low[c] = 0
                bar[i] += 1
                phase[i] = 0
    return seen


def check(nblocks, nbarriers, seed, clear_ahead=2):
    rng = random.Random(seed * 7919 + 1)
    appends = [[rng.randrange(0, 5) for _ in range(nbarriers)] for _ in range(nblocks)]
    seen = run(nblocks, nbarriers, appends, seed, clear_ahead)
    for b in range(nbarriers):
        want = sum(appends[i][b] for i in range(nblocks))
        for i in range(nblocks):
            arrivals, value = seen[i][b]
            assert arrivals == nblocks, f"block {i} passed barrier {b} with {arrivals} arrivals"
            assert value == want, f"block {i} read {value} at barrier {b}, the phase appended {want}"


@pytest.mark.parametrize("nblocks", [1, 2, 3, 5])
def test_ring_barrier_returns_each_phase_exactly(nblocks):
    for seed in range(400):
        check(nblocks, 13, seed)


@pytest.mark.parametrize("clear_ahead", [0, 1])
def test_clearing_too_close_is_caught(clear_ahead):
    """Clearing the word of the barrier just passed (0) or of the next one (1)
    loses arrivals or appends that other blocks already made, in some
    interleaving: the model must see it."""
    for seed in range(400):
        try:
            check(3, 13, seed, clear_ahead)
        except AssertionError:
            return
    pytest.fail(f"clearing {clear_ahead} ahead passed 400 interleavings")
