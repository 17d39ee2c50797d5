"""The lazy update's visited test (Algorithm 3 with the V_next filter), modelled
on the CPU under arbitrary staleness of the words it reads.

Device code: `mark_rows` / `sweep` in paper_2512_21967_gb300/csrc/bfs_kernel.cu
(one bit per vertex) and `ms_pull_tile` / `ms_sweep` in msbfs_kernel.cu (k bits
per vertex).  Stage 1 marks every hit row in V_next unless the row's V_next word
already holds the bits; the sweep turns V_next ^ V_curr into the next level and
copies V_next into V_curr.  V_next only ever gains bits and contains V_curr, so
a read of it may return any earlier value of the word, a subset of its current
bits (other blocks' marks arrive late; an L1 copy may even date from an earlier
level), and the levels must not change: a stale word can only let a redundant
mark through, and a mark of bits V_next already holds changes nothing.  The
model draws such a subset for every test and checks the levels against the
oracle; a planted read that may return bits no one has set yet must be caught."""
import random

import numpy as np
import pytest

import oracle
from paper_2512_21967_gb300 import synth


def lazy_levels(g, srcs, rng, future_bits=False):
    """Levels of k = len(srcs) traversals by the modelled lazy update: vertex v
    carries a k-bit word (bit i: source i).  Returns int32[k, n]."""
    n, k = g.n, len(srcs)
    full = (1 << k) - 1
    rp, ci = g.row_ptr, g.col_idx
    vcur = [0] * n
    vnext = [0] * n
    levels = np.full((k, n), -1, np.int32)
    for i, s in enumerate(srcs):
        vnext[int(s)] |= 1 << i
    lvl = 0
    while True:
        # sweep: new bits become level lvl
        front = [0] * n
        any_new = False
        for v in range(n):
            d = vnext[v] & ~vcur[v]
            if d:
                any_new = True
                front[v] = d
                for i in range(k):
                    if (d >> i) & 1:
                        levels[i, v] = lvl
                vcur[v] = vnext[v]
        if not any_new:
            return levels
        lvl += 1
        # stage 1 (pull): row u gathers the frontier bits of its neighbours, in a random
        # order of rows, and tests a possibly stale copy of its V_next word
        order = list(range(n))
        rng.shuffle(order)
        for u in order:
            y = 0
            for e in range(rp[u], rp[u + 1]):
                y |= front[ci[e]]
            if not y:
                continue
            # any earlier value of the word: a subset of its current bits
            seen = vnext[u] & rng.getrandbits(max(k, 1))
            if future_bits:
                seen |= rng.getrandbits(max(k, 1)) & full   # planted: bits nobody has set
            fresh = y & ~seen
            if fresh:
                vnext[u] |= fresh


def graphs():
    yield synth.rmat_graph(6, 8, seed=21)
    yield synth.grid_graph(9, 0.8, seed=22)[0]
    n = 40
    a = np.arange(n - 1, dtype=np.int32)
    yield synth.csr_from_edges(n, a, a + 1)


@pytest.mark.parametrize("k", [1, 3, 8])
def test_stale_visited_reads_keep_the_levels(k):
    rng = random.Random(5)
    for g in graphs():
        srcs = synth.pick_sources(g, k, seed=7 + k)
        want = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs)
        for _ in range(25):
            assert np.array_equal(lazy_levels(g, srcs, rng), want)


def test_reading_bits_nobody_set_is_caught():
    """Planted in the model: a visited test that may see bits not yet set skips
    marks that were needed, and some level comes out wrong."""
    rng = random.Random(9)
    g = synth.rmat_graph(6, 8, seed=21)
    srcs = synth.pick_sources(g, 3, seed=4)
    want = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs)
    assert any(not np.array_equal(lazy_levels(g, srcs, rng, future_bits=True), want) for _ in range(20))
