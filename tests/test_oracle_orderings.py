"""Pins for the oracle orderings (Section 3.2): closed forms and monotone checks."""
import json
import os

import numpy as np
import pytest

from oracle import bvss as ob
from oracle import model as om
from oracle import orderings as oo
from paper_2512_21967_gb300 import synth


def csr(n, edges):
    src = np.array([e[0] for e in edges] or [0], np.int32)[:len(edges)]
    dst = np.array([e[1] for e in edges] or [0], np.int32)[:len(edges)]
    return synth.csr_from_edges(n, src, dst)


def is_perm(p, n):
    return sorted(np.asarray(p).tolist()) == list(range(n))


def test_rcm_path_closed_form():
    # a path scrambled by a known relabel: RCM starts at an end and walks it, so
    # consecutive path vertices get consecutive new ids (bandwidth 1)
    n = 23
    perm = synth.permutation(n, 5)
    g = csr(n, [(int(perm[i]), int(perm[i + 1])) for i in range(n - 1)])
    p = oo.rcm(n, g.row_ptr, g.col_idx)
    assert is_perm(p, n)
    rp, ci = oo.relabel(n, g.row_ptr, g.col_idx, p)
    assert oo.bandwidth(n, rp, ci) == 1


def test_rcm_star_and_isolated():
    n = 9
    g = csr(n, [(0, i) for i in range(1, 7)])   # 7, 8 isolated
    p = oo.rcm(n, g.row_ptr, g.col_idx)
    assert is_perm(p, n)
    # George-Liu from 0 moves to leaf 1 (ecc 2 > 1); CM from 1: 1, 0, 2..6; then 7, 8.
    # Reversed over all n: new_id = n-1-position
    order = [1, 0, 2, 3, 4, 5, 6, 7, 8]
    exp = np.empty(n, np.int32)
    for pos, v in enumerate(order):
        exp[v] = n - 1 - pos
    assert np.array_equal(p, exp)


def test_rcm_recovers_grid_bandwidth():
    side = 12
    g, _ = synth.grid_graph(side, p=1.0, seed=3)
    assert oo.bandwidth(g.n, g.row_ptr, g.col_idx) > 3 * side
    p = oo.rcm(g.n, g.row_ptr, g.col_idx)
    assert is_perm(p, g.n)
    rp, ci = oo.relabel(g.n, g.row_ptr, g.col_idx, p)
    assert oo.bandwidth(g.n, rp, ci) <= side + 1


def test_rcm_reduces_update_divergence_on_grid():
    """Table 1b's direction: RCM lowers U_div on a randomly numbered grid."""
    g, _ = synth.grid_graph(32, p=0.9, seed=8)
    before = om.update_divergence(ob.build(g.n, g.row_ptr, g.col_idx))
    p = oo.rcm(g.n, g.row_ptr, g.col_idx)
    rp, ci = oo.relabel(g.n, g.row_ptr, g.col_idx, p)
    after = om.update_divergence(ob.build(g.n, rp, ci))
    assert after < before / 4


def test_jaccard_sigma_one_is_identity():
    g = synth.rmat_graph(6, 8, seed=3)
    p = oo.jaccard_windows(g.n, g.row_ptr, g.col_idx, sigma=1, w=16)
    assert np.array_equal(p, np.arange(g.n))


def test_jaccard_planted_twins():
    """16 window vertices, even ids all adjacent to hubs {16,17}, odd ids to
    {18,19}: J = 1 inside a group, 0 across.  Algorithm 1 with sigma = 8 must make
    cluster 0 = the even ids in ascending order, cluster 1 = the odd ids."""
    n = 20
    edges = [(v, 16 + (v % 2) * 2 + h) for v in range(16) for h in range(2)]
    g = csr(n, edges)
    p = oo.jaccard_windows(n, g.row_ptr, g.col_idx, sigma=8, w=16)
    assert [int(p[v]) for v in range(0, 16, 2)] == list(range(0, 8))
    assert [int(p[v]) for v in range(1, 16, 2)] == list(range(8, 16))
    # trailing short window [16, 20): one cluster of 4
    assert sorted(int(p[v]) for v in range(16, 20)) == [16, 17, 18, 19]
    # compression: interleaved order gives masks of 4 bits per hub row, planted
    # order gives full 8-bit masks -> ratio doubles
    b0 = ob.build(n, g.row_ptr, g.col_idx)
    rp, ci = oo.relabel(n, g.row_ptr, g.col_idx, p)
    b1 = ob.build(n, rp, ci)
    assert ob.unpadded_slices(b1) < ob.unpadded_slices(b0)


def test_jaccard_tie_goes_to_smallest_id():
    # all vertices isolated: every J is 0, so each pick is the smallest remaining id
    n = 24
    g = csr(n, [])
    p = oo.jaccard_windows(n, g.row_ptr, g.col_idx, sigma=8, w=8)
    assert np.array_equal(p, np.arange(n))


def test_hub_prepass_star():
    n = 8
    g = csr(n, [(5, i) for i in range(n) if i != 5])
    p = oo.hub_bfs_prepass(n, g.row_ptr, g.col_idx)
    assert p[5] == 0 and np.array_equal(np.sort(p), np.arange(n))
    assert [int(p[v]) for v in [0, 1, 2, 3, 4, 6, 7]] == [1, 2, 3, 4, 5, 6, 7]


def test_compress_order_beats_random_relabel():
    g = synth.rmat_graph(9, 16, seed=6)
    b0 = ob.build(g.n, g.row_ptr, g.col_idx)
    p = oo.compress_order(g.n, g.row_ptr, g.col_idx, sigma=8, w=64)
    assert is_perm(p, g.n)
    rp, ci = oo.relabel(g.n, g.row_ptr, g.col_idx, p)
    b1 = ob.build(g.n, rp, ci)
    assert om.compression_ratio(g.nnz, ob.unpadded_slices(b1)) > om.compression_ratio(g.nnz, ob.unpadded_slices(b0))


def test_relabel_preserves_levels():
    import oracle
    g = synth.rmat_graph(8, 8, seed=2)
    p = synth.permutation(g.n, 77)
    rp, ci = oo.relabel(g.n, g.row_ptr, g.col_idx, p)
    a = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, 3)
    b = oracle.bfs_levels(g.n, rp, ci, int(p[3]))
    assert np.array_equal(a, b[p])


GORDER_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gorder_hand.json")


def test_gorder_hand_worked_example():
    """Gorder's greedy on a 6-vertex graph, worked by hand from its definition
    (tests/golden/gorder_hand.json), with and without a hub cap."""
    gold = json.load(open(GORDER_GOLDEN))
    e = np.array(gold["edges"], np.int32)
    g = synth.csr_from_edges(gold["n"], e[:, 0], e[:, 1])
    for case in gold["cases"]:
        got = oo.gorder(g.n, g.row_ptr, g.col_idx, w=5, hub_cap=case["hub_cap"])
        assert got.tolist() == case["new_id"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gorder_invariants_and_objective(seed):
    g = synth.rmat_graph(7, 8, seed=seed)
    p = oo.gorder(g.n, g.row_ptr, g.col_idx)
    assert sorted(p.tolist()) == list(range(g.n))
    deg = np.diff(g.row_ptr)
    first = int(np.nonzero(p == 0)[0][0])
    assert deg[first] == deg.max() and first == int(np.argmax(deg))
    # the greedy order scores far above a random order on Gorder's own objective
    rnd = synth.permutation(g.n, 99 + seed)
    assert oo.gorder_objective(g.n, g.row_ptr, g.col_idx, p) > 1.5 * oo.gorder_objective(g.n, g.row_ptr, g.col_idx, rnd)


def test_gorder_planted_mistake_fails():
    """Forgetting to drop the vertex that leaves the window (an unbounded
    window) must change the order of the hand-worked graph's larger cousin."""
    g = synth.rmat_graph(6, 8, seed=4)
    adj = [set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    deg = [len(a) for a in adj]

    def unbounded(n):
        order, placed = [], [False] * n
        for _ in range(n):
            best, bk = -1, -1
            for u in range(n):
                if placed[u]:
                    continue
                k = deg[u] if not order else sum((2 if v in adj[u] else 0) +
                                                  sum(1 for x in adj[u] & adj[v] if deg[x] <= 64) for v in order)
                if k > bk:
                    best, bk = u, k
            placed[best] = True
            order.append(best)
        out = np.empty(n, np.int64)
        out[order] = np.arange(n)
        return out
    assert not np.array_equal(unbounded(g.n), oo.gorder(g.n, g.row_ptr, g.col_idx))
