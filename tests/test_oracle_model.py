"""Pins for the oracle statistics and queue replay (Sections 3.1.1, 3.2, 3.2.1)."""
import numpy as np

import oracle
from oracle import bvss as ob
from oracle import model as om
from paper_2512_21967_gb300 import synth


def csr(n, edges):
    src = np.array([e[0] for e in edges], np.int32)
    dst = np.array([e[1] for e in edges], np.int32)
    return synth.csr_from_edges(n, src, dst)


def test_update_divergence_hand_example():
    # slice set 0 (columns 0..7) pulled by rows 10 and 30 only, through column 0:
    # one VSS, one non-empty column {10, 30}: population std = 10.  Slice sets of
    # rows 10 and 30 (1 and 3) each hold the single row 0: std 0.  U_div = 10/3.
    g = csr(40, [(0, 10), (0, 30)])
    b = ob.build(g.n, g.row_ptr, g.col_idx)
    assert b.num_vss == 3
    assert abs(om.update_divergence(b) - 10.0 / 3.0) < 1e-12


def test_update_divergence_multi_column():
    # 40 rows pull from column 0 -> slices k=0..39 fill lanes 0..31 of sub-slot 0
    # and lanes 0..7 of sub-slot 1: rows sorted 100..139
    rows = list(range(100, 140))
    g = csr(200, [(0, r) for r in rows])
    b = ob.build(g.n, g.row_ptr, g.col_idx)
    col0 = np.std(np.array(rows[:32], float))
    col1 = np.std(np.array(rows[32:], float))
    vss0 = (col0 + col1) / 2
    # the other VSSs (slice sets of rows 100..139, each pulled by row 0) have std 0
    assert abs(om.update_divergence(b) - vss0 / b.num_vss) < 1e-9


def test_compression_ratio_bounds():
    # a complete bipartite block 8 x 8 in aligned slice sets: every mask full
    g = csr(16, [(i, 8 + j) for i in range(8) for j in range(8)])
    b = ob.build(g.n, g.row_ptr, g.col_idx)
    assert om.compression_ratio(g.nnz, ob.unpadded_slices(b)) == 1.0
    # a perfect matching between two slice sets: one bit per slice -> 1/8
    g2 = csr(16, [(i, 8 + i) for i in range(8)])
    b2 = ob.build(g2.n, g2.row_ptr, g2.col_idx)
    assert om.compression_ratio(g2.nnz, ob.unpadded_slices(b2)) == 1 / 8


def test_lazy_rule_threshold():
    assert not om.use_lazy(25_000) and om.use_lazy(25_000.5)


def test_queue_replay_path():
    # path 0-1-...-39 from 0: level l frontier is vertex l-1, slice set (l-1)//8.
    n = 40
    g = csr(n, [(i, i + 1) for i in range(n - 1)])
    b = ob.build(n, g.row_ptr, g.col_idx)
    lv = oracle.bfs_levels(n, g.row_ptr, g.col_idx, 0)
    sizes = om.queue_sizes(b, lv)
    assert len(sizes) == n            # levels 1..40, the 40th finds nothing
    assert all(s == 1 for s in sizes)  # every slice set of a path has < 128 slices


def test_queue_replay_matches_direct_simulation():
    """Simulate the level loop literally: frontier set -> every VSS of every slice
    set with a frontier column; compare the per-level VSS counts."""
    g = synth.rmat_graph(9, 16, seed=3)
    b = ob.build(g.n, g.row_ptr, g.col_idx)
    src = int(synth.pick_sources(g, 1, 5)[0])
    lv = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, src)
    frontier = {src}
    visited = {src}
    sim = []
    while True:
        sets = {c // 8 for c in frontier}
        vss = [nu for s in sets for nu in range(b.real_ptrs[s], b.real_ptrs[s + 1])]
        sim.append(len(vss))
        nxt = set()
        for nu in vss:
            s = int(b.virtual_to_real[nu])
            alpha = sum(1 << (c - 8 * s) for c in frontier if c // 8 == s)
            for u, m in ob.vss_slices(b, nu):
                if m & alpha and u not in visited:
                    nxt.add(u)
        if not nxt:
            break
        visited |= nxt
        frontier = nxt
    assert sim == om.queue_sizes(b, lv)
