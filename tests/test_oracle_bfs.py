"""Pins for the oracle BFS (``oracle.bfs_levels``) against brute force, closed
forms, invariants and a library routine -- nothing here uses the CUDA path."""
import numpy as np
import pytest

import oracle
from paper_2512_21967_gb300 import synth


def csr_from_undirected(n, edges):
    src = np.array([e[0] for e in edges], dtype=np.int32)
    dst = np.array([e[1] for e in edges], dtype=np.int32)
    return synth.csr_from_edges(n, src, dst)


def brute_force_levels(n, g, src):
    """Level = first l with v in R_l, R_0 = {src}, R_{l+1} = R_l | A R_l (Boolean),
    bitsets as Python ints (the repeated Boolean adjacency product of Section 2)."""
    rows = [0] * n
    for u in range(n):
        for v in g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]:
            rows[u] |= 1 << int(v)
    lvl = [-1] * n
    R = 1 << src
    lvl[src] = 0
    for step in range(1, n + 1):
        nxt = R
        for u in range(n):
            if rows[u] & R:
                nxt |= 1 << u
        if nxt == R:
            break
        for u in range(n):
            if (nxt >> u) & 1 and lvl[u] < 0:
                lvl[u] = step
        R = nxt
    return np.array(lvl, dtype=np.int32)


def check_invariants(g, src, lvl):
    rp, ci = g.row_ptr.astype(np.int64), g.col_idx.astype(np.int64)
    assert lvl[src] == 0
    assert np.all(lvl >= -1)
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    a, b = lvl[rows], lvl[ci]
    both = (a >= 0) & (b >= 0)
    assert np.all(np.abs(a[both] - b[both]) <= 1), "edge spans more than one level"
    assert not np.any((a >= 0) ^ (b >= 0)), "edge joins reached and unreached vertex"
    # every reached non-source vertex has a neighbour exactly one level lower
    has_parent = np.zeros(g.n, dtype=bool)
    ok = both & (b == a - 1)
    has_parent[rows[ok]] = True
    reached = np.nonzero(lvl > 0)[0]
    assert np.all(has_parent[reached])


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_random_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 65))
    m = int(rng.integers(0, 3 * n))
    edges = [(int(rng.integers(n)), int(rng.integers(n))) for _ in range(m)]
    g = csr_from_undirected(n, edges)
    for src in sorted(set([0, n - 1, int(rng.integers(n))])):
        lvl = oracle.bfs_levels(n, g.row_ptr, g.col_idx, src)
        assert np.array_equal(lvl, brute_force_levels(n, g, src))
        check_invariants(g, src, lvl)


def test_path_closed_form():
    n = 37
    g = csr_from_undirected(n, [(i, i + 1) for i in range(n - 1)])
    assert np.array_equal(oracle.bfs_levels(n, g.row_ptr, g.col_idx, 0), np.arange(n))
    c = 17
    assert np.array_equal(oracle.bfs_levels(n, g.row_ptr, g.col_idx, c), np.abs(np.arange(n) - c))


def test_star_closed_form():
    n = 20
    g = csr_from_undirected(n, [(0, i) for i in range(1, n)])
    centre = oracle.bfs_levels(n, g.row_ptr, g.col_idx, 0)
    assert centre[0] == 0 and np.all(centre[1:] == 1)
    leaf = oracle.bfs_levels(n, g.row_ptr, g.col_idx, 5)
    exp = np.full(n, 2); exp[0] = 1; exp[5] = 0
    assert np.array_equal(leaf, exp)


def test_cycle_closed_form():
    n = 31
    g = csr_from_undirected(n, [(i, (i + 1) % n) for i in range(n)])
    i = np.arange(n)
    assert np.array_equal(oracle.bfs_levels(n, g.row_ptr, g.col_idx, 0), np.minimum(i, n - i))


def test_full_grid_corner_closed_form():
    w, h = 9, 6
    edges = []
    for y in range(h):
        for x in range(w):
            if x + 1 < w:
                edges.append((y * w + x, y * w + x + 1))
            if y + 1 < h:
                edges.append((y * w + x, (y + 1) * w + x))
    g = csr_from_undirected(w * h, edges)
    lvl = oracle.bfs_levels(w * h, g.row_ptr, g.col_idx, 0)
    ys, xs = np.divmod(np.arange(w * h), w)
    assert np.array_equal(lvl, xs + ys)


def test_complete_graph_and_components():
    n = 12
    edges = [(i, j) for i in range(6) for j in range(i + 1, 6)]        # K6 on 0..5
    edges += [(6 + i, 6 + (i + 1) % 6) for i in range(6)]               # C6 on 6..11
    g = csr_from_undirected(n, edges)
    lvl = oracle.bfs_levels(n, g.row_ptr, g.col_idx, 2)
    assert lvl[2] == 0 and np.all(np.delete(lvl[:6], 2) == 1) and np.all(lvl[6:] == -1)


def test_isolated_source_and_single_vertex():
    g = csr_from_undirected(5, [(1, 2)])
    lvl = oracle.bfs_levels(5, g.row_ptr, g.col_idx, 4)
    assert lvl.tolist() == [-1, -1, -1, -1, 0]
    g1 = csr_from_undirected(1, [])
    assert oracle.bfs_levels(1, g1.row_ptr, g1.col_idx, 0).tolist() == [0]


def test_source_out_of_range():
    g = csr_from_undirected(3, [(0, 1)])
    with pytest.raises(ValueError):
        oracle.bfs_levels(3, g.row_ptr, g.col_idx, 3)


def test_rmat_invariants_and_library():
    g = synth.rmat_graph(12, 16, seed=5)
    srcs = synth.pick_sources(g, 4, seed=9)
    for s in srcs:
        lvl = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(s))
        check_invariants(g, int(s), lvl)
    sp = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as ss
    A = ss.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    d = sp.shortest_path(A, unweighted=True, indices=[int(srcs[0])])[0]
    exp = np.where(np.isinf(d), -1, d).astype(np.int32)
    assert np.array_equal(oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(srcs[0])), exp)


def test_msbfs_is_k_single_runs():
    g = synth.rmat_graph(10, 16, seed=2)
    srcs = synth.pick_sources(g, 7, seed=3)
    many = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs, threads=3)
    for i, s in enumerate(srcs):
        assert np.array_equal(many[i], oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(s)))


def test_planted_mistake_is_caught():
    """A plausible bug (levels off by one past the first ring) must fail the
    brute-force comparison: the pin is not vacuous."""
    n = 10
    g = csr_from_undirected(n, [(i, i + 1) for i in range(n - 1)])
    lvl = oracle.bfs_levels(n, g.row_ptr, g.col_idx, 0).copy()
    lvl[lvl >= 2] += 1
    assert not np.array_equal(lvl, brute_force_levels(n, g, 0))
    with pytest.raises(AssertionError):
        check_invariants(g, 0, lvl)


def check_tree(g, src, lvl, par):
    """par is a BFS tree of lvl: the source is its own parent, every reached
    vertex's parent is a neighbour one level closer, unreached ones have -1,
    and following parents from any vertex ends at the source."""
    nbr = [set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    assert par[src] == src
    for v in range(g.n):
        if lvl[v] < 0:
            assert par[v] == -1
        elif v != src:
            assert int(par[v]) in nbr[v] and lvl[par[v]] == lvl[v] - 1
            assert par[v] == min(c for c in nbr[v] if lvl[c] == lvl[v] - 1)   # the unique choice
    for v in range(g.n):
        x, steps = v, 0
        while lvl[x] > 0 and steps <= g.n:
            x, steps = int(par[x]), steps + 1
        assert lvl[v] < 0 or x == src


@pytest.mark.parametrize("seed", range(5))
def test_parents_form_the_min_id_bfs_tree(seed):
    g = synth.rmat_graph(7, 8, seed=seed)
    src = int(synth.pick_sources(g, 1, seed)[0])
    lvl, par = oracle.bfs_parents(g.n, g.row_ptr, g.col_idx, src)
    assert np.array_equal(lvl, brute_force_levels(g.n, g, src))
    check_tree(g, src, lvl, par)


def test_parents_path_closed_form():
    n = 12
    g = csr_from_undirected(n, [(i, i + 1) for i in range(n - 1)])
    _, par = oracle.bfs_parents(n, g.row_ptr, g.col_idx, 5)
    assert par.tolist() == [1, 2, 3, 4, 5, 5, 5, 6, 7, 8, 9, 10]


def test_planted_parent_mistake_is_caught():
    g = synth.rmat_graph(6, 8, seed=3)
    src = int(synth.pick_sources(g, 1, 1)[0])
    lvl, par = oracle.bfs_parents(g.n, g.row_ptr, g.col_idx, src)
    bad = par.copy()
    v = int(np.nonzero(lvl >= 2)[0][0])
    bad[v] = src if src not in g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]] else -1
    with pytest.raises(AssertionError):
        check_tree(g, src, lvl, bad)


def test_distance_stats_closed_forms():
    """Path from an end: sum n(n-1)/2, eccentricity n-1; star centre: n-1 and 1;
    full w x h grid from a corner: sum of x + y, eccentricity w + h - 2; a
    vertex of a K6 + C6 graph reaches only its own component."""
    n = 23
    g = csr_from_undirected(n, [(i, i + 1) for i in range(n - 1)])
    r, t, e = oracle.distance_stats(n, g.row_ptr, g.col_idx, [0, 11])
    assert r.tolist() == [n, n] and t[0] == n * (n - 1) // 2 and e.tolist() == [n - 1, 11]
    assert t[1] == 2 * sum(range(1, 12)) and (n - 1) / t[0] == 2 / n          # closeness of an end
    s = csr_from_undirected(9, [(0, i) for i in range(1, 9)])
    r, t, e = oracle.distance_stats(9, s.row_ptr, s.col_idx, [0, 3])
    assert r.tolist() == [9, 9] and t.tolist() == [8, 1 + 2 * 7] and e.tolist() == [1, 2]
    w, h = 7, 5
    edges = [(y * w + x, y * w + x + 1) for y in range(h) for x in range(w - 1)]
    edges += [(y * w + x, (y + 1) * w + x) for y in range(h - 1) for x in range(w)]
    gg = csr_from_undirected(w * h, edges)
    r, t, e = oracle.distance_stats(w * h, gg.row_ptr, gg.col_idx, [0])
    assert t[0] == h * w * (w - 1) // 2 + w * h * (h - 1) // 2 and e[0] == w + h - 2
    edges = [(i, j) for i in range(6) for j in range(i + 1, 6)] + [(6 + i, 6 + (i + 1) % 6) for i in range(6)]
    kc = csr_from_undirected(13, edges)
    r, t, e = oracle.distance_stats(13, kc.row_ptr, kc.col_idx, [2, 7, 12])
    assert r.tolist() == [6, 6, 1] and t.tolist() == [5, 1 + 1 + 2 + 2 + 3, 0] and e.tolist() == [1, 3, 0]


def test_distance_stats_planted_mistake():
    """Counting the source's own level once more per neighbour ring (an
    off-by-one in the sum) must break the path closed form."""
    n = 10
    g = csr_from_undirected(n, [(i, i + 1) for i in range(n - 1)])
    lv = oracle.bfs_levels(n, g.row_ptr, g.col_idx, 0)
    bad = int((lv[lv >= 0] + 1).sum())
    assert bad != oracle.distance_stats(n, g.row_ptr, g.col_idx, [0])[1][0]
