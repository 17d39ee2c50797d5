"""The C-ABI library without a GPU: it loads, exports every symbol declared in
include/blest.h, and its host-only entry points (input checks, the two vertex
orderings, the social-like classifier) agree with the oracle."""
import os
import re

import numpy as np
import pytest

import paper_2512_21967_gb300 as blest
from oracle import orderings as oo
from paper_2512_21967_gb300 import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "blest.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(blest_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = blest.lib()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), f"{name} declared in blest.h but not exported"
    assert sorted(blest.EXPORTED_SYMBOLS) == names


def csr(n, edges):
    src = np.array([e[0] for e in edges], np.int32)
    dst = np.array([e[1] for e in edges], np.int32)
    return synth.csr_from_edges(n, src, dst)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rcm_matches_oracle(seed):
    g, _ = synth.grid_graph(14 + seed, p=0.85, seed=seed)
    got = blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_BANDWIDTH)
    assert np.array_equal(got, oo.rcm(g.n, g.row_ptr, g.col_idx))


def test_rcm_matches_oracle_rmat_with_isolated():
    g = synth.rmat_graph(9, 4, seed=8)
    got = blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_BANDWIDTH)
    assert np.array_equal(got, oo.rcm(g.n, g.row_ptr, g.col_idx))


# windows up to 65536 store window positions in 16 bits, wider ones in 32 (the last case)
@pytest.mark.parametrize("scale,w", [(8, 16), (9, 64), (10, 1024), (9, 131072)])
def test_compress_order_matches_oracle(scale, w):
    g = synth.rmat_graph(scale, 16, seed=scale)
    got = blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS, window=w, threads=3)
    assert np.array_equal(got, oo.compress_order(g.n, g.row_ptr, g.col_idx, sigma=8, w=w))


def test_compress_order_ragged_last_window():
    g = synth.rmat_graph(7, 8, seed=4)
    # n = 128, w = 48: windows of 48, 48, 32
    got = blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS, window=48)
    assert np.array_equal(got, oo.compress_order(g.n, g.row_ptr, g.col_idx, sigma=8, w=48))


def test_none_order_is_identity_and_auto_classifies():
    g = synth.rmat_graph(10, 16, seed=1)
    assert np.array_equal(blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE),
                          np.arange(g.n))
    gg, _ = synth.grid_graph(40, 0.9, seed=2)
    for graph, social in ((g, True), (gg, False)):
        assert blest.blest_is_social(graph.n, graph.row_ptr, graph.col_idx) == social
        assert oo.is_social_like(graph.n, graph.row_ptr, graph.col_idx) == social
    auto = blest.blest_compute_order(gg.n, gg.row_ptr, gg.col_idx, blest.BLEST_ORDER_AUTO)
    assert np.array_equal(auto, oo.rcm(gg.n, gg.row_ptr, gg.col_idx))


def test_classifier_agrees_with_oracle_on_mixed_graphs():
    for seed in range(4):
        g = synth.rmat_graph(9, 2 + 4 * seed, seed=seed)
        assert blest.blest_is_social(g.n, g.row_ptr, g.col_idx) == oo.is_social_like(g.n, g.row_ptr, g.col_idx)
    path = csr(50, [(i, i + 1) for i in range(49)])
    assert not blest.blest_is_social(path.n, path.row_ptr, path.col_idx)


def test_unsorted_rows_duplicates_and_loops_are_cleaned():
    g = synth.rmat_graph(8, 8, seed=3)
    rng = np.random.default_rng(0)
    rows = []
    for u in range(g.n):
        r = list(g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]])
        r += r[:1] + [u]            # a duplicate and a self-loop
        rng.shuffle(r)
        rows.append(r)
    rp = np.zeros(g.n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([x for r in rows for x in r], np.int32)
    a = blest.blest_compute_order(g.n, rp, ci, blest.BLEST_ORDER_BANDWIDTH)
    assert np.array_equal(a, oo.rcm(g.n, g.row_ptr, g.col_idx))


def test_input_errors():
    g = csr(4, [(0, 1), (1, 2)])
    with pytest.raises(blest.BlestError) as e:
        blest.blest_compute_order(4, g.row_ptr, np.array([0, 1, 1, 9], np.int32), blest.BLEST_ORDER_NONE)
    assert e.value.name == "BLEST_ERR_INVALID_ARG"
    asym_rp = np.array([0, 1, 1, 1, 1], np.int32)
    with pytest.raises(blest.BlestError) as e:
        blest.blest_compute_order(4, asym_rp, np.array([2], np.int32), blest.BLEST_ORDER_NONE)
    assert e.value.name == "BLEST_ERR_NOT_SYMMETRIC"
    with pytest.raises(blest.BlestError) as e:
        blest.blest_compute_order(4, np.array([0, 2, 1, 2, 2], np.int32), g.col_idx, blest.BLEST_ORDER_NONE)
    assert e.value.name == "BLEST_ERR_INVALID_ARG"
    with pytest.raises(blest.BlestError) as e:
        blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, 7)
    assert e.value.name == "BLEST_ERR_INVALID_ARG"
    with pytest.raises(blest.BlestError):
        blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS, window=12)
    # n = 0 is a valid, empty graph
    assert blest.blest_compute_order(0, np.zeros(1, np.int32), np.zeros(0, np.int32), blest.BLEST_ORDER_AUTO).size == 0


def test_null_handle_calls_fail_cleanly():
    lib = blest.lib()
    assert lib.blest_bfs(None, 0, None) == 1
    assert lib.blest_sync(None) == 1
    lib.blest_destroy(None)
    assert blest.blest_export_size(None, 0) == -1


def test_graph_load_rejects_bad_files(tmp_path):
    """A checkpoint is untrusted input: wrong magic, a truncated file and an
    out-of-range row id are refused on the host, before any device work."""
    p = tmp_path / "bad.blest"
    p.write_bytes(b"NOTBLEST" + bytes(200))
    with pytest.raises(blest.BlestError) as e:
        blest.blest_graph_load(str(p))
    assert e.value.status == blest.BLEST_ERR_INVALID_ARG
    with pytest.raises(blest.BlestError):
        blest.blest_graph_load(str(tmp_path / "missing.blest"))
    # a valid-looking header for n = 16 with one VSS, then a truncated body
    import struct
    hdr = b"BLESTG1\x00" + struct.pack("<iiqiiqqq", 1, 16, 4, 2, 0, 1, 2, 0)
    p.write_bytes(hdr + bytes(16))
    with pytest.raises(blest.BlestError) as e:
        blest.blest_graph_load(str(p))
    assert "shorter" in str(e.value)


@pytest.mark.parametrize("scale,seed", [(7, 1), (8, 3), (9, 5)])
def test_gorder_prepass_matches_oracle(scale, seed):
    """The compression ordering with the Gorder pre-pass (C++) equals the
    oracle's, vertex for vertex (the R-MAT scale-9 graph has hubs above the
    degree cap of 64)."""
    g = synth.rmat_graph(scale, 8, seed=seed)
    got = blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS, window=64,
                                    prepass="gorder")
    exp = oo.compress_order(g.n, g.row_ptr, g.col_idx, 8, 64, prepass="gorder")
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("order", ["compress", "bandwidth"])
def test_orders_do_not_depend_on_host_threads(order):
    """Scale 19 has BFS levels above both parallel thresholds (1024 vertices in the
    pseudo-peripheral search, 65536 in the order-preserving expansion)."""
    g = synth.rmat_graph(19, 16, seed=12)
    o = blest.BLEST_ORDER_COMPRESS if order == "compress" else blest.BLEST_ORDER_BANDWIDTH
    one = blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, o, window=4096, threads=1)
    many = blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, o, window=4096, threads=6)
    assert np.array_equal(one, many)
    assert np.array_equal(np.sort(one), np.arange(g.n))


@pytest.mark.parametrize("threads", [1, 4])
def test_batch_create_reports_the_first_bad_graph(threads):
    """Batch graphs are prepared concurrently; the lowest-numbered invalid graph is
    the one reported, whatever the thread count (this fails before any GPU call)."""
    graphs = [synth.rmat_graph(8, 8, seed=40 + i) for i in range(12)]
    items = [(g.n, g.row_ptr, g.col_idx) for g in graphs]
    for b in (9, 5):   # an out-of-range column in graphs 9 and 5
        ci = graphs[b].col_idx.copy()
        ci[0] = graphs[b].n + 3
        items[b] = (graphs[b].n, graphs[b].row_ptr, ci)
    with pytest.raises(blest.BlestError) as e:
        blest.blest_batch_create(items, [blest.BLEST_ORDER_COMPRESS] * 6 + [blest.BLEST_ORDER_BANDWIDTH] * 6,
                                 threads=threads)
    assert e.value.name == "BLEST_ERR_INVALID_ARG"
    assert "graph 5:" in str(e.value) and "graph 9:" not in str(e.value)


def test_batch_preparation_runs_to_the_device_step():
    """Every graph of a valid batch is cleaned, reordered and relabelled on 4
    threads; without a GPU creation then stops at the first device call, with a
    GPU it returns a handle."""
    graphs = [synth.rmat_graph(9, 8, seed=60 + i) for i in range(6)] + \
             [synth.grid_graph(24 + i, 0.9, seed=70 + i)[0] for i in range(6)]
    items = [(g.n, g.row_ptr, g.col_idx) for g in graphs]
    orders = [blest.BLEST_ORDER_COMPRESS] * 6 + [blest.BLEST_ORDER_BANDWIDTH] * 6
    try:
        h = blest.blest_batch_create(items, orders, threads=4)
    except blest.BlestError as e:
        assert e.name == "BLEST_ERR_CUDA", str(e)
    else:
        blest.blest_destroy(h)


def _drop_entries(g, drops):
    """g's CSR without the entries (row, col) in drops."""
    drops = set(drops)
    rows = [[int(x) for x in g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]] if (u, int(x)) not in drops]
            for u in range(g.n)]
    rp = np.zeros(g.n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    return rp, np.array([x for r in rows for x in r], np.int32)


@pytest.mark.parametrize("threads", [1, 4])
def test_symmetry_check_in_long_rows(threads):
    """Rows of 256 entries or more are searched with a forward-only cursor per
    chunk of rows; a reverse missing there, alone or several in one row, in
    either direction, must be reported with an edge whose reverse is absent."""
    from paper_2512_21967_gb300 import synth
    g = synth.rmat_graph(12, 16, seed=3)
    deg = np.diff(g.row_ptr)
    hubs = np.flatnonzero(deg >= 256)
    assert len(hubs) >= 3
    blest.blest_compute_order(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE, threads=threads)   # symmetric
    rng = np.random.default_rng(11)
    edges = {(u, int(x)) for u in range(g.n) for x in g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]}
    for trial in range(12):
        v = int(rng.choice(hubs))
        row = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
        below = row[row < v]
        us = [int(x) for x in rng.choice(below, size=min(len(below), 1 + trial % 3), replace=False)]
        # trial even: drop (v, u) from the long row v, so the upper edges (u, v) lose their
        # reverses; odd: drop (u, v) from the rows u, so the lower edges (v, u) of row v do
        drops = [(v, u) for u in us] if trial % 2 == 0 else [(u, v) for u in us]
        rp, ci = _drop_entries(g, drops)
        with pytest.raises(blest.BlestError) as e:
            blest.blest_compute_order(g.n, rp, ci, blest.BLEST_ORDER_NONE, threads=threads)
        assert e.value.name == "BLEST_ERR_NOT_SYMMETRIC"
        a, b = (int(t) for t in str(e.value).split("edge (")[1].split(")")[0].split(", "))
        kept = edges - set(drops)
        assert (a, b) in kept and (b, a) not in kept, (drops, (a, b))
