"""GPU parity of the BLEST kernels against the oracle, through the C ABI.
Levels and BVSS arrays are integer results: every comparison is bit-exact."""
import numpy as np
import pytest

import oracle
import paper_2512_21967_gb300 as blest
from oracle import bvss as ob
from oracle import model as om
from oracle import orderings as oo
from paper_2512_21967_gb300 import synth

from gpu_helpers import ORDERS, assert_bvss_equal, check_levels, csr, export_bvss, oracle_bvss, oracle_order

pytestmark = pytest.mark.gpu

MODES = [(u, p) for u in (blest.BLEST_UPDATE_EAGER, blest.BLEST_UPDATE_LAZY)
         for p in (blest.BLEST_PULL_POPC, blest.BLEST_PULL_MMA)]


@pytest.fixture(scope="module")
def torch_cuda(gpu):
    import torch
    torch.cuda.init()
    return torch


# ------------------------------------------------------------ pull tiles

@pytest.mark.parametrize("pull", [blest.BLEST_PULL_POPC, blest.BLEST_PULL_MMA])
def test_pull_tile_exhaustive(torch_cuda, pull):
    """Every (8-bit mask, alpha) pair in every one of the 4 sub-slots (Figure 2c's
    fragment contract): hit iff popc(mask & alpha) > 0 (Eq. 1)."""
    torch = torch_cuda
    alphas = np.repeat(np.arange(256, dtype=np.uint8), 8)          # 8 tiles per alpha
    tiles = len(alphas)
    j = np.tile(np.arange(8), 256)[:, None, None]
    lane = np.arange(32)[None, :, None]
    q = np.arange(4)[None, None, :]
    byte = (j * 32 + lane + 64 * q) % 256                           # all 256 values per sub-slot
    masks = (byte.astype(np.uint32) << (8 * q).astype(np.uint32)).sum(axis=2).astype(np.uint32)
    exp = np.zeros((tiles, 32), np.uint8)
    for qq in range(4):
        hit = (byte[:, :, qq] & alphas[:, None]) != 0
        exp |= (hit.astype(np.uint8) << qq)
    d_m = torch.from_numpy(masks.view(np.int32).reshape(-1)).cuda()
    d_a = torch.from_numpy(alphas).cuda()
    d_h = torch.zeros(tiles * 32, dtype=torch.uint8, device="cuda")
    blest.blest_debug_pull(d_m, d_a, tiles, pull, d_h)
    assert np.array_equal(d_h.cpu().numpy().reshape(tiles, 32), exp)


# ------------------------------------------------------------- BVSS build

@pytest.mark.parametrize("order", ["none", "bandwidth", "compress"])
@pytest.mark.parametrize("scale", [7, 10])
def test_bvss_build_matches_oracle(gpu, order, scale):
    g = synth.rmat_graph(scale, 16, seed=scale + 1)
    o = ORDERS[order]
    h = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, o, window=256)
    try:
        got = export_bvss(h)
        ref_id = oracle_order(g, o, window=256)
        assert np.array_equal(got["new_id"], ref_id)
        assert_bvss_equal(got, oracle_bvss(g, ref_id))
        st = blest.blest_get_stats(h)
        b = oracle_bvss(g, ref_id)
        assert st["unpadded_slices"] == ob.unpadded_slices(b)
        assert abs(st["compression_ratio"] - om.compression_ratio(g.nnz, ob.unpadded_slices(b))) < 1e-12
        assert abs(st["update_divergence"] - om.update_divergence(b)) <= 1e-9 * max(1.0, om.update_divergence(b))
    finally:
        blest.blest_destroy(h)


def test_bvss_build_edge_shapes(gpu):
    from test_oracle_bvss import fig1_graph
    cases = [fig1_graph(),
             csr(45, [(0, 44), (1, 2), (30, 31), (44, 3), (20, 21)]),          # ragged n, empty slice set
             csr(300, [(0, i) for i in range(1, 300)]),                          # hub: 3 VSSs in slice set 0
             csr(1, []), csr(9, [])]
    for g in cases:
        h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE)
        try:
            assert_bvss_equal(export_bvss(h), ob.build(g.n, g.row_ptr, g.col_idx))
        finally:
            blest.blest_destroy(h)


# ------------------------------------------------------------- traversals

@pytest.fixture(scope="module")
def cfg1(gpu):
    """R-MAT scale 16, edgefactor 16, 64 seeded degree>0 sources."""
    g, srcs = synth.rmat_workload(16, 64, seed_graph=1, seed_src=1001)
    exp = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs, threads=8)
    return g, srcs, exp


@pytest.mark.parametrize("order", ["none", "compress", "bandwidth"])
def test_rmat16_all_sources_all_modes(cfg1, order):
    g, srcs, exp = cfg1
    h = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, ORDERS[order], window=4096)
    try:
        for upd, pull in MODES:
            blest.blest_set_option(h, blest.BLEST_OPT_UPDATE, upd)
            blest.blest_set_option(h, blest.BLEST_OPT_PULL, pull)
            variants = [(2, 2, 1, 0, 0, 0), (1, 3, 0, 0, 0, 0), (2, 3, 1, 0, 0, 0), (1, 2, 0, 0, 0, 0)]
            if upd == blest.BLEST_UPDATE_LAZY:
                variants += [(1, 2, 1, 4, 0, 0), (1, 2, 0, 8, 0, 0), (1, 2, 1, 8, 0, 0), (2, 2, 2, 0, 0, 0),
                             (1, 3, 2, 0, 0, 0), (1, 2, 1, 2, 0, 0), (2, 2, 2, 2, 0, 0), (2, 2, 0, 2, 0, 0),
                             (2, 2, 2, 8, 0, 0), (1, 2, 1, 0, 1, 0), (2, 2, 2, 0, 1, 0), (1, 2, 0, 2, 1, 0),
                             (2, 2, 2, 2, 1, 0), (2, 2, 2, 2, 0, 1), (1, 2, 1, 2, 0, 1), (2, 2, 2, 2, 1, 1),
                             (2, 2, 2, 3, 0, 0), (1, 2, 1, 3, 0, 1), (2, 2, 2, 3, 0, 1),
                             (2, 2, 3, 2, 0, 1), (1, 2, 3, 0, 0, 0), (2, 2, 3, 8, 0, 0), (2, 2, 3, 2, 1, 1),
                             (2, 2, 4, 2, 0, 1), (1, 2, 4, 0, 0, 0), (2, 2, 4, 2, 1, 0), (2, 3, 4, 0, 0, 0)]
            for unroll, minb, filt, depth, layout, sched in variants:
                blest.blest_set_option(h, blest.BLEST_OPT_SCHEDULE, sched)
                blest.blest_set_option(h, blest.BLEST_OPT_UNROLL, unroll)
                blest.blest_set_option(h, blest.BLEST_OPT_MIN_BLOCKS, minb)
                blest.blest_set_option(h, blest.BLEST_OPT_VISITED_FILTER, filt)
                blest.blest_set_option(h, blest.BLEST_OPT_STAGE_DEPTH, depth)
                blest.blest_set_option(h, blest.BLEST_OPT_LAYOUT, layout)
                for i, s in enumerate(srcs):
                    got = blest.blest_bfs(h, int(s))
                    assert np.array_equal(got, exp[i]), f"mode {(upd, pull, unroll, minb, filt, depth, layout, sched)} source {s}"
    finally:
        blest.blest_destroy(h)


def test_queue_sizes_match_replay(cfg1):
    """Per-level VSS counts equal the oracle replay: only slice sets with a
    column in the previous frontier are processed (Section 3.1.1), once each."""
    g, srcs, exp = cfg1
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE)
    try:
        b = ob.build(g.n, g.row_ptr, g.col_idx)
        blest.blest_set_option(h, blest.BLEST_OPT_RECORD_LEVELS, 1)
        for upd, depth, layout, sched in ((blest.BLEST_UPDATE_EAGER, 0, 0, 0), (blest.BLEST_UPDATE_LAZY, 0, 0, 0),
                                          (blest.BLEST_UPDATE_LAZY, 8, 0, 0), (blest.BLEST_UPDATE_LAZY, 2, 0, 0),
                                          (blest.BLEST_UPDATE_LAZY, 2, 1, 0), (blest.BLEST_UPDATE_LAZY, 0, 1, 0),
                                          (blest.BLEST_UPDATE_LAZY, 2, 0, 1), (blest.BLEST_UPDATE_LAZY, 2, 1, 1),
                                          (blest.BLEST_UPDATE_LAZY, 3, 0, 1)):
            blest.blest_set_option(h, blest.BLEST_OPT_UPDATE, upd)
            blest.blest_set_option(h, blest.BLEST_OPT_SCHEDULE, sched)
            blest.blest_set_option(h, blest.BLEST_OPT_STAGE_DEPTH, depth)
            blest.blest_set_option(h, blest.BLEST_OPT_LAYOUT, layout)
            for i in range(4):
                blest.blest_bfs(h, int(srcs[i]))
                info, sizes = blest.blest_get_run_info(h, 4096)
                ref = om.queue_sizes(b, exp[i])
                assert info["levels"] == len(ref)
                assert sizes.tolist() == ref
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("upd", [blest.BLEST_UPDATE_EAGER, blest.BLEST_UPDATE_LAZY])
def test_grid_high_diameter(gpu, upd):
    g, srcs = synth.grid_workload(192, 6, seed_graph=3, seed_src=1003)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_BANDWIDTH)
    try:
        blest.blest_set_option(h, blest.BLEST_OPT_UPDATE, upd)
        check_levels(g, h, srcs)
    finally:
        blest.blest_destroy(h)


def test_small_graphs_closed_forms(gpu):
    cases = []
    n = 77
    cases.append((csr(n, [(i, i + 1) for i in range(n - 1)]), [0, 38, 76]))                 # path: |i - c|
    cases.append((csr(40, [(0, i) for i in range(1, 40)]), [0, 13]))                        # star
    cases.append((csr(33, [(i, (i + 1) % 33) for i in range(33)]), [5]))                    # cycle
    cases.append((csr(12, [(i, j) for i in range(6) for j in range(i + 1, 6)]), [1, 9]))    # K6 + isolated
    cases.append((csr(1, []), [0]))                                                          # single vertex
    cases.append((csr(50, [(1, 2)]), [49, 1]))                                               # isolated source
    for g, srcs in cases:
        for order in ORDERS.values():
            h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, order)
            try:
                for upd, pull in MODES:
                    blest.blest_set_option(h, blest.BLEST_OPT_UPDATE, upd)
                    blest.blest_set_option(h, blest.BLEST_OPT_PULL, pull)
                    check_levels(g, h, srcs)
            finally:
                blest.blest_destroy(h)


def test_invalid_sources_and_empty_graph(gpu):
    g = csr(10, [(0, 1)])
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE)
    try:
        for bad in (-1, 10):
            with pytest.raises(blest.BlestError) as e:
                blest.blest_bfs(h, bad)
            assert e.value.name == "BLEST_ERR_INVALID_ARG"
        with pytest.raises(blest.BlestError):
            blest.blest_msbfs(h, [0, 11])
        assert blest.blest_bfs(h, 0)[1] == 1          # handle still usable
    finally:
        blest.blest_destroy(h)
    h0 = blest.blest_graph_create(0, np.zeros(1, np.int32), np.zeros(0, np.int32), blest.BLEST_ORDER_NONE)
    try:
        with pytest.raises(blest.BlestError):
            blest.blest_bfs(h0, 0)
        assert blest.blest_msbfs(h0, []).size == 0
    finally:
        blest.blest_destroy(h0)


def test_barrier_timeout_is_reported_and_recoverable(gpu):
    """A barrier that waits for a block that does not exist gives up after the
    configured limit with BLEST_ERR_TIMEOUT; the handle keeps working."""
    g = synth.rmat_graph(10, 16, seed=3)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE)
    try:
        blest.blest_set_option(h, blest.BLEST_OPT_BARRIER_TIMEOUT_US, 20000)
        blest.blest_set_option(h, blest.BLEST_OPT_TEST_PHANTOM_BLOCK, 1)
        with pytest.raises(blest.BlestError) as e:
            blest.blest_bfs(h, 0)
        assert e.value.name == "BLEST_ERR_TIMEOUT"
        with pytest.raises(blest.BlestError) as e:
            blest.blest_msbfs(h, [0, 1])
        assert e.value.name == "BLEST_ERR_TIMEOUT"
        blest.blest_set_option(h, blest.BLEST_OPT_TEST_PHANTOM_BLOCK, 0)
        blest.blest_set_option(h, blest.BLEST_OPT_BARRIER_TIMEOUT_US, 2000000)
        assert np.array_equal(blest.blest_bfs(h, 0), oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, 0))
    finally:
        blest.blest_destroy(h)


# ---------------------------------------------------------- multi-source

@pytest.mark.parametrize("k", [1, 7, 64, 65, 130, 256, 300])
def test_msbfs_matches_k_oracle_runs(gpu, k):
    g = synth.rmat_graph(12, 16, seed=5)
    srcs = synth.pick_sources(g, k, seed=77)
    srcs[-1] = srcs[0]                                   # a duplicate source
    exp = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs, threads=8)
    for order in (blest.BLEST_ORDER_NONE, blest.BLEST_ORDER_COMPRESS):
        h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, order)
        try:
            assert np.array_equal(blest.blest_msbfs(h, srcs), exp)
        finally:
            blest.blest_destroy(h)


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("pull", [blest.BLEST_PULL_POPC, blest.BLEST_PULL_MMA])
@pytest.mark.parametrize("chunk", [64, 128, 256])
def test_msbfs_pull_backends_and_launch_sizes(gpu, pull, chunk, levels):
    """Both multi-source pull back-ends (CUDA-core OR, b1 tensor-core MMA), both
    level layouts (vertex-major, bit planes) and every launch size give the
    oracle's levels, for source counts across word and launch boundaries, on a
    power-law graph and on a ragged grid."""
    g = synth.rmat_graph(11, 16, seed=5)
    gg, _ = synth.grid_graph(37, 0.9, seed=6)
    for graph, order in ((g, blest.BLEST_ORDER_COMPRESS), (gg, blest.BLEST_ORDER_BANDWIDTH)):
        h = blest.blest_graph_create(graph.n, graph.row_ptr, graph.col_idx, order)
        try:
            blest.blest_set_option(h, blest.BLEST_OPT_MS_PULL, pull)
            blest.blest_set_option(h, blest.BLEST_OPT_MS_CHUNK, chunk)
            blest.blest_set_option(h, blest.BLEST_OPT_MS_LEVELS, levels)
            for k in (3, 64, 65, 130, 300):
                srcs = synth.pick_sources(graph, k, seed=31 + k)
                exp = oracle.msbfs_levels(graph.n, graph.row_ptr, graph.col_idx, srcs, threads=8)
                for filt in (1, 2, 0):
                    blest.blest_set_option(h, blest.BLEST_OPT_MS_VISITED_FILTER, filt)
                    assert np.array_equal(blest.blest_msbfs(h, srcs), exp), (k, pull, chunk, filt)
        finally:
            blest.blest_destroy(h)


def test_msbfs_autotune_keeps_levels_exact(gpu):
    g = synth.rmat_graph(12, 16, seed=9)
    srcs = synth.pick_sources(g, 150, seed=3)
    exp = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs, threads=8)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS)
    try:
        r = blest.blest_autotune_msbfs(h, srcs)
        # CUDA-core pull: 3 launch sizes x 3 grid sizes x 2 level layouts x 3 visited tests;
        # MMA: bit planes with the V_curr test only
        assert r["candidates"] == 3 * 3 * 2 * 3 + 3 * 3
        assert r["levels"] in (1, 2)
        assert r["popc_ms"] > 0 and r["mma_ms"] > 0 and r["best_ms"] == min(r["popc_ms"], r["mma_ms"])
        assert r["chunk"] in (64, 128, 256) and r["pull"] in (blest.BLEST_PULL_POPC, blest.BLEST_PULL_MMA)
        assert np.array_equal(blest.blest_msbfs(h, srcs), exp)
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("levels", [1, 2])
def test_msbfs_more_than_256_levels(gpu, levels):
    """A long thin grid: levels above 255 take the 16-plane path of the bit-plane
    output (and the vertex-major layout stores them as they are)."""
    rows, cols = 3, 400
    edges = [(r * cols + c, r * cols + c + 1) for r in range(rows) for c in range(cols - 1)]
    edges += [(r * cols + c, (r + 1) * cols + c) for r in range(rows - 1) for c in range(cols)]
    src, dst = np.array(edges, np.int32).T
    g = synth.csr_from_edges(rows * cols, src, dst)
    srcs = np.array([0, cols - 1, rows * cols - 1, 600, 5], np.int32)
    exp = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs)
    assert exp.max() > 300
    for order in (blest.BLEST_ORDER_NONE, blest.BLEST_ORDER_BANDWIDTH):
        h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, order)
        try:
            blest.blest_set_option(h, blest.BLEST_OPT_MS_LEVELS, levels)
            assert np.array_equal(blest.blest_msbfs(h, srcs), exp)
        finally:
            blest.blest_destroy(h)


def test_msbfs_grid_and_isolated(gpu):
    g, srcs = synth.grid_workload(96, 20, seed_graph=4, seed_src=9)
    srcs = np.concatenate([srcs, [int(np.argmin(g.degrees()))]]).astype(np.int32)
    exp = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs, threads=8)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_BANDWIDTH)
    try:
        assert np.array_equal(blest.blest_msbfs(h, srcs), exp)
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("k", [5, 70, 200])
def test_msbfs_ragged_vertex_count(gpu, k):
    """n = 37^2 = 1369 is not a multiple of the 32 vertices a warp transposes at a
    time, and the three k give row strides 8, 72 and 200 (1, 2 and 4 words)."""
    g, _ = synth.grid_graph(37, 0.9, seed=6)
    assert g.n % 32 != 0
    srcs = synth.pick_sources(g, k, seed=21)
    exp = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs, threads=8)
    for order in (blest.BLEST_ORDER_NONE, blest.BLEST_ORDER_BANDWIDTH):
        h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, order)
        try:
            assert np.array_equal(blest.blest_msbfs(h, srcs), exp)
        finally:
            blest.blest_destroy(h)


def min_over_sources(g, srcs):
    per = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs, threads=8).astype(np.int64)
    per = np.where(per < 0, np.iinfo(np.int64).max, per).min(axis=0)
    return np.where(per == np.iinfo(np.int64).max, -1, per).astype(np.int32)


def test_multiroot_is_min_over_sources(gpu):
    g = synth.rmat_graph(11, 8, seed=6)
    srcs = synth.pick_sources(g, 40, seed=3)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS)
    try:
        for upd in (blest.BLEST_UPDATE_EAGER, blest.BLEST_UPDATE_LAZY):
            blest.blest_set_option(h, blest.BLEST_OPT_UPDATE, upd)
            assert np.array_equal(blest.blest_bfs_multiroot(h, srcs), min_over_sources(g, srcs))
            assert np.array_equal(blest.blest_bfs_multiroot(h, srcs[:3]), min_over_sources(g, srcs[:3]))
    finally:
        blest.blest_destroy(h)


def test_batch_of_uneven_graphs(gpu):
    rng = np.random.default_rng(5)
    graphs, srcs, orders = [], [], []
    for i in range(12):
        if i % 2 == 0:
            g = synth.rmat_graph(int(rng.integers(6, 12)), 16, seed=100 + i)
            orders.append(blest.BLEST_ORDER_COMPRESS)
        else:
            g, _ = synth.grid_graph(int(rng.integers(8, 60)), 0.9, seed=200 + i)
            orders.append(blest.BLEST_ORDER_BANDWIDTH)
        graphs.append(g)
        srcs.append(int(synth.pick_sources(g, 1, seed=300 + i)[0]))
    h = blest.blest_batch_create([(g.n, g.row_ptr, g.col_idx) for g in graphs], orders)
    try:
        for upd in (blest.BLEST_UPDATE_EAGER, blest.BLEST_UPDATE_LAZY):
            blest.blest_set_option(h, blest.BLEST_OPT_UPDATE, upd)
            got = blest.blest_batch_bfs(h, srcs)
            off = 0
            for g, s in zip(graphs, srcs):
                assert np.array_equal(got[off:off + g.n], oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, s))
                off += g.n
    finally:
        blest.blest_destroy(h)


def test_batch_multiroot_autotune_keeps_levels_exact(gpu):
    """The multi-root autotuner times variants of the batch's own launch (all
    graphs' roots at once) and the kept variant gives every graph its levels."""
    graphs, srcs, orders = [], [], []
    for i in range(10):
        if i % 2 == 0:
            g = synth.rmat_graph(8 + i % 4, 16, seed=600 + i)
            orders.append(blest.BLEST_ORDER_COMPRESS)
        else:
            g, _ = synth.grid_graph(20 + 7 * i, 0.9, seed=700 + i)
            orders.append(blest.BLEST_ORDER_BANDWIDTH)
        graphs.append(g)
        srcs.append(int(synth.pick_sources(g, 1, seed=800 + i)[0]))
    offs = np.concatenate([[0], np.cumsum([g.n for g in graphs])[:-1]])
    h = blest.blest_batch_create([(g.n, g.row_ptr, g.col_idx) for g in graphs], orders)
    try:
        r = blest.blest_autotune_multiroot(h, (offs + np.asarray(srcs)).astype(np.int32))
        assert r["candidates"] > 20 and r["best_ms"] > 0
        got = blest.blest_batch_bfs(h, srcs)
        for g, s, o in zip(graphs, srcs, offs):
            assert np.array_equal(got[o:o + g.n], oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, s))
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("update", ["eager", "lazy"])
def test_device_api_with_torch_stream(torch_cuda, update):
    """Device output into rows of a caller's tensor on the caller's stream
    (the lazy path writes levels straight into that buffer)."""
    torch = torch_cuda
    g = synth.rmat_graph(13, 16, seed=9)
    srcs = synth.pick_sources(g, 5, seed=1)
    exp = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS)
    try:
        blest.blest_set_option(h, blest.BLEST_OPT_UPDATE,
                               blest.BLEST_UPDATE_EAGER if update == "eager" else blest.BLEST_UPDATE_LAZY)
        s = torch.cuda.Stream()
        out = torch.empty((len(srcs), g.n), dtype=torch.int32, device="cuda")
        for i, src in enumerate(srcs):
            blest.blest_bfs_device(h, int(src), out[i], stream=s)
        blest.blest_sync(h)
        assert np.array_equal(out.cpu().numpy(), exp)
        out2 = torch.empty((len(srcs), g.n), dtype=torch.int32, device="cuda")
        blest.blest_msbfs_device(h, srcs, out2, stream=s)
        blest.blest_sync(h)
        assert np.array_equal(out2.cpu().numpy(), exp)
    finally:
        blest.blest_destroy(h)


def test_autotune_keeps_levels_exact(gpu):
    g, srcs = synth.rmat_workload(13, 8, seed_graph=7, seed_src=7)
    exp = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs, threads=8)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS)
    try:
        r = blest.blest_autotune(h, srcs[:3])
        # 5 probe variants pick the update scheme, then every variant of that scheme (>= 32) is timed
        assert r["candidates"] >= 37 and 0 < r["best_ms"] <= r["rule_ms"]
        for i, s in enumerate(srcs):
            assert np.array_equal(blest.blest_bfs(h, int(s)), exp[i])
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("update", ["eager", "lazy"])
def test_batch_graph_capture_replay(torch_cuda, update):
    """One captured CUDA graph replayed with new sources gives every graph's own
    single-source levels."""
    torch = torch_cuda
    graphs, orders = [], []
    for i in range(20):
        if i % 2 == 0:
            graphs.append(synth.rmat_graph(6 + i % 7, 16, seed=400 + i))
            orders.append(blest.BLEST_ORDER_COMPRESS)
        else:
            graphs.append(synth.grid_graph(10 + 3 * i, 0.9, seed=500 + i)[0])
            orders.append(blest.BLEST_ORDER_BANDWIDTH)
    h = blest.blest_batch_create([(g.n, g.row_ptr, g.col_idx) for g in graphs], orders)
    try:
        blest.blest_set_option(h, blest.BLEST_OPT_UPDATE,
                               blest.BLEST_UPDATE_EAGER if update == "eager" else blest.BLEST_UPDATE_LAZY)
        total = sum(g.n for g in graphs)
        out = torch.empty(total, dtype=torch.int32, device="cuda")
        blest.blest_batch_graph_capture(h, out)
        for rep in range(3):
            srcs = [int(synth.pick_sources(g, 1, seed=600 + 31 * rep + i)[0]) for i, g in enumerate(graphs)]
            blest.blest_batch_graph_launch(h, srcs)
            blest.blest_sync(h)
            got = out.cpu().numpy()
            off = 0
            for g, s in zip(graphs, srcs):
                assert np.array_equal(got[off:off + g.n], oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, s))
                off += g.n
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("order", ["none", "compress", "bandwidth"])
def test_parents_match_oracle(gpu, order):
    g = synth.rmat_graph(12, 16, seed=31)
    srcs = synth.pick_sources(g, 4, seed=2)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, ORDERS[order])
    try:
        for s in srcs:
            lv, par = blest.blest_bfs_parents(h, int(s))
            elv, epar = oracle.bfs_parents(g.n, g.row_ptr, g.col_idx, int(s))
            assert np.array_equal(lv, elv) and np.array_equal(par, epar)
    finally:
        blest.blest_destroy(h)
    gg, srcs2 = synth.grid_workload(64, 3, seed_graph=8, seed_src=8)
    h = blest.blest_graph_create(gg.n, gg.row_ptr, gg.col_idx, blest.BLEST_ORDER_BANDWIDTH)
    try:
        for s in srcs2:
            lv, par = blest.blest_bfs_parents(h, int(s))
            elv, epar = oracle.bfs_parents(gg.n, gg.row_ptr, gg.col_idx, int(s))
            assert np.array_equal(lv, elv) and np.array_equal(par, epar)
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("update", ["eager", "lazy"])
def test_stale_levels_do_not_leak(gpu, update):
    """Two components: a traversal of the second after one of the first must
    report the first as unreached, although the handle's internal level array
    still holds the earlier levels (a lazy traversal with a reordering does not
    clear it and reads the reached rows off its visited bitmap)."""
    a = synth.rmat_graph(10, 8, seed=41, relabel=False)
    b = synth.rmat_graph(9, 8, seed=42, relabel=False)
    n = a.n + b.n
    src = np.concatenate([np.repeat(np.arange(a.n), np.diff(a.row_ptr)),
                          a.n + np.repeat(np.arange(b.n), np.diff(b.row_ptr))]).astype(np.int32)
    dst = np.concatenate([a.col_idx, a.n + b.col_idx]).astype(np.int32)
    g = synth.csr_from_edges(n, src, dst, relabel=synth.permutation(n, 43))
    comp = synth.components(g)
    big = np.bincount(comp).argsort()[::-1]
    s1 = int(np.nonzero(comp == big[0])[0][0])
    s2 = int(np.nonzero(comp == big[1])[0][0])
    upd = blest.BLEST_UPDATE_EAGER if update == "eager" else blest.BLEST_UPDATE_LAZY
    for order in (blest.BLEST_ORDER_COMPRESS, blest.BLEST_ORDER_BANDWIDTH, blest.BLEST_ORDER_NONE):
        h = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, order, window=64)
        try:
            blest.blest_set_option(h, blest.BLEST_OPT_UPDATE, upd)
            blest.blest_set_option(h, blest.BLEST_OPT_LAYOUT, 1 if update == "lazy" and order != blest.BLEST_ORDER_NONE else 0)
            for s in (s1, s2, s1, s2):
                got = blest.blest_bfs(h, s)
                assert np.array_equal(got, oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, s))
            got = blest.blest_bfs_multiroot(h, [s2])
            assert np.array_equal(got, oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, s2))
        finally:
            blest.blest_destroy(h)


@pytest.mark.parametrize("scale,seed", [(8, 3), (10, 5)])
def test_compact_layout_matches_oracle(gpu, scale, seed):
    """The device-built compact layout equals the oracle's, array for array
    (identity order, so BVSS ids are original ids)."""
    g = synth.rmat_graph(scale, 16, seed=seed)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE)
    try:
        c = ob.compact(g.n, g.row_ptr, g.col_idx)
        assert np.array_equal(blest.blest_export(h, blest.BLEST_ARRAY_COMPACT_OFFSETS), c.goff)
        assert np.array_equal(blest.blest_export(h, blest.BLEST_ARRAY_COMPACT_ROWS), c.rows)
        assert np.array_equal(blest.blest_export(h, blest.BLEST_ARRAY_COMPACT_MASKS), c.masks)
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("update", ["eager", "lazy"])
def test_level_timeline_and_arrivals(cfg1, update):
    """Record mode: the level stamps increase, and every block's end of stage 1
    lies between that level's stage-1 start and the stamp taken after the
    barrier that waits for all blocks (causality on the global timer)."""
    g, srcs, exp = cfg1
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS)
    try:
        blest.blest_set_option(h, blest.BLEST_OPT_UPDATE,
                               blest.BLEST_UPDATE_EAGER if update == "eager" else blest.BLEST_UPDATE_LAZY)
        blest.blest_set_option(h, blest.BLEST_OPT_RECORD_LEVELS, 1)
        for s in srcs[:3]:
            assert np.array_equal(blest.blest_bfs(h, int(s)), exp[list(srcs).index(s)])
            info, _ = blest.blest_get_run_info(h, 64)
            L = info["levels"]
            t = blest.blest_get_level_times(h, 2 * L + 4).astype(np.int64)
            first, last = blest.blest_get_level_arrivals(h, L)
            first, last = first.astype(np.int64), last.astype(np.int64)
            sf, sl = blest.blest_get_level_arrivals(h, L, phase=1)
            assert t[1] <= t[0] <= t[2]
            for l in range(1, L + 1):
                after = t[2 * l + 1] if update == "lazy" else t[2 * l + 2]
                assert first[l - 1] <= last[l - 1] <= after
                assert t[2 * l] <= after
                if update == "lazy":
                    # a block's sweep starts after the barrier that waits for every block's stage 1,
                    # and the next level starts after the barrier that waits for every sweep
                    assert last[l - 1] <= int(sf[l - 1]) <= int(sl[l - 1]) <= t[2 * l + 2]
                else:
                    assert int(sf[l - 1]) == 2**64 - 1 and int(sl[l - 1]) == 0
            assert t[2 * L + 2] <= t[2 * L + 3]
    finally:
        blest.blest_destroy(h)


def test_distance_stats_match_oracle(gpu):
    """Closeness / diameter statistics over 300 sources (two multi-source
    batches) on an R-MAT graph with isolated vertices, and on a grid."""
    g = synth.rmat_graph(11, 8, seed=77)
    srcs = synth.pick_sources(g, 300, seed=5)
    srcs[7] = int(np.nonzero(np.diff(g.row_ptr) == 0)[0][0])   # an isolated source
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS)
    try:
        got = blest.blest_distance_stats(h, srcs)
        exp = oracle.distance_stats(g.n, g.row_ptr, g.col_idx, srcs, threads=8)
        for a, b in zip(got, exp):
            assert np.array_equal(a, b)
        assert got[0][7] == 1 and got[1][7] == 0 and got[2][7] == 0
        with pytest.raises(blest.BlestError):
            blest.blest_distance_stats(h, [0, g.n])
    finally:
        blest.blest_destroy(h)
    gg, gs = synth.grid_workload(48, 5, seed_graph=9, seed_src=9)
    h = blest.blest_graph_create(gg.n, gg.row_ptr, gg.col_idx, blest.BLEST_ORDER_BANDWIDTH)
    try:
        got = blest.blest_distance_stats(h, gs)
        exp = oracle.distance_stats(gg.n, gg.row_ptr, gg.col_idx, gs)
        for a, b in zip(got, exp):
            assert np.array_equal(a, b)
    finally:
        blest.blest_destroy(h)


def test_checkpoint_round_trip(gpu, tmp_path):
    """A saved and reloaded handle has the same arrays, statistics and levels;
    a file with one row id corrupted is refused."""
    g = synth.rmat_graph(12, 16, seed=13)
    srcs = synth.pick_sources(g, 6, seed=3)
    h = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS, window=256)
    path = str(tmp_path / "g.blest")
    try:
        blest.blest_graph_save(h, path)
        h2 = blest.blest_graph_load(path)
        try:
            for which in (blest.BLEST_ARRAY_REAL_PTRS, blest.BLEST_ARRAY_VIRTUAL_TO_REAL, blest.BLEST_ARRAY_ROW_IDS,
                          blest.BLEST_ARRAY_MASKS, blest.BLEST_ARRAY_NEW_ID, blest.BLEST_ARRAY_VSS_COUNT):
                assert np.array_equal(blest.blest_export(h, which), blest.blest_export(h2, which))
            assert blest.blest_get_stats(h) == blest.blest_get_stats(h2)
            for s in srcs:
                assert np.array_equal(blest.blest_bfs(h2, int(s)), oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(s)))
        finally:
            blest.blest_destroy(h2)
    finally:
        blest.blest_destroy(h)
    raw = bytearray(open(path, "rb").read())
    # corrupt the last int32 of the row-id array: it sits just before masks and counts
    nvss = int(np.frombuffer(bytes(raw[32:40]), np.int64)[0])
    tail = 4 * 32 * nvss + 4 * nvss
    pos = len(raw) - tail - 4
    raw[pos:pos + 4] = np.array([g.n + 5], np.int32).tobytes()
    bad = str(tmp_path / "bad.blest")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(blest.BlestError) as e:
        blest.blest_graph_load(bad)
    assert "row id" in str(e.value)


def test_checkpoint_batch_handle(gpu, tmp_path):
    graphs = [synth.rmat_graph(9, 8, seed=s) for s in (1, 2)] + [synth.grid_graph(20, 0.9, seed=3)[0]]
    h = blest.blest_batch_create([(g.n, g.row_ptr, g.col_idx) for g in graphs],
                                 [blest.BLEST_ORDER_COMPRESS, blest.BLEST_ORDER_COMPRESS, blest.BLEST_ORDER_BANDWIDTH])
    path = str(tmp_path / "b.blest")
    try:
        blest.blest_graph_save(h, path)
        want = blest.blest_batch_bfs(h, [3, 5, 7])
    finally:
        blest.blest_destroy(h)
    h2 = blest.blest_graph_load(path)
    try:
        got = blest.blest_batch_bfs(h2, [3, 5, 7])
        assert np.array_equal(got, want)
        off = 0
        for g, s in zip(graphs, (3, 5, 7)):
            assert np.array_equal(got[off:off + g.n], oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, s))
            off += g.n
    finally:
        blest.blest_destroy(h2)


# ------------------------------------------------------------ full sizes
# The benchmark's own workloads at their full sizes, built and tuned as bench.py
# builds and tunes them.  Sampled sources are compared element by element with
# the oracle's single-source BFS, which takes a second or two at these sizes.

def _bench_like_handle(g, order, tune_srcs):
    h = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, order, window=4096)
    for key, val in ((blest.BLEST_OPT_UNROLL, 2), (blest.BLEST_OPT_MIN_BLOCKS, 2),
                     (blest.BLEST_OPT_VISITED_FILTER, 3), (blest.BLEST_OPT_STAGE_DEPTH, 2)):
        blest.blest_set_option(h, key, val)
    blest.blest_autotune(h, tune_srcs)
    return h


@pytest.mark.parametrize("workload", ["rmat23", "grid4096"])
def test_full_size_single_source_sampled(gpu, workload):
    """R-MAT scale 23 (compression order) and the 4096 x 4096 grid (RCM), the
    autotuned variant the benchmark times, three sampled sources each."""
    if workload == "rmat23":
        g, srcs = synth.rmat_workload(23, 64, seed_graph=2, seed_src=1002)
        order = blest.BLEST_ORDER_COMPRESS
    else:
        g, srcs = synth.grid_workload(4096, 64, seed_graph=3, seed_src=1003)
        order = blest.BLEST_ORDER_BANDWIDTH
    h = _bench_like_handle(g, order, srcs[:4])
    try:
        check_levels(g, h, [srcs[0], srcs[37], srcs[-1]])
    finally:
        blest.blest_destroy(h)


def test_full_size_multi_source_sampled(torch_cuda):
    """R-MAT scale 22, k = 64 sources in one launch into device memory, as the
    benchmark runs it; three sampled rows against the oracle."""
    torch = torch_cuda
    g, srcs = synth.rmat_workload(22, 64, seed_graph=4, seed_src=1004)
    h = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS, window=4096)
    try:
        s = torch.cuda.Stream()
        out = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
        blest.blest_msbfs_device(h, srcs[:64], out, stream=s)
        blest.blest_sync(h)
        for i in (0, 29, 63):
            exp = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(srcs[i]))
            assert np.array_equal(out[i].cpu().numpy(), exp), f"row {i} (source {srcs[i]}) differs"
    finally:
        blest.blest_destroy(h)
