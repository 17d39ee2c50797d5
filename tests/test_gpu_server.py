"""The query server: continuous batching must not change any result.  Every
query's levels equal the oracle's for its sources, whether the query runs
alone or mixed with concurrent queries on other graphs."""
import numpy as np
import pytest

import oracle
import paper_2512_21967_gb300 as blest
from paper_2512_21967_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served(gpu):
    graphs = [synth.rmat_graph(10, 16, seed=71), synth.rmat_graph(12, 16, seed=72), synth.rmat_graph(11, 8, seed=73),
              synth.grid_graph(40, 0.9, seed=74)[0], synth.grid_graph(64, 0.9, seed=75)[0],
              synth.rmat_graph(9, 16, seed=76)]
    # the last graph keeps its own vertex ids (no reordering)
    orders = [blest.BLEST_ORDER_COMPRESS] * 3 + [blest.BLEST_ORDER_BANDWIDTH] * 2 + [blest.BLEST_ORDER_NONE]
    handles = [blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, o) for g, o in zip(graphs, orders)]
    rng = np.random.default_rng(7)
    queries = []
    for i in range(36):
        gi = int(rng.integers(len(graphs)))
        k = int(rng.integers(1, 9))
        srcs = synth.pick_sources(graphs[gi], k, seed=900 + i)
        queries.append((gi, srcs, oracle.msbfs_levels(graphs[gi].n, graphs[gi].row_ptr, graphs[gi].col_idx, srcs)))
    yield graphs, handles, queries
    for h in handles:
        blest.blest_destroy(h)


def test_results_alone_and_in_the_mix(served):
    graphs, handles, queries = served
    srv = blest.blest_server_create(handles, max_batch_sources=16, max_inflight=3)
    try:
        alone = []
        for gi, srcs, exp in queries:
            out = np.full((len(srcs), graphs[gi].n), 99, np.int32)
            t = blest.blest_server_submit(srv, gi, srcs, out)
            blest.blest_server_wait(srv, t, 30.0)
            assert np.array_equal(out, exp)
            alone.append(out)
        before = blest.blest_server_get_stats(srv)["launches"]
        outs, tickets = [], []
        blest.blest_server_pause(srv, True)               # build a backlog, then let it coalesce
        for gi, srcs, exp in queries:
            out = np.full((len(srcs), graphs[gi].n), 99, np.int32)
            outs.append(out)
            tickets.append(blest.blest_server_submit(srv, gi, srcs, out))
        assert blest.blest_server_get_stats(srv)["queries_waiting"] == len(queries)
        blest.blest_server_pause(srv, False)
        lat = [blest.blest_server_wait(srv, t, 60.0) for t in tickets]
        st = blest.blest_server_get_stats(srv)
        for out, ref, (_, _, exp) in zip(outs, alone, queries):
            assert np.array_equal(out, ref) and np.array_equal(out, exp)
        assert st["launches"] - before < len(queries), "queries of the same graph were not coalesced"
        assert st["queries_done"] == 2 * len(queries) and st["queries_waiting"] == 0
        assert all(x >= 0 for x in lat)
    finally:
        blest.blest_server_destroy(srv)


def test_narrow_launches_keep_results(served):
    """Graphs whose last launch ran more than narrow_levels levels (the grids here,
    40 to 130 levels) launch on a narrow grid of 8 SMs; results stay the oracle's."""
    graphs, handles, queries = served
    srv = blest.blest_server_create(handles, max_batch_sources=16, max_inflight=4, narrow_sms=8, narrow_levels=10)
    try:
        for _ in range(2):                                 # the first pass learns each graph's level count
            outs, tickets = [], []
            for gi, srcs, exp in queries:
                out = np.full((len(srcs), graphs[gi].n), 99, np.int32)
                outs.append(out)
                tickets.append(blest.blest_server_submit(srv, gi, srcs, out))
            for t in tickets:
                blest.blest_server_wait(srv, t, 60.0)
            for out, (_, _, exp) in zip(outs, queries):
                assert np.array_equal(out, exp)
    finally:
        blest.blest_server_destroy(srv)


@pytest.mark.parametrize("long_slots", [1, 2])
def test_long_slot_cap_keeps_results(served, long_slots):
    """With launches of long graphs (here the grids: their last launch ran more
    than narrow_levels levels) capped below the slot count, every query still
    completes with the oracle's levels, long and short alike."""
    graphs, handles, queries = served
    srv = blest.blest_server_create(handles, max_batch_sources=8, max_inflight=3, narrow_levels=10,
                                    long_slots=long_slots)
    try:
        for _ in range(2):                                 # the first pass learns each graph's level count
            outs, tickets = [], []
            for gi, srcs, exp in queries:
                out = np.full((len(srcs), graphs[gi].n), 99, np.int32)
                outs.append(out)
                tickets.append(blest.blest_server_submit(srv, gi, srcs, out))
            for t in tickets:
                blest.blest_server_wait(srv, t, 60.0)
            for out, (_, _, exp) in zip(outs, queries):
                assert np.array_equal(out, exp)
    finally:
        blest.blest_server_destroy(srv)


def test_memory_cap_admits_one_launch_at_a_time(served):
    graphs, handles, queries = served
    n_max = max(g.n for g in graphs)
    cap = 4 * 16 * n_max * 4      # room for roughly one 16-source launch of the largest graph
    srv = blest.blest_server_create(handles, memory_cap_bytes=cap, max_batch_sources=16, max_inflight=4)
    try:
        outs, tickets = [], []
        for gi, srcs, exp in queries[:20]:
            out = np.empty((len(srcs), graphs[gi].n), np.int32)
            outs.append(out)
            tickets.append(blest.blest_server_submit(srv, gi, srcs, out))
        for t in tickets:
            blest.blest_server_wait(srv, t, 60.0)
        for out, (_, _, exp) in zip(outs, queries[:20]):
            assert np.array_equal(out, exp)
        assert blest.blest_server_get_stats(srv)["memory_peak"] <= cap
    finally:
        blest.blest_server_destroy(srv)


def test_device_output_and_bad_queries(served):
    import torch
    graphs, handles, queries = served
    srv = blest.blest_server_create(handles, max_batch_sources=8, max_queries_per_launch=1, max_inflight=1)
    try:
        gi, srcs, exp = queries[0]
        d = torch.empty((len(srcs), graphs[gi].n), dtype=torch.int32, device="cuda")
        blest.blest_server_wait(srv, blest.blest_server_submit(srv, gi, srcs, d), 30.0)
        assert np.array_equal(d.cpu().numpy(), exp)
        with pytest.raises(blest.BlestError) as e:
            blest.blest_server_submit(srv, gi, np.zeros(9, np.int32))
        assert e.value.name == "BLEST_ERR_TOO_LARGE"
        with pytest.raises(blest.BlestError):
            blest.blest_server_submit(srv, len(handles), [0])
        with pytest.raises(blest.BlestError):
            blest.blest_server_submit(srv, 0, [graphs[0].n])
        with pytest.raises(blest.BlestError):
            blest.blest_server_wait(srv, 123456789, 0.0)
    finally:
        blest.blest_server_destroy(srv)
