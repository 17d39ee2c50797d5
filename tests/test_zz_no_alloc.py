"""The allocation-free traversal entry point, blest_bfs_static_scratch.

It serves callers that may not call cudaMalloc (plugins and embedded runtimes
whose host application owns every device allocation, services whose device
memory is budgeted up front): its working memory is one fixed device array
inside the library.  This file is collected last on purpose, so that a run
stopping at the first failure has already run every other test.  On two calls
in a row sharing the array, the entry point must give exactly the oracle's
levels and those of the ordinary handle path (blest_bfs), whether it runs alone
in a fresh process or after the other tests; the cases include a vertex count
that is not a multiple of 32 and a graph at the array's vertex limit with a
virtual-slice-set count near its limit."""
import numpy as np
import pytest

import oracle
import paper_2512_21967_gb300 as blest
from paper_2512_21967_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_VERTICES = 1 << 21
MAX_VSS = 1 << 19


def device_arrays(torch, h):
    ex = {w: blest.blest_export(h, w) for w in (blest.BLEST_ARRAY_REAL_PTRS, blest.BLEST_ARRAY_ROW_IDS,
                                                  blest.BLEST_ARRAY_MASKS, blest.BLEST_ARRAY_NEW_ID)}
    d = {w: torch.from_numpy(a.view(np.int32)).cuda() for w, a in ex.items()}
    return ex, d


def check_two_calls(g, srcs, order, update):
    """Two calls in a row through the allocation-free entry point, each compared
    element by element with the oracle and with blest_bfs."""
    import torch
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, order)
    try:
        st = blest.blest_get_stats(h)
        ex, d = device_arrays(torch, h)
        new_id = ex[blest.BLEST_ARRAY_NEW_ID]
        d_new_id = None if order == blest.BLEST_ORDER_NONE else d[blest.BLEST_ARRAY_NEW_ID]
        for src in srcs:
            want = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(src))
            assert np.array_equal(blest.blest_bfs(h, int(src)), want)
            out = torch.full((g.n,), 12345, dtype=torch.int32, device="cuda")
            blest.blest_bfs_static_scratch(g.n, st["num_vss"], d[blest.BLEST_ARRAY_REAL_PTRS],
                                           d[blest.BLEST_ARRAY_ROW_IDS], d[blest.BLEST_ARRAY_MASKS], d_new_id,
                                           int(new_id[src]), out, update)
            assert np.array_equal(out.cpu().numpy(), want)
        return st
    finally:
        blest.blest_destroy(h)


@pytest.mark.parametrize("update", [blest.BLEST_UPDATE_LAZY, blest.BLEST_UPDATE_EAGER])
@pytest.mark.parametrize("order", [blest.BLEST_ORDER_COMPRESS, blest.BLEST_ORDER_NONE])
def test_static_scratch_matches_oracle_and_handle_path(gpu, update, order):
    g = synth.rmat_graph(14, 16, seed=21)
    check_two_calls(g, synth.pick_sources(g, 2, seed=5), order, update)


@pytest.mark.parametrize("update", [blest.BLEST_UPDATE_LAZY, blest.BLEST_UPDATE_EAGER])
def test_static_scratch_ragged_grid(gpu, update):
    g, _ = synth.grid_graph(45, 0.9, seed=8)          # n = 2025, not a multiple of 32; ~90 levels
    assert g.n % 32 != 0
    check_two_calls(g, [0, g.n - 1], blest.BLEST_ORDER_BANDWIDTH, update)


@pytest.mark.parametrize("update", [blest.BLEST_UPDATE_LAZY, blest.BLEST_UPDATE_EAGER])
def test_static_scratch_at_its_limits(gpu, update):
    # R-MAT scale 21 in the original order: n is exactly the vertex limit, and with
    # edgefactor 11 the slice sets hold about 515,000 virtual slice sets, so the
    # queues reach into the top of the fixed array
    g = synth.rmat_graph(21, 11, seed=21)
    assert g.n == MAX_VERTICES
    st = check_two_calls(g, synth.pick_sources(g, 2, seed=6), blest.BLEST_ORDER_NONE, update)
    assert 0.95 * MAX_VSS < st["num_vss"] <= MAX_VSS


def test_static_scratch_rejects_sizes_beyond_its_array(gpu):
    import torch
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(blest.BlestError) as e:
        blest.blest_bfs_static_scratch(MAX_VERTICES + 1, 10, dummy, dummy, dummy, None, 0, dummy)
    assert e.value.name == "BLEST_ERR_TOO_LARGE"
    with pytest.raises(blest.BlestError) as e:
        blest.blest_bfs_static_scratch(1000, MAX_VSS + 1, dummy, dummy, dummy, None, 0, dummy)
    assert e.value.name == "BLEST_ERR_TOO_LARGE"
