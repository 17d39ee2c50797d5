"""The allocation-free traversal entry point, blest_bfs_static_scratch.

It serves callers that may not call cudaMalloc (allocation-forbidding graph
capture, plugins whose host owns device memory, pre-budgeted services): its
working memory is one fixed device array inside the library.  This file is
collected last on purpose, so that a run stopping at the first failure has
already run every other test.  The entry point must give exactly the levels of
the ordinary handle path (blest_bfs), on two calls in a row sharing the array,
whether it runs alone in a fresh process or after the other tests."""
import numpy as np
import pytest

import paper_2512_21967_gb300 as blest
from paper_2512_21967_gb300 import synth

pytestmark = pytest.mark.gpu


def device_arrays(torch, h):
    ex = {w: blest.blest_export(h, w) for w in (blest.BLEST_ARRAY_REAL_PTRS, blest.BLEST_ARRAY_ROW_IDS,
                                                  blest.BLEST_ARRAY_MASKS, blest.BLEST_ARRAY_NEW_ID)}
    d = {w: torch.from_numpy(a.view(np.int32)).cuda() for w, a in ex.items()}
    return ex, d


@pytest.mark.parametrize("update", [blest.BLEST_UPDATE_LAZY, blest.BLEST_UPDATE_EAGER])
@pytest.mark.parametrize("order", [blest.BLEST_ORDER_COMPRESS, blest.BLEST_ORDER_NONE])
def test_static_scratch_matches_handle_path(gpu, update, order):
    import torch
    g = synth.rmat_graph(14, 16, seed=21)
    srcs = synth.pick_sources(g, 2, seed=5)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, order)
    try:
        st = blest.blest_get_stats(h)
        ex, d = device_arrays(torch, h)
        new_id = ex[blest.BLEST_ARRAY_NEW_ID]
        d_new_id = None if order == blest.BLEST_ORDER_NONE else d[blest.BLEST_ARRAY_NEW_ID]
        for src in srcs:                                       # two calls in a row share the array
            expected = blest.blest_bfs(h, int(src))
            out = torch.full((g.n,), 12345, dtype=torch.int32, device="cuda")
            blest.blest_bfs_static_scratch(g.n, st["num_vss"], d[blest.BLEST_ARRAY_REAL_PTRS],
                                           d[blest.BLEST_ARRAY_ROW_IDS], d[blest.BLEST_ARRAY_MASKS], d_new_id,
                                           int(new_id[src]), out, update)
            assert np.array_equal(out.cpu().numpy(), expected)
    finally:
        blest.blest_destroy(h)


def test_static_scratch_rejects_sizes_beyond_its_array(gpu):
    import torch
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(blest.BlestError) as e:
        blest.blest_bfs_static_scratch((1 << 21) + 1, 10, dummy, dummy, dummy, None, 0, dummy)
    assert e.value.name == "BLEST_ERR_TOO_LARGE"
    with pytest.raises(blest.BlestError) as e:
        blest.blest_bfs_static_scratch(1000, (1 << 19) + 1, dummy, dummy, dummy, None, 0, dummy)
    assert e.value.name == "BLEST_ERR_TOO_LARGE"
