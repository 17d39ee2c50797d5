"""The sharded single-source traversal on the device, with its ranks emulated
in one process on one GPU: each rank has its own handle of the same graph, and
every level runs each rank's pull, merges their words with blest_shard_merge
(the exchange a collective would do), then runs each rank's finalisation
sweep.  No kernel waits on another: the host sequences the steps.  Every rank
must end with the oracle's levels."""
import numpy as np
import pytest

import oracle
import paper_2512_21967_gb300 as blest
from paper_2512_21967_gb300 import shard, synth

pytestmark = pytest.mark.gpu


def emulate_ranks(graph, order, src, world):
    import torch
    hs = [blest.blest_graph_create(graph.n, graph.row_ptr, graph.col_idx, order) for _ in range(world)]
    try:
        outs = [torch.full((graph.n,), 777, dtype=torch.int32, device="cuda") for _ in range(world)]
        stream = torch.cuda.current_stream()      # steps, copies and the merge in one stream order
        steps = [shard.DeviceShard(h, r, world, src, outs[r], stream) for r, h in enumerate(hs)]
        for s in steps:
            s.begin()
        nw = steps[0].nwords
        levels = 0
        while True:
            words = [s.pull().clone() for s in steps]
            gathered = torch.cat(words)
            merged = torch.empty_like(words[0])
            blest.blest_shard_merge(merged, gathered, nw, world, stream)
            more = [s.finish(merged) for s in steps]
            levels += 1
            assert len(set(more)) == 1, "ranks disagree on the end of the traversal"
            if not more[0]:
                break
        return [o.cpu().numpy() for o in outs], levels
    finally:
        for h in hs:
            blest.blest_destroy(h)


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("order", [blest.BLEST_ORDER_COMPRESS, blest.BLEST_ORDER_NONE])
def test_sharded_rmat_matches_oracle(gpu, world, order):
    g = synth.rmat_graph(12, 16, seed=14)
    for src in synth.pick_sources(g, 2, seed=8):
        want = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(src))
        outs, levels = emulate_ranks(g, order, int(src), world)
        assert levels == int(want.max()) + 1
        for got in outs:
            assert np.array_equal(got, want)


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_grid_matches_oracle(gpu, world):
    g, _ = synth.grid_graph(41, 0.9, seed=3)       # n = 1681, ragged, ~80 levels, several components
    want = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, 0)
    outs, _ = emulate_ranks(g, blest.BLEST_ORDER_BANDWIDTH, 0, world)
    for got in outs:
        assert np.array_equal(got, want)


def test_shard_merge_ors_word_arrays(gpu):
    import torch
    rng = np.random.default_rng(4)
    a = rng.integers(-2**31, 2**31, size=(3, 1000), dtype=np.int64).astype(np.int32)
    src = torch.from_numpy(a.reshape(-1)).cuda()
    dst = torch.empty(1000, dtype=torch.int32, device="cuda")
    blest.blest_shard_merge(dst, src, 1000, 3)
    assert np.array_equal(dst.cpu().numpy(), a[0] | a[1] | a[2])


def test_shard_rejects_bad_ranks(gpu):
    import torch
    g = synth.rmat_graph(8, 8, seed=1)
    h = blest.blest_graph_create(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE)
    try:
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for rank, world in ((2, 2), (-1, 2), (0, 0)):
            with pytest.raises(blest.BlestError):
                blest.blest_shard_begin(h, rank, world, 0, out)
        words = torch.empty((g.n + 31) // 32, dtype=torch.int32, device="cuda")
        with pytest.raises(blest.BlestError):
            blest.blest_shard_pull(h, words)       # no traversal begun
    finally:
        blest.blest_destroy(h)
