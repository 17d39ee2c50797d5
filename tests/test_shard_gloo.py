"""The sharded single-source traversal's host side on CPU ranks (gloo): the
level driver of paper_2512_21967_gb300.shard with an all-gather + OR exchange
between 2, 3 and 4 processes, on a power-law graph, a grid with several
components, a long path and a source without edges.  Each rank's device steps are replaced by a CPU
stand-in with the same contract (it pulls only the slice sets s with
s mod world = rank, returns its V_next words, and finishes a level from the
merged words), so the test checks what runs on the host: that the partition
covers every slice set once, that the OR exchange merges the ranks' marks,
that every rank ends the traversal at the same level, and that the levels are
the oracle's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class CpuShard:
    """CPU stand-in for one rank's device steps (lazy update, Algorithm 3): the
    vertex order is the original one, slice set s = vertices 8s .. 8s + 7."""

    def __init__(self, g, src, rank, world):
        self.g, self.src, self.rank, self.world = g, int(src), rank, world
        self.n = g.n
        self.nwords = (g.n + 31) // 32

    def _words(self, bits):
        padded = np.zeros(self.nwords * 32, np.uint8)
        padded[:self.n] = bits
        return np.packbits(padded.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").astype(np.uint32).reshape(-1)

    def _bits(self, words):
        w = np.asarray(words, dtype=np.uint32).astype(">u4").view(np.uint8).reshape(-1, 4)
        return np.unpackbits(w, axis=1)[:, ::-1].reshape(-1)[:self.n].astype(bool)

    def _finalise(self, lvl):
        new = self.vnext & ~self.vis
        self.levels[new] = lvl
        self.vis |= new
        self.frontier = new
        owned = (np.arange(self.n) // 8) % self.world == self.rank
        self.queue = np.unique(np.flatnonzero(new & owned) // 8)
        return bool(new.any())

    def begin(self):
        self.vis = np.zeros(self.n, bool)
        self.vnext = np.zeros(self.n, bool)
        self.levels = np.full(self.n, -1, np.int32)
        self.vnext[self.src] = True
        self.lvl = 0
        self._finalise(0)
        self.lvl = 1

    def pull(self):
        import torch
        rp, ci = self.g.row_ptr, self.g.col_idx
        for s in self.queue:
            for c in range(8 * s, min(8 * s + 8, self.n)):
                if self.frontier[c]:
                    self.vnext[ci[rp[c]:rp[c + 1]]] = True
        return torch.from_numpy(self._words(self.vnext).view(np.int32).copy())

    def finish(self, merged):
        self.vnext = self._bits(merged.numpy().view(np.uint32))
        more = self._finalise(self.lvl)
        self.lvl += 1
        return more


def _gloo_exchange(words):
    import torch
    import torch.distributed as dist
    world = dist.get_world_size()
    parts = [torch.empty_like(words) for _ in range(world)]
    dist.all_gather(parts, words)
    merged = parts[0].clone()
    for p in parts[1:]:
        merged |= p
    return merged


def _worker(rank, world, port, q, case):
    import torch.distributed as dist

    from paper_2512_21967_gb300 import shard, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, src = _graph(case)
        step = CpuShard(g, src, rank, world)
        levels = shard.run_levels(step, _gloo_exchange)
        q.put((rank, levels, step.levels.tolist()))
    finally:
        dist.destroy_process_group()


def _graph(case):
    from paper_2512_21967_gb300 import synth
    if case == "rmat":
        g = synth.rmat_graph(9, 8, seed=12)
        return g, int(synth.pick_sources(g, 1, seed=3)[0])
    if case == "isolated":                          # a source with no edges: one pulled level
        g = synth.rmat_graph(9, 8, seed=12)
        return g, int(np.flatnonzero(np.diff(g.row_ptr) == 0)[0])
    if case == "path":                              # 150 levels; most ranks own no frontier at a level
        n = 150
        a = np.arange(n - 1, dtype=np.int32)
        return synth.csr_from_edges(n, a, a + 1), 0
    g, _ = synth.grid_graph(23, 0.85, seed=5)       # n = 529, many levels, several components
    return g, 0


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("case", ["rmat", "grid", "isolated", "path"])
def test_sharded_levels_on_gloo_ranks(world, case):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, case)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g, src = _graph(case)
    want = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, src)
    nlevels = {lv for _, lv, _ in out}
    assert len(nlevels) == 1, "every rank must end the traversal at the same level"
    assert nlevels.pop() == int(want.max()) + 1     # levels 1 .. max + 1 are pulled
    for _, _, levels in out:
        assert np.array_equal(np.asarray(levels, np.int32), want)


def test_one_rank_alone_pulls_every_slice_set():
    """world = 1: the stand-in's partition is the whole graph, with no exchange."""
    import oracle
    from paper_2512_21967_gb300 import shard
    g, src = _graph("grid")
    step = CpuShard(g, src, 0, 1)
    shard.run_levels(step, lambda w: w)
    assert np.array_equal(step.levels, oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, src))


def test_a_rank_that_skips_the_exchange_is_caught():
    """Planted on the CPU: a rank that finishes from its own words only (no
    exchange) misses the other rank's marks, so its levels differ."""
    import oracle
    from paper_2512_21967_gb300 import shard
    g, src = _graph("rmat")
    step = CpuShard(g, src, 0, 2)
    shard.run_levels(step, lambda w: w)
    assert not np.array_equal(step.levels, oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, src))
