"""Sharded single-source BFS: one rank per GPU, the pull split by slice set.

Rank r of `world` pulls only the queued VSSs of the slice sets s with
s mod world = r.  After every level's pull, the ranks OR their V_next words
together (the exchange; the paper names multi-GPU BFS as future work in
Section 6), and every rank runs the same finalisation sweep on the combined
words, so each ends with the full level array.  The steps are the C ABI's
blest_shard_begin / blest_shard_pull / blest_shard_merge / blest_shard_finish;
this module only sequences them around the caller's collective.
"""
from __future__ import annotations

from typing import Callable


def run_levels(step, exchange: Callable) -> int:
    """Drive one rank through a traversal: step.begin(); then per level
    words = step.pull(), merged = exchange(words), step.finish(merged) until
    finish reports the traversal over.  Returns the number of levels pulled."""
    step.begin()
    levels = 0
    while True:
        words = step.pull()
        merged = exchange(words)
        levels += 1
        if not step.finish(merged):
            return levels


class DeviceShard:
    """This rank's steps on its GPU through the C ABI.  d_levels: CUDA int32
    tensor of n entries that receives the levels in original ids.  Every step
    runs on `stream` (default: torch's current stream on d_levels' device), the
    stream the exchange must use too, so that the words it reads are the pull's."""

    def __init__(self, h: int, rank: int, world: int, src: int, d_levels, stream=None):
        import torch

        from . import _n_of
        self.h, self.rank, self.world, self.src = h, rank, world, int(src)
        self.d_levels = d_levels
        self.stream = stream if stream is not None else torch.cuda.current_stream(d_levels.device)
        self.nwords = (_n_of(h) + 31) // 32
        self.words = torch.empty(max(self.nwords, 1), dtype=torch.int32, device=d_levels.device)

    def begin(self):
        from . import blest_shard_begin
        blest_shard_begin(self.h, self.rank, self.world, self.src, self.d_levels, self.stream)

    def pull(self):
        from . import blest_shard_pull
        blest_shard_pull(self.h, self.words, self.stream)
        return self.words

    def finish(self, merged) -> bool:
        from . import blest_shard_finish
        return blest_shard_finish(self.h, merged, self.stream)


def allgather_or(group=None, stream=None) -> Callable:
    """Exchange over torch.distributed: all-gather every rank's words, then OR
    them with blest_shard_merge (NCCL has no bitwise reduction).  Runs on torch's
    current stream, or on `stream` for the merge: the stream of the steps."""
    import torch
    import torch.distributed as dist

    from . import blest_shard_merge

    def exchange(words):
        world = dist.get_world_size(group)
        gathered = torch.empty(world * words.numel(), dtype=words.dtype, device=words.device)
        dist.all_gather_into_tensor(gathered, words, group=group)
        merged = torch.empty_like(words)
        blest_shard_merge(merged, gathered, words.numel(), world,
                          stream if stream is not None else torch.cuda.current_stream(words.device))
        return merged

    return exchange


def sharded_bfs(h: int, src: int, rank: int, world: int, d_levels, exchange: Callable, stream=None) -> int:
    """One rank of a sharded single-source BFS from original vertex src on
    handle h; exchange(words) must return the OR of every rank's words (for
    example allgather_or()).  Returns the number of levels pulled."""
    return run_levels(DeviceShard(h, rank, world, src, d_levels, stream), exchange)
