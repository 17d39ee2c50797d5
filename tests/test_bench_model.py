"""The multi-source byte model of bench.py against the same model written as
plain loops over levels, slice sets and (source, vertex) pairs, on oracle
levels of small graphs (CPU tensors)."""
import numpy as np
import pytest

import oracle
from paper_2512_21967_gb300 import synth

torch = pytest.importorskip("torch")


def plain_ms_bytes(levels, new_id, w_s, nvss, n):
    total, pairs_all = 0, 0
    for c0 in range(0, levels.shape[0], 256):
        lv = levels[c0:c0 + 256]
        k = lv.shape[0]
        W = 1 if k <= 64 else (2 if k <= 128 else 4)
        sets_at = {}                                  # level -> slice sets holding a vertex first reached there
        pairs, lmax = 0, 0
        for i in range(k):
            for v in range(n):
                if lv[i, v] >= 0:
                    pairs += 1
                    lmax = max(lmax, int(lv[i, v]))
                    sets_at.setdefault(int(lv[i, v]), set()).add(int(new_id[v]) // 8)
        stage1 = sum(int(w_s[s]) + 64 * W for ss in sets_at.values() for s in ss)
        sweep = 24 * W * n
        for l in range(1, lmax + 2):
            q = sum(int(nvss[s]) for s in sets_at.get(l - 1, ()))
            sweep += 24 * W * n if q * 128 > n else 24 * W * 8 * len(sets_at.get(l, ()))
        total += stage1 + sweep + 8 * pairs + 4 * k * n + (8 * W + 4) * n
        pairs_all += pairs
    return total, pairs_all


@pytest.mark.parametrize("case", ["rmat-k5", "grid-k70", "rmat-k300", "fullgrid-k1"])
def test_ms_byte_model_matches_plain_definition(case):
    import bench
    if case.startswith("rmat"):
        g = synth.rmat_graph(8, 8, seed=3)
    elif case.startswith("fullgrid"):
        g, _ = synth.grid_graph(40, 1.0, seed=4)     # one source: 10 of 79 levels sweep sparsely
    else:
        g, _ = synth.grid_graph(33, 0.8, seed=4)     # 64 levels, one of them sparse
    k = int(case.split("-k")[1])
    srcs = synth.pick_sources(g, k, seed=5)
    levels = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, srcs)
    rng = np.random.default_rng(6)
    new_id = rng.permutation(g.n).astype(np.int64)
    nss = (g.n + 7) // 8
    nvss = rng.integers(1, 4, nss)
    w_s = rng.integers(20, 2000, nss)
    got = bench.ms_traversal_bytes(torch.from_numpy(levels), torch.from_numpy(new_id), torch.from_numpy(w_s),
                                   torch.from_numpy(nvss), nss, g.n, torch)
    assert got == plain_ms_bytes(levels, new_id, w_s, nvss, g.n)


def test_parallel_cpu_baseline_counts_the_oracle_work():
    """The multi-source host baseline reports the oracle's reached edges over its
    wall time, with the threads it used."""
    import bench
    g = synth.rmat_graph(10, 8, seed=8)
    srcs = synth.pick_sources(g, 6, seed=9)
    out = bench.cpu_baseline_parallel(g, srcs, 4, threads=3)
    assert out["kind"] == "oracle" and out["cores"] == 3 and out["unit"] == "GTEPS"
    edges = sum(oracle.reached_edges(g.row_ptr, oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(s)))
                for s in srcs[:4])
    assert out["value"] > 0 and out["source_bfs_per_s"] > 0
    secs = 4 / out["source_bfs_per_s"]                  # the reported rate gives the wall time back
    assert abs(out["value"] * 1e9 * secs - edges) <= 0.01 * edges
