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
        total += stage1 + sweep + 4 * k * n + (8 * W + 4) * n
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


def plain_ss_bytes(levels, new_id, w_s, nvss, n, lazy, output_path, nroots):
    """The single-source model written as loops over levels and vertices."""
    nwords = (n + 31) // 32
    sets_at, words_at = {}, {}
    reached = 0
    for v in range(n):
        if levels[v] >= 0:
            reached += 1
            sets_at.setdefault(int(levels[v]), set()).add(int(new_id[v]) // 8)
            words_at.setdefault(int(levels[v]), set()).add(int(new_id[v]) // 32)
    stage1 = sum(int(w_s[s]) for ss in sets_at.values() for s in ss)
    lmax = max(sets_at) if sets_at else -1
    sweep = 0
    for l in range(0, lmax + 2 if lazy else 1):
        queue = nroots if l == 0 else sum(int(nvss[s]) for s in sets_at.get(l - 1, ()))
        new_words = len(words_at.get(l, ()))
        if queue <= nwords // 64:                      # sparse: dirty bitmap + touched words only
            sweep += 4 * ((nwords + 31) // 32) + 8 * new_words
        else:
            sweep += 8 * nwords
        sweep += 4 * new_words * (1 if lazy or l > 0 else 2)
    init = 4 * n + 4 * nwords * (2 if lazy else 5)
    body = stage1 + sweep + 4 * reached
    out = {0: 0, 1: 4 * reached, 2: 12 * n}[output_path]
    return init + body + out, reached, body + 16 * n, body + 4 * n


@pytest.mark.parametrize("output_path", [0, 1, 2])
@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("case", ["rmat", "grid", "fullgrid"])
def test_single_source_byte_model_matches_plain_definition(case, lazy, output_path):
    """The byte model behind the headline roofline, on oracle levels; the grid
    cases have levels whose queue is short enough for the sparse sweep."""
    import bench
    if case == "rmat":
        g = synth.rmat_graph(9, 8, seed=2)
    elif case == "grid":
        g = synth.grid_graph(30, 0.85, seed=3)[0]
    else:
        g = synth.grid_graph(160, 1.0, seed=3)[0]   # n = 25600: queues of <= 12 VSSs are sparse
    src = int(synth.pick_sources(g, 1, seed=4)[0])
    levels = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, src)
    rng = np.random.default_rng(5)
    new_id = rng.permutation(g.n).astype(np.int64) if case != "fullgrid" else np.arange(g.n, dtype=np.int64)
    nss = (g.n + 7) // 8
    w_s = rng.integers(20, 2000, nss)
    nvss = rng.integers(1, 3, nss)
    got = bench.traversal_bytes(torch.from_numpy(levels), torch.from_numpy(new_id), torch.from_numpy(w_s),
                                torch.from_numpy(nvss), nss, g.n, lazy, output_path, 1, torch)
    want = plain_ss_bytes(levels, new_id, w_s, nvss, g.n, lazy, output_path, 1)
    assert got == want
    if case == "fullgrid":
        # some processed levels take the sparse sweep and some the dense one
        cap = ((g.n + 31) // 32) // 64
        queues = [sum(int(nvss[s]) for s in {int(new_id[v]) // 8 for v in np.flatnonzero(levels == l)})
                  for l in range(int(levels.max()) + 1)]
        assert min(queues) <= cap < max(queues)


def test_traffic_ratio_applies_only_to_its_workload_variant_and_sources(tmp_path):
    """A captured DRAM ratio is reported only for the workload and kernel variant it
    was taken on, and only while the kernel sources hash to the captured value."""
    import bench
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel as captured\n")
    cap = tmp_path / "traffic.txt"
    cap.write_text(f"# header: comment lines are skipped\n"
                   f"kernel_sources_sha256: {bench.kernel_sources_sha256([str(src)])}\n"
                   "wl/lazy-layout1.ratio: 0.93\n"
                   "wl/lazy-layout1.capture: one launch\n"
                   "wl/lazy-layout0.ratio: 1.17\n")
    look = lambda w, v: bench.traffic_ratio(str(cap), [str(src)], workload=w, variant=v)
    assert look("wl", "lazy-layout1") == (0.93, "one launch")
    assert look("wl", "lazy-layout0")[0] == 1.17
    assert look("wl", "eager-layout0")[0] is None
    assert look("other", "lazy-layout1")[0] is None
    src.write_text("// kernel changed\n")
    ratio, why = look("wl", "lazy-layout1")
    assert ratio is None and "changed" in why
    assert bench.traffic_ratio(str(tmp_path / "absent.txt"), [str(src)], workload="wl", variant="x")[0] is None


def test_committed_traffic_captures_match_the_kernel_sources():
    """The committed captures are of the kernels as they are now (a kernel change
    must come with a new capture, or the bench lines lose their traffic)."""
    import bench
    assert bench.traffic_ratio(workload="rmat23", variant="lazy-layout1")[0] is not None
    assert bench.traffic_ratio(workload="rmat23", variant="lazy-layout0")[0] is not None
    assert bench.traffic_ratio(bench.MS_TRAFFIC_FILE, bench.MS_KERNEL_SOURCES, workload="rmat22-ms64",
                               variant="popc-levels2-v2-c256")[0] is not None


def test_clock_record_from_nvidia_smi_samples():
    """The clock record that decides whether a timed run is kept: median SM clock,
    every throttle reason active in any sample, unreadable lines skipped."""
    import bench
    idle = "0, 2070, 2070, 210.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1965, 2070, 1398.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1800, 2070, 1200.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active"
    r = bench.parse_clock_samples("\n".join([idle, idle, capped]))
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"] and r["power_w_max"] == 1398.1
    r = bench.parse_clock_samples("\n".join([hot, capped, "0, [N/A], 2070, 5, x, a, b, c, d", "short, line"]))
    assert r["samples"] == 2 and r["sm_mhz"] == (1800.0 + 1965.0) / 2
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.parse_clock_samples("")["reasons"] == ["no samples"]
