#!/usr/bin/env python
"""GTEPS benchmark of the GB300 BVSS breadth-first search.

Default workload: single-source BFS on an R-MAT graph of scale 23 (8,388,608
vertices, edgefactor 16, quadrant probabilities (0.57, 0.19, 0.19, 0.05),
seeded relabel, symmetrised, self-loops and duplicates dropped), reordered
with the compression-oriented ordering, 64 seeded sources from vertices of
degree > 0 timed one at a time.  One step = the 64 traversals.

GTEPS = undirected edges in the reached component / device traversal time
(Graph500 convention); reordering and the BVSS build are timed separately.
The L2 is flushed (a 256 MiB write) before every traversal, outside its CUDA
event pair.

Arms:
  --impl ours       (default) the CUDA path through the C ABI.
  --impl reference  the CPU oracle (plain queue BFS, one thread) on the same
                    workload, a bounded sample of sources per step.
Multi-GPU (torchrun, N > 1): every rank runs the whole step on its own GPU on
its own copy of the graph ("replicas only"; single-source BFS has no sharding
without a per-level exchange), value = all ranks' edges / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GTEPS (1 GB300, bit-exact levels), single vs batched multi-source; % HBM roofline"

WORKLOADS = {
    # name: (kind, size, sources, order, seed_graph, seed_src, msbfs_k)
    "rmat23": ("rmat", 23, 64, "compress", 2, 1002, 0),
    "rmat16": ("rmat", 16, 64, "compress", 1, 1001, 0),
    "rmat21": ("rmat", 21, 64, "compress", 2, 1002, 0),
    "grid4096": ("grid", 4096, 64, "bandwidth", 3, 1003, 0),
    "rmat22-ms64": ("rmat", 22, 64, "compress", 4, 1004, 64),
    "rmat22-ms256": ("rmat", 22, 256, "compress", 4, 1004, 256),
    "rmat22-single": ("rmat", 22, 64, "compress", 4, 1004, 0),
    "batch128": ("batch", 128, 128, "per-kind", 4, 0, 0),
    "serve": ("serve", 16, 0, "per-kind", 5, 0, 0),
    "window-sweep": ("wsweep", 20, 16, "compress", 6, 1006, 0),
    # the sharded single-source traversal, 2 ranks emulated on one GPU (config 2's graph and sources)
    "rmat23-shard2": ("shard", 23, 8, "compress", 2, 1002, 0),
}


# DRAM traffic of the traversal kernel comes from an ncu capture (profiles/),
# valid only for the kernel sources it was taken on: the capture records their
# sha256 and the ratio of DRAM bytes to the algorithmic bytes of its launch.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "bfs_kernel_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2512_21967_gb300", "csrc", f)
                  for f in ("bfs_kernel.cu", "device_common.cuh", "bfs_launch.h")]
MS_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "msbfs_kernel_traffic.txt")
MS_KERNEL_SOURCES = [os.path.join(ROOT, "paper_2512_21967_gb300", "csrc", f)
                     for f in ("msbfs_kernel.cu", "msbfs_launch.h", "msbfs_bits.h", "device_common.cuh")]


def kernel_sources_sha256(sources=None):
    import hashlib
    d = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(f, "rb") as fh:
            d.update(fh.read())
    return d.hexdigest()


def traffic_ratio(path=None, sources=None, workload=None, variant=None):
    """(DRAM bytes per algorithmic byte, note) from a committed ncu capture, or
    (None, why).  A capture file names the kernel sources' hash and holds one ratio
    per workload and kernel variant (`<workload>/<variant>.ratio`, with its
    `.capture` line); a ratio is used only for that workload and variant, and
    only while the kernel sources are the ones captured."""
    try:
        kv = {}
        with open(path or TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha256") != kernel_sources_sha256(sources):
            return None, "kernel sources changed since the ncu capture"
        key = f"{workload}/{variant}"
        if f"{key}.ratio" not in kv:
            return None, f"no capture of the {variant} variant on {workload}"
        return float(kv[f"{key}.ratio"]), kv.get(f"{key}.capture", "")
    except (OSError, KeyError, ValueError):
        return None, "no ncu capture committed"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def build_workload(name, window):
    from paper_2512_21967_gb300 import synth
    kind, size, nsrc, order, sg, ss, k = WORKLOADS[name]
    t0 = time.time()
    if kind == "batch":
        return synth.batch_workload(size, sg), None, order, k, time.time() - t0
    if kind in ("rmat", "shard"):
        g, srcs = synth.rmat_workload(size, nsrc, seed_graph=sg, seed_src=ss)
    else:
        g, srcs = synth.grid_workload(size, nsrc, seed_graph=sg, seed_src=ss)
    return g, srcs, order, k, time.time() - t0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        return parse_clock_samples(out)


def parse_clock_samples(text):
    """The clock record of a timed region from nvidia-smi's CSV samples (the
    fields of ClockSampler.FIELDS, no header, no units): median SM clock, the
    maximum SM clock, every throttle reason seen active in any sample, the sample
    count and the highest power draw.  Lines with unreadable numbers are skipped."""
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm_v, smax_v, power_v = float(f[1]), float(f[2]), float(f[3])
        except ValueError:
            continue
        sm.append(sm_v)
        smax.append(smax_v)
        power.append(power_v)
        for nm, val in zip(names, f[5:9]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
            "samples": len(sm), "power_w_max": float(max(power))}


# ------------------------------------------------------------- byte model

def byte_model(h, g, n):
    """Per-slice-set algorithmic bytes of one stage-1 visit: every VSS of the
    set costs 5 B per unpadded slice (4 B row id + 1 B mask) + 8 B to read its
    queue entry + 8 B to write it one level earlier.  Also returns the vertex
    order (original -> BVSS id) and the number of VSSs of each slice set."""
    import paper_2512_21967_gb300 as blest
    rp = blest.blest_export(h, blest.BLEST_ARRAY_REAL_PTRS).astype(np.int64)
    cnt = blest.blest_export(h, blest.BLEST_ARRAY_VSS_COUNT).astype(np.int64)
    per_vss = 5 * cnt + 16
    pref = np.zeros(len(per_vss) + 1, np.int64)
    pref[1:] = np.cumsum(per_vss)
    w_s = pref[rp[1:]] - pref[rp[:-1]]
    new_id = blest.blest_export(h, blest.BLEST_ARRAY_NEW_ID).astype(np.int64)
    return w_s, new_id, rp[1:] - rp[:-1]


def traversal_bytes(levels_t, new_id_t, w_s_t, nvss_t, nss, n, lazy, output_path, nroots, torch):
    """Algorithmic bytes of one single-source (or multi-root) traversal, from its
    level array in original ids, under the model of the fused kernel:
      init: the level array cleared to -1 (4 B per vertex) and the visited
        bitmaps cleared (V_curr and V_next; eager also its 3 frontier bitmaps);
      stage 1: per level l and slice set s holding a vertex at level l-1, the
        visit bytes of s (5 B per unpadded slice + 16 B per VSS);
      sweeps (level 0, and every processed level when lazy): a dense sweep reads
        V_next and V_curr (8 B per word); a sparse one (queue of at most n/2048
        VSSs, or at most n/2048 roots at level 0) reads only the dirty bitmap
        (4 B per 32 words) and the words holding a newly reached vertex; every
        word holding a newly reached vertex is written back (4 B; eager level 0
        also writes its frontier word);
      level writes: 4 B per reached vertex, plus 4 B for its original id when
        the sweeps write levels straight to the output (output_path 1);
      unpermute (output_path 2: levels kept in BVSS ids): read the order, gather
        L, write the output, 12 B per vertex; nothing when the graph keeps its
        own order (output_path 0, levels written in place).
    Returns (bytes, reached vertices, bytes under the survey's formula with the
    unpermute counted, the same without)."""
    reached = levels_t >= 0
    nreached = int(reached.sum().item())
    lv = levels_t[reached].long()
    r = new_id_t[reached].long()
    s = r >> 3
    nwords = (n + 31) // 32
    cap = nwords >> 6                            # a queue this short takes the sparse sweep
    dirty_read = 4 * ((nwords + 31) // 32)
    key = torch.unique(lv * nss + s)
    stage1 = int(w_s_t[key % nss].sum().item())
    lmax = int(lv.max().item()) if nreached else -1
    # words holding a vertex first reached at level l
    wkey = torch.unique(lv * nwords + (r >> 5))
    words_new = torch.bincount(wkey // nwords, minlength=lmax + 2).cpu().numpy()
    # queue of processed level l = the VSSs of the slice sets holding a vertex at level l - 1
    qn = torch.bincount(key // nss, weights=nvss_t[key % nss].double(), minlength=lmax + 2).cpu().numpy()
    sweep = 0
    for l in range(0, (lmax + 2) if lazy else 1):
        q = nroots if l == 0 else float(qn[l - 1])
        wn = int(words_new[l]) if l < len(words_new) else 0
        sweep += (dirty_read + 8 * wn) if q <= cap else 8 * nwords
        sweep += 4 * wn * (2 if (not lazy and l == 0) else 1)
    init = 4 * n + 4 * nwords * (2 if lazy else 5)
    body = stage1 + sweep + 4 * nreached
    total = init + body + {0: 0, 1: 4 * nreached, 2: 12 * n}[int(output_path)]
    return total, nreached, body + 4 * n + 12 * n, body + 4 * n


def ms_traversal_bytes(levels_t, new_id_t, w_s_t, nvss_t, nss, n, torch):
    """Algorithmic bytes of one multi-source traversal (levels_t: k x n, original
    ids) under the model of the batched kernel, per launch of at most 256
    sources with W = ceil(k/64) words per vertex:
      stage 1, per level l and slice set s holding a vertex first reached at l-1
        by any source: the visit bytes of s (5 B per unpadded slice + 16 B per
        VSS) + its 8 x W frontier words (64 W B);
      sweeps: level 0 and every processed level read V_next, V_curr and write the
        frontier (24 W B per vertex); a level whose queue has at most n/128 VSSs
        sweeps only the slice sets holding a newly reached vertex (8 vertices each);
      levels: 4 B written per (source, vertex) of the output, 8 W + 4 B per
        vertex read by the final pass (visited words, vertex order).  How the
        kernel keeps levels during the traversal (bit planes) is its own
        overhead and is not counted.
    Returns (bytes, reached pairs)."""
    k_all = int(levels_t.shape[0])
    total, pairs_all = 0, 0
    s_of_v = (new_id_t >> 3).long()
    for c0 in range(0, k_all, 256):
        lv_c = levels_t[c0:c0 + 256]
        k = int(lv_c.shape[0])
        W = 1 if k <= 64 else (2 if k <= 128 else 4)
        keys = None
        pairs, lmax = 0, 0
        for i in range(0, k, 8):
            lv = lv_c[i:i + 8]
            reached = lv >= 0
            pairs += int(reached.sum().item())
            if not bool(reached.any()):
                continue
            lmax = max(lmax, int(lv.max().item()))
            kk = torch.unique(lv.long()[reached] * nss + s_of_v.expand_as(lv)[reached])
            keys = kk if keys is None else torch.unique(torch.cat([keys, kk]))
        stage1 = 0
        sweep = 24 * W * n                                   # level 0
        if keys is not None:
            lvl_of = keys // nss
            ss = keys % nss
            stage1 = int(w_s_t[ss].sum().item()) + 64 * W * int(keys.numel())
            qn = torch.bincount(lvl_of, weights=nvss_t[ss].double(), minlength=lmax + 1).cpu().numpy()
            sets = torch.bincount(lvl_of, minlength=lmax + 2).cpu().numpy()
            for l in range(1, lmax + 2):                     # processed levels 1 .. lmax + 1
                if float(qn[l - 1]) * 128 <= n:
                    sweep += 24 * W * 8 * int(sets[l])
                else:
                    sweep += 24 * W * n
        total += stage1 + sweep + 4 * k * n + (8 * W + 4) * n
        pairs_all += pairs
    return total, pairs_all


# ------------------------------------------------------------------ ours

def aggregate_over_ranks(local_ms, local_edges, world, device):
    """Replicas: every rank traversed its own copy; the job's time is the slowest
    rank's and its work is the sum of all ranks' edges."""
    if world <= 1:
        return float(local_ms), float(local_edges)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    e = torch.tensor([float(local_edges)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def run_ours(args):
    import torch

    import paper_2512_21967_gb300 as blest

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if WORKLOADS[args.workload][0] == "batch":
        return run_ours_batch(args, torch, blest, dev, rank, world)
    if WORKLOADS[args.workload][0] == "serve":
        return run_ours_serve(args, torch, blest, dev, rank, world)
    if WORKLOADS[args.workload][0] == "wsweep":
        return run_ours_window_sweep(args, torch, blest, dev, rank, world)
    if WORKLOADS[args.workload][0] == "shard":
        return run_ours_shard(args, torch, blest, dev, rank, world)
    g, srcs, order_name, msk, t_gen = build_workload(args.workload, args.window)
    order = {"compress": blest.BLEST_ORDER_COMPRESS, "bandwidth": blest.BLEST_ORDER_BANDWIDTH,
             "none": blest.BLEST_ORDER_NONE}[order_name]
    t0 = time.time()
    h = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, order, window=args.window)
    t_create = time.time() - t0
    st = blest.blest_get_stats(h)
    udiv_before = None
    if order == blest.BLEST_ORDER_BANDWIDTH:
        # the update divergence of the same graph without reordering (what RCM improves on)
        h0 = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_NONE, window=args.window)
        udiv_before = blest.blest_get_stats(h0)["update_divergence"]
        blest.blest_destroy(h0)
    if args.sources:
        srcs = srcs[:args.sources]
    tune = None
    if args.update != "auto":
        blest.blest_set_option(h, blest.BLEST_OPT_UPDATE,
                               blest.BLEST_UPDATE_EAGER if args.update == "eager" else blest.BLEST_UPDATE_LAZY)
    if args.pull == "mma":
        blest.blest_set_option(h, blest.BLEST_OPT_PULL, blest.BLEST_PULL_MMA)
    if args.blocks_per_sm:
        blest.blest_set_option(h, blest.BLEST_OPT_BLOCKS_PER_SM, args.blocks_per_sm)
    blest.blest_set_option(h, blest.BLEST_OPT_UNROLL, args.unroll)
    blest.blest_set_option(h, blest.BLEST_OPT_MIN_BLOCKS, args.minb)
    blest.blest_set_option(h, blest.BLEST_OPT_VISITED_FILTER, args.filter)
    blest.blest_set_option(h, blest.BLEST_OPT_STAGE_DEPTH, args.depth)
    blest.blest_set_option(h, blest.BLEST_OPT_SCHEDULE, args.sched)
    blest.blest_set_option(h, blest.BLEST_OPT_LAYOUT, args.layout)
    if not args.no_tune and not msk:
        # the autotuner times every kernel variant on 4 of the sources (untimed setup)
        t0 = time.time()
        tune = blest.blest_autotune(h, srcs[:4])
        tune["seconds"] = round(time.time() - t0, 2)
    n = g.n
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)      # flushes, events and traversals all on this stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    deg_t = torch.from_numpy(g.degrees()).to(dev)
    w_s, new_id, nvss = byte_model(h, g, n)
    w_s_t = torch.from_numpy(w_s).to(dev)
    new_id_t = torch.from_numpy(new_id).to(dev)
    nss = (n + 7) // 8

    if msk:
        model = (w_s_t, new_id_t, torch.from_numpy(nvss).to(dev), nss)
        return run_ours_msbfs(args, torch, blest, h, g, srcs, msk, dev, stream, flush, st, t_gen, t_create,
                              rank, world, model)

    out = torch.empty(n, dtype=torch.int32, device=dev)
    edges = np.zeros(len(srcs), np.int64)
    abytes = np.zeros(len(srcs), np.int64)
    abytes_survey = np.zeros((len(srcs), 2), np.int64)
    nvss_t = torch.from_numpy(nvss).to(dev)
    lazy = None
    run_info = None

    def one_step(timed_events=None):
        for i, s in enumerate(srcs):
            flush.fill_(i & 0xFF)
            if timed_events is not None:
                timed_events[i][0].record(stream)
            blest.blest_bfs_device(h, int(s), out, stream=stream)
            if timed_events is not None:
                timed_events[i][1].record(stream)

    # warm-up; the first pass also measures edges and bytes per source
    for w in range(args.warmup):
        if w == 0:
            for i, s in enumerate(srcs):
                blest.blest_bfs_device(h, int(s), out, stream=stream)
                blest.blest_sync(h)
                edges[i] = int((deg_t[out >= 0]).sum().item()) // 2
                if lazy is None:
                    run_info, _ = blest.blest_get_run_info(h)
                    lazy = run_info["update"] == blest.BLEST_UPDATE_LAZY
                abytes[i], _, abytes_survey[i, 0], abytes_survey[i, 1] = traversal_bytes(
                    out, new_id_t, w_s_t, nvss_t, nss, n, lazy, run_info["output_path"], 1, torch)
        else:
            one_step()
    blest.blest_sync(h)
    torch.cuda.synchronize(dev)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid) if rank == 0 else None
    events = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in srcs]
              for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    torch.cuda.nvtx.range_push("timed")    # lets a profiler capture only the timed launches
    for k in range(args.steps):
        one_step(events[k])
    torch.cuda.nvtx.range_pop()
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    blest.blest_sync(h)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    per = np.array([[e[0].elapsed_time(e[1]) for e in step] for step in events])  # ms
    bfs_ms = float(per.sum())
    wall_ms = t_start.elapsed_time(t_end)
    tot_edges = float(edges.sum()) * args.steps
    bfs_ms_max, edges_all = aggregate_over_ranks(bfs_ms, tot_edges, world, dev)
    value = edges_all / (bfs_ms_max / 1e3) / 1e9
    avg_launch_ms = float(per.mean())
    avg_bytes = float(abytes.mean())
    hbm, peak_kind = peaks()
    achieved = avg_bytes / (avg_launch_ms / 1e3) / 1e9
    layout_run = (tune or {}).get("layout", args.layout)
    tr_ratio, tr_note = traffic_ratio(workload=args.workload,
                                      variant=f"{'lazy' if lazy else 'eager'}-layout{layout_run}")

    # end to end through the host-buffer C call
    e2e = None
    if rank == 0 and not args.no_e2e:
        host = np.empty(n, np.int32)
        t0 = time.perf_counter()
        for s in srcs:
            blest.blest_bfs(h, int(s), host)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": float(edges.sum()) / e2e_s / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int(len(srcs) * n * 4),
               "what": "blest_bfs(handle, src, host levels) for the 64 sources, levels copied to host memory"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(g, srcs, args.cpu_sources, edges_of=None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(bfs_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"single-source BFS, {g.name}, {len(srcs)} seeded sources, {order_name} order",
                       "n": g.n, "directed_edges": g.nnz, "sources_per_step": len(srcs),
                       "order": order_name, "window": args.window,
                       "update": "lazy" if lazy else "eager", "pull": ["popc", "mma"][run_info["pull"]],
                       "variant": {k: tune[k] for k in ("unroll", "min_blocks", "visited_filter", "blocks_per_sm",
                                                        "stage_depth", "layout", "schedule")}
                       if tune else {"unroll": args.unroll, "min_blocks": args.minb, "visited_filter": args.filter,
                                     "blocks_per_sm": args.blocks_per_sm, "stage_depth": args.depth,
                                     "layout": args.layout, "schedule": args.sched},
                       "autotune": tune,
                       "grid_blocks": run_info["grid_blocks"],
                       "l2": "flushed by a 256 MiB write before every traversal, outside its event pair",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                         "traffic": round(tr_ratio * avg_bytes) if tr_ratio else None, "traffic_note": tr_note,
                         "kernel": "bfs_kernel (fused persistent traversal)",
                         "bytes_model": "init + stage-1 visits + dense/sparse sweeps + level writes"
                                        + {0: " (in place, no reordering)", 1: " (direct, no unpermute)",
                                           2: " + unpermute"}[run_info["output_path"]],
                         "bytes_survey_with_unpermute": float(abytes_survey[:, 0].mean()),
                         "bytes_survey_without_unpermute": float(abytes_survey[:, 1].mean()),
                         "bytes_per_launch": avg_bytes, "avg_launch_ms": round(avg_launch_ms, 5)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(args.steps * len(srcs)),
            "clocks": clocks,
            "ms_per_step_wall": round(wall_ms / args.steps, 4),
            "bvss": dict({k: st[k] for k in ("num_slice_sets", "num_vss", "num_slices", "unpadded_slices",
                                             "connectivity_bits", "update_divergence", "compression_ratio",
                                             "bvss_bytes")},
                         **({"update_divergence_without_reordering": udiv_before} if udiv_before is not None
                            else {})),
            "preprocess_s": {"generate": round(t_gen, 2), "create_total": round(t_create, 2),
                             "order": round(st["order_seconds"], 2), "build": round(st["build_seconds"], 2)},
            "gteps_per_source_ms": {"min": round(float(per.min()), 4), "median": round(float(np.median(per)), 4),
                                    "max": round(float(per.max()), 4)},
        }
        print(json.dumps(line), flush=True)
    blest.blest_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ours_msbfs(args, torch, blest, h, g, srcs, k, dev, stream, flush, st, t_gen, t_create, rank, world,
                   model):
    n = g.n
    out = torch.empty((k, n), dtype=torch.int32, device=dev)
    deg_t = torch.from_numpy(g.degrees()).to(dev)
    ms_tune = None
    if args.ms_pull != "auto":
        blest.blest_set_option(h, blest.BLEST_OPT_MS_PULL,
                               blest.BLEST_PULL_MMA if args.ms_pull == "mma" else blest.BLEST_PULL_POPC)
    elif not args.no_tune:
        # untimed: pull back-end (CUDA-core / tensor-core), sources per launch, blocks per SM
        t0 = time.time()
        ms_tune = blest.blest_autotune_msbfs(h, srcs[:k])
        ms_tune["seconds"] = round(time.time() - t0, 2)
        ms_tune["pull"] = ["popc", "mma"][ms_tune["pull"]]
    for _ in range(args.warmup):
        blest.blest_msbfs_device(h, srcs[:k], out, stream=stream)
    blest.blest_sync(h)
    edges = int(((out >= 0).to(torch.int64) * deg_t[None, :]).sum().item()) // 2
    w_s_t, new_id_t, nvss_t, nss = model
    ms_bytes, _ = ms_traversal_bytes(out, new_id_t, w_s_t, nvss_t, nss, n, torch)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler() if rank == 0 else None
    evs = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        blest.blest_msbfs_device(h, srcs[:k], out, stream=stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    blest.blest_sync(h)
    clocks = sampler.stop() if sampler else None
    ms = float(sum(e[0].elapsed_time(e[1]) for e in evs))
    value = edges * args.steps / (ms / 1e3) / 1e9
    # the same sources as single-source traversals looped one at a time (autotuned variant)
    loop_srcs = srcs[:min(k, 64)]
    tune = blest.blest_autotune(h, loop_srcs[:4])
    one = torch.empty(n, dtype=torch.int32, device=dev)
    for s_ in loop_srcs[:8]:
        blest.blest_bfs_device(h, int(s_), one, stream=stream)
    torch.cuda.synchronize(dev)
    le = []
    for s_ in loop_srcs:
        flush.fill_(7)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        blest.blest_bfs_device(h, int(s_), one, stream=stream)
        e1.record(stream)
        le.append((e0, e1))
    torch.cuda.synchronize(dev)
    blest.blest_sync(h)
    loop_ms = float(sum(a_.elapsed_time(b_) for a_, b_ in le))
    loop_rate = len(loop_srcs) / (loop_ms / 1e3)
    batched_rate = k * args.steps / (ms / 1e3)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_parallel(g, srcs[:k], 2 * (os.cpu_count() or 1))
    hbm, peak_kind = peaks()
    achieved = ms_bytes / (ms / args.steps / 1e3) / 1e9
    # the variant that ran: the autotuner's choice, else the handle's defaults (CUDA-core
    # pull, 256 sources per launch, V_next test; bit planes on a lazy-update graph)
    msv = ms_tune or {"pull": args.ms_pull if args.ms_pull != "auto" else "popc", "chunk": 256,
                      "visited_filter": 2, "levels": 0}
    ms_levels = msv["levels"] or (2 if st["update"] == blest.BLEST_UPDATE_LAZY else 1)
    ms_ratio, ms_note = traffic_ratio(MS_TRAFFIC_FILE, MS_KERNEL_SOURCES, workload=args.workload,
                                      variant=f"{msv['pull']}-levels{ms_levels}-v{msv['visited_filter']}"
                                              f"-c{msv['chunk']}")
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": f"multi-source BFS k={k}, {g.name}", "n": n, "directed_edges": g.nnz,
                           "k": k, "source_bfs_per_s": round(batched_rate, 2),
                           "single_source_loop_bfs_per_s": round(loop_rate, 2),
                           "batched_over_loop": round(batched_rate / loop_rate, 2),
                           "autotune": ms_tune,
                           "single_source_variant": {kk: tune[kk] for kk in ("update", "unroll", "stage_depth",
                                                                              "visited_filter", "blocks_per_sm")}},
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                             "traffic": round(ms_ratio * ms_bytes) if ms_ratio else None,
                             "traffic_note": ms_note,
                             "kernel": "msbfs_kernel + msbfs_output_kernel (one traversal launch and one "
                                       "output launch per 64-256 sources; the event pair also covers the "
                                       "call's clears and source upload)",
                             "bytes_per_launch": ms_bytes, "avg_launch_ms": round(ms / args.steps, 5)},
                "cpu_baseline": cpu,
                "gpu_launches": args.steps, "clocks": clocks,
                "bvss": {kk: st[kk] for kk in ("num_vss", "unpadded_slices", "compression_ratio")},
                "preprocess_s": {"generate": round(t_gen, 2), "create_total": round(t_create, 2)}}
        print(json.dumps(line), flush=True)
    blest.blest_destroy(h)


def run_ours_batch(args, torch, blest, dev, rank, world):
    """Many graphs of uneven size in one persistent launch: one traversal of their
    disjoint union (one source per graph), captured once as a CUDA graph and
    replayed every step."""
    items, _, _, _, t_gen = build_workload(args.workload, args.window)
    graphs = [it[0] for it in items]
    srcs = [it[1] for it in items]
    orders = [blest.BLEST_ORDER_COMPRESS if it[2] == "rmat" else blest.BLEST_ORDER_BANDWIDTH for it in items]
    t0 = time.time()
    h = blest.blest_batch_create([(g.n, g.row_ptr, g.col_idx) for g in graphs], orders, window=args.window)
    t_create = time.time() - t0
    st = blest.blest_get_stats(h)
    if args.update != "auto":
        blest.blest_set_option(h, blest.BLEST_OPT_UPDATE,
                               blest.BLEST_UPDATE_EAGER if args.update == "eager" else blest.BLEST_UPDATE_LAZY)
    blest.blest_set_option(h, blest.BLEST_OPT_STAGE_DEPTH, args.depth)
    n = sum(g.n for g in graphs)
    tune = None
    if not args.no_tune:
        # untimed: every kernel variant timed as the one multi-root launch the batch runs
        offs = np.concatenate([[0], np.cumsum([g.n for g in graphs])[:-1]]).astype(np.int64)
        t0 = time.time()
        tune = blest.blest_autotune_multiroot(h, (offs + np.asarray(srcs, np.int64)).astype(np.int32))
        tune["seconds"] = round(time.time() - t0, 2)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    blest.blest_batch_graph_capture(h, out)
    deg = torch.from_numpy(np.concatenate([g.degrees() for g in graphs])).to(dev)
    for _ in range(args.warmup):
        blest.blest_batch_graph_launch(h, srcs, stream=stream)
    blest.blest_sync(h)
    edges = int(deg[out >= 0].sum().item()) // 2
    info, _ = blest.blest_get_run_info(h)
    # one multi-root traversal of the union: the single-source byte model applies as it is
    w_s, new_id, nvss = byte_model(h, None, n)
    batch_bytes, _, _, _ = traversal_bytes(out, torch.from_numpy(new_id).to(dev), torch.from_numpy(w_s).to(dev),
                                           torch.from_numpy(nvss).to(dev), (n + 7) // 8, n,
                                           info["update"] == blest.BLEST_UPDATE_LAZY, info["output_path"],
                                           len(srcs), torch)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler() if rank == 0 else None
    evs = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        blest.blest_batch_graph_launch(h, srcs, stream=stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    blest.blest_sync(h)
    clocks = sampler.stop() if sampler else None
    ms = float(sum(e[0].elapsed_time(e[1]) for e in evs))
    value = edges * args.steps / (ms / 1e3) / 1e9
    hbm, peak_kind = peaks()
    achieved = batch_bytes / (ms / args.steps / 1e3) / 1e9
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(achieved / hbm, 4), "peak_kind": peak_kind, "traffic": None,
                             "traffic_note": "no capture of this workload",
                             "kernel": "bfs_kernel over the union of the graphs (one CUDA-graph replay per step)",
                             "bytes_per_launch": batch_bytes, "avg_launch_ms": round(ms / args.steps, 5)},
                "config": {"workload": f"{len(graphs)} graphs of uneven size (R-MAT scale 10..18, grids 64..1024), "
                                       "one source each, one persistent launch replayed as a CUDA graph",
                           "n": n, "directed_edges": int(sum(g.nnz for g in graphs)), "graphs": len(graphs),
                           "levels": info["levels"], "update": ["auto", "eager", "lazy"][info["update"]],
                           "autotune": tune},
                "gpu_launches": args.steps, "clocks": clocks,
                "preprocess_s": {"generate": round(t_gen, 2), "create_total": round(t_create, 2),
                                 "order": round(st["order_seconds"], 2)}}
        print(json.dumps(line), flush=True)
    blest.blest_destroy(h)


def serve_stream(blest, srv, stream):
    """Submit the stream at its arrival times; latency of a query = completion
    time - scheduled arrival (so a lagging client is charged to the server)."""
    import threading
    t0 = time.perf_counter()
    lat = [None] * len(stream)
    tickets = [None] * len(stream)
    submit_at = [0.0] * len(stream)
    lock = threading.Lock()
    done = threading.Event()
    failed = []

    def waiter():
        try:
            for i in range(len(stream)):
                while tickets[i] is None:
                    if failed:
                        return
                    time.sleep(0.0001)
                srv_lat = blest.blest_server_wait(srv, tickets[i], 120.0)
                with lock:
                    lat[i] = (submit_at[i] - stream[i][0]) + srv_lat
        except BaseException as ex:   # a failed query ends the run instead of leaving it waiting
            failed.append(ex)
        finally:
            done.set()

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    try:
        for i, (t_arr, g, srcs) in enumerate(stream):
            if failed:
                break
            now = time.perf_counter() - t0
            if t_arr > now:
                time.sleep(t_arr - now)
            submit_at[i] = time.perf_counter() - t0
            tickets[i] = blest.blest_server_submit(srv, g, srcs, None)
    except BaseException as ex:
        failed.append(ex)
    # every query has a deadline of its arrival + 120 s in the waiter; this bounds the whole run
    if not done.wait(timeout=(stream[-1][0] if stream else 0.0) + 300.0):
        failed.append(TimeoutError("serving run did not finish"))
    if failed:
        raise failed[0]
    wall = time.perf_counter() - t0
    return np.array(lat), wall


def run_ours_serve(args, torch, blest, dev, rank, world):
    """Serving: 16 resident graphs (8 R-MAT, scales 16..22; 8 grids, sides
    256..2048), a Poisson stream of queries (uniform graph, 1..32 uniform
    sources) at several rates, served with continuous batching under a 40 GB
    device-memory cap, against the same stream served one query per launch."""
    items = synth_serving()
    graphs = [it[0] for it in items]
    pools = [it[1] for it in items]
    t0 = time.time()
    handles = [blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx,
                                           blest.BLEST_ORDER_COMPRESS if it[2] == "rmat" else blest.BLEST_ORDER_BANDWIDTH,
                                           window=args.window) for g, it in zip(graphs, items)]
    t_create = time.time() - t0
    results = []
    rates = [float(r) for r in args.rates.split(",")]
    for rate in rates:
        stream = synth_query_stream(args.queries, len(graphs), rate, 55, pools)
        row = {"rate_qps": rate, "queries": len(stream)}
        for mode in ("batched", "one_at_a_time"):
            if mode == "one_at_a_time":
                # the same stream's first queries: one query per launch saturates far below
                # these rates, so the full stream would take many minutes per rate
                stream = stream[:min(len(stream), args.oaat_queries)]
            if mode == "batched":
                srv = blest.blest_server_create(handles, memory_cap_bytes=40 << 30, max_batch_sources=64,
                                                max_inflight=args.serve_inflight, blocks_per_sm=1,
                                                narrow_sms=args.serve_narrow_sms, narrow_levels=256,
                                                long_slots=args.serve_long_slots)
            else:
                srv = blest.blest_server_create(handles, memory_cap_bytes=40 << 30, max_batch_sources=32,
                                                max_inflight=1, blocks_per_sm=0, max_queries_per_launch=1)
            try:
                lat, wall = serve_stream(blest, srv, stream)
                st = blest.blest_server_get_stats(srv)
            finally:
                blest.blest_server_destroy(srv)
            row[mode] = {"queries": len(stream), "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                         "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                         "throughput_qps": round(len(stream) / wall, 2), "launches": st["launches"],
                         "mean_sources_per_launch": round(st["sources_launched"] / max(1, st["launches"]), 2),
                         "memory_peak_gb": round(st["memory_peak"] / 2**30, 2)}
            if mode == "batched":
                # where the tail comes from: latency by graph kind and by graph
                gids = np.array([q[1] for q in stream])
                pct = lambda m, p: round(float(np.percentile(lat[m], p)) * 1e3, 3)
                row[mode]["by_kind"] = {kind: {"queries": int(m.sum()), "p50_ms": pct(m, 50), "p99_ms": pct(m, 99)}
                                        for kind in ("rmat", "grid")
                                        for m in [np.isin(gids, [i for i, it in enumerate(items) if it[2] == kind])]
                                        if m.any()}
                row[mode]["by_graph"] = [{"graph": i, "kind": items[i][2], "n": graphs[i].n,
                                          "queries": int((gids == i).sum()), "p50_ms": pct(gids == i, 50),
                                          "p99_ms": pct(gids == i, 99)}
                                         for i in range(len(graphs)) if (gids == i).any()]
        results.append(row)
    for h in handles:
        blest.blest_destroy(h)
    best = max(r["batched"]["throughput_qps"] for r in results)
    if rank == 0:
        line = {"metric": METRIC, "value": best, "unit": "queries/s", "n_gpus": world, "steps": len(rates),
                "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u64", "data": "synthetic",
                "config": {"workload": "serving: 16 resident graphs (8 R-MAT s16..22, 8 grids 256..2048, p=0.9), "
                                       f"Poisson queries with 1..32 sources, {args.queries} per rate, 40 GB cap",
                           "server": {"max_inflight": args.serve_inflight, "max_batch_sources": 64,
                                      "narrow_sms": args.serve_narrow_sms, "narrow_levels": 256,
                                      "long_slots": args.serve_long_slots or max(1, args.serve_inflight - 1)},
                           "results_copied": "no (levels stay in device memory)"},
                "serving": results, "preprocess_s": {"create_total": round(t_create, 2)}}
        print(json.dumps(line), flush=True)


def run_ours_shard(args, torch, blest, dev, rank, world):
    """The sharded single-source traversal with 2 ranks emulated on one GPU:
    each rank has its own handle of config 2's graph; every level runs rank 0's
    pull, rank 1's pull, the OR merge and both ranks' sweeps in one stream, each
    step timed with CUDA events.  No collective runs (one GPU): the line reports
    the device time of every step, the words a collective would move, and, for
    reference, the fused single-handle traversal of the same sources."""
    from paper_2512_21967_gb300 import shard
    g, srcs, _, _, t_gen = build_workload(args.workload, args.window)
    W = 2
    t0 = time.time()
    h0 = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, blest.BLEST_ORDER_COMPRESS, window=args.window)
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".blest")
    os.close(fd)
    try:
        blest.blest_graph_save(h0, path)
        h1 = blest.blest_graph_load(path)         # the same BVSS and order without a second reordering
    finally:
        os.remove(path)
    t_create = time.time() - t0
    hs = [h0, h1]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    outs = [torch.empty(g.n, dtype=torch.int32, device=dev) for _ in range(W)]
    nw = (g.n + 31) // 32
    merged = torch.empty(nw, dtype=torch.int32, device=dev)
    gathered = torch.empty(W * nw, dtype=torch.int32, device=dev)
    deg_t = torch.from_numpy(g.degrees()).to(dev)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def traverse(src, timed):
        steps = [shard.DeviceShard(h, r, W, int(src), outs[r], stream) for r, h in enumerate(hs)]
        for st in steps:
            st.begin()
        t = {"pull": [0.0] * W, "merge": 0.0, "sweep": [0.0] * W}
        levels = 0
        while True:
            for r, st in enumerate(steps):
                a = ev()
                words = st.pull()
                gathered[r * nw:(r + 1) * nw].copy_(words)      # what the all-gather delivers
                b = ev()
                if timed:
                    b.synchronize()
                    t["pull"][r] += a.elapsed_time(b)
            a = ev()
            blest.blest_shard_merge(merged, gathered, nw, W, stream)
            b = ev()
            more = []
            for r, st in enumerate(steps):
                c = ev()
                blest.blest_shard_sweep(hs[r], merged, stream)
                d = ev()
                more.append(blest.blest_shard_more(hs[r]))
                if timed:
                    t["sweep"][r] += c.elapsed_time(d)
            if timed:
                t["merge"] += a.elapsed_time(b)
            levels += 1
            assert len(set(more)) == 1, "ranks disagree on the end of the traversal"
            if not more[0]:
                return t, levels

    for s_ in srcs[:2]:                                # warm-up
        traverse(s_, False)
    torch.cuda.synchronize(dev)
    tot = {"pull0": 0.0, "pull1": 0.0, "merge": 0.0, "sweep": 0.0}
    edges, nlev = 0, 0
    for s_ in srcs:
        flush.fill_(3)
        t, levels = traverse(s_, True)
        tot["pull0"] += t["pull"][0]
        tot["pull1"] += t["pull"][1]
        tot["merge"] += t["merge"]
        tot["sweep"] += max(t["sweep"])
        nlev += levels
        assert torch.equal(outs[0], outs[1])
        edges += int(deg_t[outs[0] >= 0].sum().item()) // 2
    # the fused single-handle traversal of the same sources, for reference
    fused = 0.0
    for s_ in srcs:
        flush.fill_(5)
        a = ev()
        blest.blest_bfs_device(h0, int(s_), outs[0], stream=stream)
        b = ev()
        b.synchronize()
        fused += a.elapsed_time(b)
    for h in hs:
        blest.blest_destroy(h)
    k = len(srcs)
    emulated_ms = (tot["pull0"] + tot["pull1"] + tot["merge"] + tot["sweep"]) / k
    if rank == 0:
        line = {"metric": METRIC, "value": round(edges / (emulated_ms * k / 1e3) / 1e9, 4), "unit": "GTEPS",
                "n_gpus": world, "steps": 1, "warmup": 2, "ms_per_step": round(emulated_ms * k, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": f"sharded single-source BFS, {g.name}, {k} sources, 2 ranks emulated on one GPU "
                                       "(steps in sequence, no collective)",
                           "n": g.n, "directed_edges": g.nnz, "ranks": W, "levels_per_traversal": nlev / k,
                           "value_is": "edges / the sum of every step's device time (both ranks' pulls in sequence)"},
                "per_traversal_ms": {"pull_rank0": round(tot["pull0"] / k, 4), "pull_rank1": round(tot["pull1"] / k, 4),
                                     "merge": round(tot["merge"] / k, 4), "sweep": round(tot["sweep"] / k, 4),
                                     "fused_single_handle": round(fused / k, 4)},
                "exchange_bytes_per_level_per_rank": nw * 4,
                # per level: each rank's pull and words-out, the merge, each rank's words-in and sweep;
                # per traversal: each rank's root mark and level-0 sweep
                "gpu_launches": int(nlev * (2 * W + 1 + 2 * W) + k * 2 * W),
                "preprocess_s": {"generate": round(t_gen, 2), "create_and_load": round(t_create, 2)}}
        print(json.dumps(line), flush=True)


def run_ours_window_sweep(args, torch, blest, dev, rank, world):
    """Effect of the JaccardWithWindows window w on compression and BFS time (the
    experiment of Fig. 3, here on an R-MAT graph of scale 20): for each w, the
    reordering time, the BVSS compression ratio and the GTEPS of the autotuned
    single-source traversal over 16 sources."""
    from paper_2512_21967_gb300 import synth
    _, scale, nsrc, _, sg, ss, _ = WORKLOADS["window-sweep"]
    g, srcs = synth.rmat_workload(scale, nsrc, seed_graph=sg, seed_src=ss)
    deg_t = torch.from_numpy(g.degrees()).to(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = torch.empty(g.n, dtype=torch.int32, device=dev)
    rows = []
    # each window with the BFS-from-hubs pre-pass; the last entries (g<w>) use the Gorder pre-pass
    for spec in args.windows.split(","):
        prepass = "gorder" if spec.startswith("g") else "hub"
        w = int(spec[1:] if prepass == "gorder" else spec)
        order = blest.BLEST_ORDER_NONE if w == 0 else blest.BLEST_ORDER_COMPRESS
        h = blest.blest_graph_create_ex(g.n, g.row_ptr, g.col_idx, order, window=max(w, 8), prepass=prepass)
        st = blest.blest_get_stats(h)
        blest.blest_autotune(h, srcs[:4])
        w_s, new_id, nvss = byte_model(h, g, g.n)
        w_s_t, new_id_t = torch.from_numpy(w_s).to(dev), torch.from_numpy(new_id).to(dev)
        nvss_t = torch.from_numpy(nvss).to(dev)
        edges, ms, nbytes = 0, 0.0, 0
        for s_ in srcs:
            blest.blest_bfs_device(h, int(s_), out, stream=stream)
        blest.blest_sync(h)
        for s_ in srcs:
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            blest.blest_bfs_device(h, int(s_), out, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms += e0.elapsed_time(e1)
            edges += int(deg_t[out >= 0].sum().item()) // 2
            info, _ = blest.blest_get_run_info(h)
            nbytes += traversal_bytes(out, new_id_t, w_s_t, nvss_t, (g.n + 7) // 8, g.n,
                                      info["update"] == blest.BLEST_UPDATE_LAZY, info["output_path"], 1,
                                      torch)[0]
        blest.blest_sync(h)
        rows.append({"window": w if w else "none", "prepass": prepass if w else None,
                     "order_s": round(st["order_seconds"], 3),
                     "compression_ratio": round(st["compression_ratio"], 4), "num_vss": st["num_vss"],
                     "bfs_ms_mean": round(ms / len(srcs), 4), "gteps": round(edges / (ms / 1e3) / 1e9, 2),
                     "roofline_frac": round(nbytes / (ms / 1e3) / 1e9 / peaks()[0], 4)})
        blest.blest_destroy(h)
    if rank == 0:
        best = max(r["gteps"] for r in rows)
        print(json.dumps({"metric": METRIC, "value": best, "unit": "GTEPS", "n_gpus": world, "steps": len(rows),
                          "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                          "config": {"workload": f"window sweep, {g.name}, {len(srcs)} sources"},
                          "window_sweep": rows}), flush=True)


def synth_serving():
    from paper_2512_21967_gb300 import synth
    return synth.serving_workload()


def synth_query_stream(num, ng, rate, seed, pools):
    from paper_2512_21967_gb300 import synth
    return synth.query_stream(num, ng, rate, seed, pools)


# ------------------------------------------------------------- CPU oracle

def cpu_baseline(g, srcs, nsrc, edges_of=None):
    """The oracle (plain single-threaded queue BFS) timed on the host on the
    first ``nsrc`` sources of the same workload."""
    import oracle
    sample = [int(s) for s in srcs[:nsrc]]
    tot_e, tot_t = 0, 0.0
    for s in sample:
        t0 = time.perf_counter()
        lv = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, s)
        tot_t += time.perf_counter() - t0
        tot_e += oracle.reached_edges(g.row_ptr, lv)
    return {"value": round(tot_e / tot_t / 1e9, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{len(sample)} of the {len(srcs)} sources, one thread, nproc={os.cpu_count()}",
            "seconds": round(tot_t, 2)}


def cpu_baseline_parallel(g, srcs, nsrc, threads=None):
    """The oracle over all host cores, one source per thread (every run is the
    plain queue BFS; threads only split the list of sources): the host baseline
    of the multi-source workloads, on the first ``nsrc`` sources."""
    import oracle
    threads = threads or os.cpu_count() or 1
    sample = np.ascontiguousarray(srcs[:nsrc], dtype=np.int32)
    t0 = time.perf_counter()
    lv = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, sample, threads=threads)
    secs = time.perf_counter() - t0
    edges = sum(oracle.reached_edges(g.row_ptr, lv[i]) for i in range(len(sample)))
    return {"value": round(edges / secs / 1e9, 5), "unit": "GTEPS", "cores": int(min(threads, len(sample))),
            "kind": "oracle", "source_bfs_per_s": round(len(sample) / secs, 3),
            "sample": f"{len(sample)} of the {len(srcs)} sources, one source per thread on {threads} threads, "
                      f"nproc={os.cpu_count()}",
            "seconds": round(secs, 2)}


def reference_jobs(args):
    """The workload of --impl reference as oracle jobs (graph, its sources), with
    the same workload string, unit and size as our arm's line for it."""
    from paper_2512_21967_gb300 import synth
    kind, size, nsrc, order, sg, ss, k = WORKLOADS[args.workload]
    if kind == "batch":
        items = synth.batch_workload(size, sg)
        label = (f"{len(items)} graphs of uneven size (R-MAT scale 10..18, grids 64..1024), "
                 "one source each, one persistent launch replayed as a CUDA graph")
        return [(it[0], [int(it[1])]) for it in items], label, "GTEPS", {"graphs": len(items)}
    if kind == "serve":
        items = synth_serving()
        graphs, pools = [it[0] for it in items], [it[1] for it in items]
        rate = float(args.rates.split(",")[0])
        stream = synth_query_stream(args.queries, len(graphs), rate, 55, pools)
        label = ("serving: 16 resident graphs (8 R-MAT s16..22, 8 grids 256..2048, p=0.9), "
                 f"Poisson queries with 1..32 sources, {args.queries} per rate, 40 GB cap")
        return [(graphs[gq], [int(x) for x in q]) for (_, gq, q) in stream], label, "queries/s", {}
    if kind in ("rmat", "wsweep", "shard"):
        g, srcs = synth.rmat_workload(size, nsrc, seed_graph=sg, seed_src=ss)
    else:
        g, srcs = synth.grid_workload(size, nsrc, seed_graph=sg, seed_src=ss)
    conf = {"n": g.n, "directed_edges": g.nnz}
    if kind == "wsweep":
        label = f"window sweep, {g.name}, {len(srcs)} sources"
    elif k:
        # the multi-source baseline: one source per host thread
        t = os.cpu_count() or 1
        label = f"multi-source BFS k={k}, {g.name}"
        return ([(g, [int(x) for x in srcs[i:i + t]]) for i in range(0, k, t)], label, "GTEPS",
                dict(conf, k=k, threads=t))
    else:
        label = f"single-source BFS, {g.name}, {len(srcs)} seeded sources, {order} order"
    return [(g, [int(x)]) for x in srcs], label, "GTEPS", conf


def run_reference(args):
    """The oracle (plain single-threaded queue BFS, one source at a time, on the
    original vertex order) on a bounded sample of the workload per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    jobs, label, unit, conf = reference_jobs(args)
    threads = conf.get("threads", 1)
    # one serving query, or one source per thread of a multi-source job, per step keeps a step bounded
    per_step = 1 if unit == "queries/s" or threads > 1 else max(1, args.ref_sources)

    def run_job(job):
        g, sources = job
        if threads > 1:
            lv = oracle.msbfs_levels(g.n, g.row_ptr, g.col_idx, np.asarray(sources, np.int32), threads=threads)
            return sum(oracle.reached_edges(g.row_ptr, lv[i]) for i in range(len(sources)))
        e = 0
        for s_ in sources:
            e += oracle.reached_edges(g.row_ptr, oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, s_))
        return e

    for w in range(args.warmup):
        run_job(jobs[w % len(jobs)])
    tot_e, tot_t, done = 0, 0.0, 0
    for k_ in range(args.steps):
        for j in range(per_step):
            t0 = time.perf_counter()
            tot_e += run_job(jobs[(k_ * per_step + j) % len(jobs)])
            tot_t += time.perf_counter() - t0
            done += 1
    value = tot_e / tot_t / 1e9 if unit == "GTEPS" else done / tot_t
    if threads > 1:
        sample = (f"{len(jobs[0][1])} sources per step, one source per thread on {threads} threads, "
                  f"nproc={os.cpu_count()}; the oracle runs on the original vertex order")
    else:
        what = "query" if unit == "queries/s" else "source"
        sample = (f"{per_step} {what}(s) per step, one thread, nproc={os.cpu_count()}; "
                  "the oracle runs on the original vertex order, one source at a time")
    line = {"metric": METRIC, "value": round(value, 5), "unit": unit, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_t / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": dict({"workload": label, "per_step": per_step}, **conf),
            "cpu_baseline": {"value": round(value, 5), "unit": unit, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat23")
    ap.add_argument("--window", type=int, default=4096)
    ap.add_argument("--update", choices=["auto", "eager", "lazy"], default="auto")
    ap.add_argument("--pull", choices=["popc", "mma"], default="popc")
    ap.add_argument("--ms-pull", choices=["auto", "popc", "mma"], default="auto",
                    help="multi-source pull back-end; auto = the multi-source autotuner's choice")
    ap.add_argument("--unroll", type=int, default=2)
    ap.add_argument("--minb", type=int, default=2)
    ap.add_argument("--filter", type=int, default=4,
                    help="visited filter: 0 off, 1 V_curr, 2/3 V_next (L2/L1) while few rows are visited, "
                         "4 V_next (L1) at every level")
    ap.add_argument("--sources", type=int, default=0, help="use only the first N sources of the workload")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner, use the flags as given")
    ap.add_argument("--depth", type=int, default=2,
                    help="lazy stage-1 prefetch: 0 none, 2 register double buffer, 4 or 8 TMA ring stages")
    ap.add_argument("--queries", type=int, default=2000, help="serving: queries per arrival rate")
    ap.add_argument("--rates", default="100,400,1600", help="serving: arrival rates in queries/s")
    ap.add_argument("--serve-inflight", type=int, default=4, help="serving: launches in flight at once")
    ap.add_argument("--serve-long-slots", type=int, default=0,
                    help="serving: launches of long (high-diameter) graphs in flight at once; 0 = inflight - 1")
    ap.add_argument("--serve-narrow-sms", type=int, default=0,
                    help="serving: SMs of a launch on a graph whose last launch ran more than 256 levels (0 = all)")
    ap.add_argument("--oaat-queries", type=int, default=2000,
                    help="serving: queries per rate for the one-query-per-launch comparison")
    ap.add_argument("--windows", default="0,8,64,512,4096,16384,65536,g4096",
                    help="window sweep: JaccardWithWindows windows (0 = no reordering; g<w> = Gorder pre-pass)")
    ap.add_argument("--sched", type=int, default=0, help="stage-1 schedule of depth 2: 0 static, 1 static + dynamic tail")
    ap.add_argument("--layout", type=int, default=0, help="BVSS layout of the lazy register paths: 0 padded, 1 compact")
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--cpu-sources", type=int, default=12)
    ap.add_argument("--ref-sources", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 1:
        args.warmup = 1
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
