"""Seeded synthetic graph inputs (R-MAT, 4-neighbour grids) as sorted int32 CSR.

This module holds none of the traversal arithmetic: it only produces graphs and
source lists.  The CPU oracle and the CUDA path both consume what it returns, so
they always see identical inputs.

Every random draw is SplitMix64 used as a counter-based generator
(``draw(seed, i) = mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``); ``draws`` below is
the numpy restatement of the C definition in ``synth.c`` and the two are tested
against each other.

Workload recipes (used by the tests and the benchmark):

* R-MAT, Graph500 quadrant probabilities (A, B, C, D) = (0.57, 0.19, 0.19, 0.05),
  ``edgefactor * 2**scale`` generated edges, a seeded Fisher-Yates relabel,
  symmetrised with self-loops and duplicates dropped.  Stand-in for the
  Kronecker/R-MAT family the paper measures on (GAP-kron, Table 2 and Table 3).
* 2D grid, side x side, 4-neighbour edges each kept with probability p, ids
  randomly permuted.  Stand-in for the road / high-diameter graphs (GAP-road,
  europe_osm).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsynth.so")
_lock = threading.Lock()
_lib = None

GAMMA = np.uint64(0x9E3779B97F4A7C15)
RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_build/libsynth.so`` (host code, gcc)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.synth_draw.restype = ctypes.c_uint64
            lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_rmat_edges.restype = ctypes.c_int
            lib.synth_rmat_edges.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_uint64, i32p, i32p, ctypes.c_int]
            lib.synth_permutation.restype = None
            lib.synth_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, i32p]
            lib.synth_grid_edges.restype = ctypes.c_int64
            lib.synth_grid_edges.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, i32p, i32p]
            lib.synth_build_csr.restype = ctypes.c_int
            lib.synth_build_csr.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p, i32p, i32p,
                                            ctypes.POINTER(i32p), ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
            lib.synth_free.restype = None
            lib.synth_free.argtypes = [ctypes.c_void_p]
            lib.synth_components.restype = None
            lib.synth_components.argtypes = [ctypes.c_int64, i32p, i32p, i32p]
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


# --------------------------------------------------------------------- draws

def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def draws(seed: int, start: int, count: int) -> np.ndarray:
    """SplitMix64 draws ``start .. start+count-1`` of stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(seed) + i * GAMMA)


def bounded(x: np.ndarray, bound: int) -> np.ndarray:
    """Multiply-high map of uint64 draws into [0, bound)."""
    x = np.asarray(x, dtype=np.uint64)
    hi = x >> np.uint64(32)
    lo = x & np.uint64(0xFFFFFFFF)
    b = np.uint64(bound)
    # (x * b) >> 64 computed exactly for bound < 2^32
    assert bound < (1 << 32)
    return ((hi * b) + ((lo * b) >> np.uint64(32))) >> np.uint64(32)


# --------------------------------------------------------------------- graphs

@dataclass
class Graph:
    """Symmetric simple graph as sorted int32 CSR."""
    n: int
    row_ptr: np.ndarray   # int32[n+1]
    col_idx: np.ndarray   # int32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, relabel: np.ndarray | None = None,
                   name: str = "") -> Graph:
    """Symmetrise, drop self-loops and duplicates, sort rows (C, multi-threaded)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    rp = np.empty(n + 1, dtype=np.int32)
    colp = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64(0)
    rl = None
    if relabel is not None:
        relabel = np.ascontiguousarray(relabel, dtype=np.int32)
        rl = _p32(relabel)
    rc = lib.synth_build_csr(n, len(src), _p32(src), _p32(dst), rl, _p32(rp), ctypes.byref(colp),
                             ctypes.byref(nnz), _threads())
    if rc != 0:
        raise RuntimeError(f"synth_build_csr failed with code {rc}")
    try:
        m = nnz.value
        col = np.ctypeslib.as_array(colp, shape=(max(m, 1),))[:m].copy() if m > 0 else np.empty(0, np.int32)
    finally:
        lib.synth_free(ctypes.cast(colp, ctypes.c_void_p))
    return Graph(n, rp, col, name)


def permutation(n: int, seed: int) -> np.ndarray:
    """perm[v] = new label of v (Fisher-Yates driven by SplitMix64)."""
    lib = _load()
    p = np.empty(n, dtype=np.int32)
    lib.synth_permutation(n, seed, _p32(p))
    return p


def rmat_edges(scale: int, m: int, seed: int, abc=RMAT_ABC) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = lib.synth_rmat_edges(scale, m, abc[0], abc[1], abc[2], seed, _p32(src), _p32(dst), _threads())
    if rc != 0:
        raise ValueError("bad R-MAT parameters")
    return src, dst


def rmat_graph(scale: int, edgefactor: int = 16, seed: int = 1, relabel: bool = True) -> Graph:
    """R-MAT on 2^scale vertices, edgefactor*2^scale generated edges, relabelled,
    symmetrised, deduplicated.  Relabel stream = seed + 1 (edges use seed)."""
    n = 1 << scale
    src, dst = rmat_edges(scale, edgefactor * n, seed)
    perm = permutation(n, seed + 1) if relabel else None
    return csr_from_edges(n, src, dst, perm, name=f"rmat-s{scale}-ef{edgefactor}-seed{seed}")


def grid_edges(side: int, p: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    cap = max(1, 2 * side * (side - 1))
    src = np.empty(cap, dtype=np.int32)
    dst = np.empty(cap, dtype=np.int32)
    k = lib.synth_grid_edges(side, p, seed, _p32(src), _p32(dst))
    if k < 0:
        raise ValueError("bad grid side")
    return src[:k], dst[:k]


def grid_graph(side: int, p: float = 0.9, seed: int = 3, relabel: bool = True) -> tuple[Graph, int]:
    """side x side 4-neighbour grid, each edge kept with probability p, ids
    permuted (relabel stream = seed + 1).  Returns (graph, id of corner (0,0))."""
    n = side * side
    src, dst = grid_edges(side, p, seed)
    perm = permutation(n, seed + 1) if relabel else np.arange(n, dtype=np.int32)
    g = csr_from_edges(n, src, dst, perm if relabel else None, name=f"grid-{side}-p{p}-seed{seed}")
    return g, int(perm[0])


def components(g: Graph) -> np.ndarray:
    """comp[v] = smallest vertex id of v's connected component."""
    lib = _load()
    comp = np.empty(g.n, dtype=np.int32)
    lib.synth_components(g.n, _p32(g.row_ptr), _p32(g.col_idx), _p32(comp))
    return comp


def pick_sources(g: Graph, k: int, seed: int, pool: np.ndarray | None = None) -> np.ndarray:
    """k sources drawn uniformly (with repetition) from ``pool`` (default: the
    vertices of degree > 0), draw i -> pool[bounded(draw(seed, i), len(pool))]."""
    if pool is None:
        pool = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    if len(pool) == 0:
        raise ValueError("no eligible source vertex")
    idx = bounded(draws(seed, 0, k), len(pool)).astype(np.int64)
    return pool[idx].astype(np.int32)


def largest_component_pool(g: Graph) -> np.ndarray:
    comp = components(g)
    labels, counts = np.unique(comp, return_counts=True)
    big = labels[np.argmax(counts)]
    return np.nonzero(comp == big)[0].astype(np.int32)


# ------------------------------------------------------------------ workloads

def rmat_workload(scale: int, nsrc: int = 64, seed_graph: int = 1, seed_src: int = 1001):
    g = rmat_graph(scale, 16, seed_graph)
    return g, pick_sources(g, nsrc, seed_src)


def grid_workload(side: int, nsrc: int = 64, p: float = 0.9, seed_graph: int = 3, seed_src: int = 1003):
    g, corner = grid_graph(side, p, seed_graph)
    pool = largest_component_pool(g)
    srcs = np.concatenate([[corner], pick_sources(g, nsrc, seed_src, pool)]).astype(np.int32)
    return g, srcs


def batch_workload(num: int = 128, seed: int = 4, rmat_scales=(10, 18), grid_sides=(64, 1024)):
    """Many graphs of uneven size: even indices are R-MAT graphs with scale drawn
    uniformly from rmat_scales (inclusive, edgefactor 16), odd indices are grids
    with side drawn uniformly from grid_sides (inclusive, keep probability 0.9).
    Graph i uses stream seed*1000 + i; its size is draw i of stream `seed`; its one
    source is draw 0 of stream seed*1000 + 500 + i over its largest component
    (grids) or its degree > 0 vertices (R-MAT).  Returns [(graph, source, kind)]."""
    sz = draws(seed, 0, num)
    out = []
    for i in range(num):
        gs = seed * 1000 + i
        if i % 2 == 0:
            lo, hi = rmat_scales
            scale = lo + int(bounded(sz[i:i + 1], hi - lo + 1)[0])
            g = rmat_graph(scale, 16, gs)
            src = int(pick_sources(g, 1, seed * 1000 + 500 + i)[0])
            out.append((g, src, "rmat"))
        else:
            lo, hi = grid_sides
            side = lo + int(bounded(sz[i:i + 1], hi - lo + 1)[0])
            g, _ = grid_graph(side, 0.9, gs)
            src = int(pick_sources(g, 1, seed * 1000 + 500 + i, largest_component_pool(g))[0])
            out.append((g, src, "grid"))
    return out


def serving_workload(seed: int = 5, rmat_scales=(16, 22), grid_sides=(256, 2048), num_rmat: int = 8,
                     num_grid: int = 8):
    """Resident graph set of the serving workload: num_rmat R-MAT graphs with
    scales spread evenly over rmat_scales and num_grid grids with sides spread
    evenly over grid_sides (keep probability 0.9); graph i uses stream
    seed*1000 + i.  Returns [(graph, source pool, kind)]."""
    out = []
    for i in range(num_rmat):
        scale = rmat_scales[0] + round(i * (rmat_scales[1] - rmat_scales[0]) / max(1, num_rmat - 1))
        g = rmat_graph(scale, 16, seed * 1000 + i)
        out.append((g, np.nonzero(g.degrees() > 0)[0].astype(np.int32), "rmat"))
    for i in range(num_grid):
        side = grid_sides[0] + round(i * (grid_sides[1] - grid_sides[0]) / max(1, num_grid - 1))
        g, _ = grid_graph(side, 0.9, seed * 1000 + num_rmat + i)
        out.append((g, largest_component_pool(g), "grid"))
    return out


def query_stream(num: int, num_graphs: int, rate: float, seed: int, pools, max_sources: int = 32):
    """Poisson stream: query i arrives at the sum of i+1 exponential gaps of mean
    1/rate (inverse CDF of draw 3i of stream `seed`), targets graph
    bounded(draw 3i+1, num_graphs) and has 1 + bounded(draw 3i+2, max_sources)
    sources drawn from that graph's pool (stream seed + 1 + i)."""
    d = draws(seed, 0, 3 * num)
    u = (d[0::3] >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    gaps = -np.log1p(-u) / rate
    t = np.cumsum(gaps)
    gi = bounded(d[1::3], num_graphs).astype(np.int64)
    ks = 1 + bounded(d[2::3], max_sources).astype(np.int64)
    out = []
    for i in range(num):
        pool = pools[gi[i]]
        idx = bounded(draws(seed + 1 + i, 0, int(ks[i])), len(pool)).astype(np.int64)
        out.append((float(t[i]), int(gi[i]), pool[idx].astype(np.int32)))
    return out
