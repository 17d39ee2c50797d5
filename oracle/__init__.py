"""CPU oracle for the BLEST breadth-first search -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product (``paper_2512_21967_gb300``)
never imports it, and the oracle imports nothing from the product: the two share
no code.  Inputs for both come from ``paper_2512_21967_gb300.synth``, which holds
no traversal arithmetic.

Contents, each plain and slow on purpose:

* ``bfs_levels`` / ``msbfs_levels`` -- FIFO-queue BFS in plain C
  (``bfs_oracle.c``) on the ORIGINAL vertex order.  Section 2 (Background and
  Notation) defines level[u] as the length of a shortest s -> u path; the method
  computes exactly that, so this is the definition written out.  Pinned by brute
  force (Boolean adjacency powers, n <= 64), closed forms (path, star, cycle,
  grid, complete, disconnected) and the level invariants, in
  ``tests/test_oracle_bfs.py``.
* ``bvss`` -- the BVSS arrays of Section 3.1 (realPtrs, virtualToReal, rowIds,
  masks) built slice set by slice set, and the compact layout (groups of four
  slices, only the last group of a slice set padded).  Pinned by decode round
  trips back to the adjacency, the Figure 1 caption example and the Table 3
  column relations.
* ``bfs_parents`` -- the BFS tree with the smallest-id parent, from the oracle
  levels; pinned by tree invariants and a closed form.
* ``distance_stats`` -- reached count, distance sum and eccentricity per
  source (closeness and diameter, Section 6); pinned by closed forms.
* ``orderings`` -- Reverse Cuthill-McKee (Section 3.2.1) and JaccardWithWindows
  (Algorithm 1) with the pre-pass, in pure Python.  Pinned by closed forms
  (sigma = 1 gives the identity; planted twin groups; path and grid bandwidth).
  The quality of the compression-oriented ordering on the paper's datasets is
  PARITY UNPINNED: those datasets are not available, so only monotone checks
  against a random relabel are possible.
* ``model`` -- compression ratio, update divergence (Section 3.2.1), the
  lazy/eager rule (Section 5, threshold 25,000) and the replay of active virtual
  slice sets per level used for the algorithmic byte count.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc) into ``oracle/_build/liboracle.so``."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_bfs.restype = ctypes.c_int64
            lib.oracle_bfs.argtypes = [ctypes.c_int64, i32p, i32p, ctypes.c_int32, i32p, i32p]
            lib.oracle_bfs_many.restype = ctypes.c_int64
            lib.oracle_bfs_many.argtypes = [ctypes.c_int64, i32p, i32p, ctypes.c_int64, i32p, i32p, ctypes.c_int]
            _lib = lib
    return _lib


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _csr(n, row_ptr, col_idx):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    if rp.shape != (n + 1,):
        raise ValueError("row_ptr must have n+1 entries")
    return rp, ci


def bfs_levels(n: int, row_ptr, col_idx, src: int) -> np.ndarray:
    """int32 level array of a BFS from ``src`` (-1 = unreachable)."""
    rp, ci = _csr(n, row_ptr, col_idx)
    lvl = np.empty(max(n, 1), dtype=np.int32)
    q = np.empty(max(n, 1), dtype=np.int32)
    r = _load().oracle_bfs(n, _p32(rp), _p32(ci), int(src), _p32(lvl), _p32(q))
    if r < 0:
        raise ValueError(f"source {src} out of range [0, {n})")
    return lvl[:n]


def msbfs_levels(n: int, row_ptr, col_idx, srcs, threads: int = 1) -> np.ndarray:
    """k independent BFS runs, result [k, n] (row i = source srcs[i]).  Threads
    only split the list of sources; every run is the plain queue BFS."""
    rp, ci = _csr(n, row_ptr, col_idx)
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    out = np.empty((len(s), max(n, 1)), dtype=np.int32)
    r = _load().oracle_bfs_many(n, _p32(rp), _p32(ci), len(s), _p32(s), _p32(out), int(threads))
    if r < 0:
        raise ValueError("a source is out of range")
    return out[:, :n]


def bfs_parents(n: int, row_ptr, col_idx, src: int) -> tuple[np.ndarray, np.ndarray]:
    """BFS tree in the parent-array form of Section 2 with a unique choice:
    parent[v] = smallest id among the neighbours of v at level[v] - 1;
    parent[src] = src; -1 for unreached vertices.  From the oracle levels."""
    lv = bfs_levels(n, row_ptr, col_idx, src)
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    ok = (lv[rows] >= 1) & (lv[ci] == lv[rows] - 1)
    par = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(par, rows[ok], ci[ok])
    par = np.where(lv < 0, -1, par)
    par[src] = src
    return lv, par.astype(np.int32)


def distance_stats(n: int, row_ptr, col_idx, srcs, threads: int = 1):
    """Per source: (vertices reached, sum of their distances, eccentricity),
    from the oracle levels -- the quantities behind closeness centrality and
    the diameter bound, the multi-source applications named in Section 6."""
    lv = msbfs_levels(n, row_ptr, col_idx, srcs, threads=threads).astype(np.int64)
    ok = lv >= 0
    reached = ok.sum(axis=1).astype(np.int64)
    total = np.where(ok, lv, 0).sum(axis=1).astype(np.int64)
    ecc = np.where(ok, lv, -1).max(axis=1).astype(np.int32) if n > 0 else np.full(len(srcs), -1, np.int32)
    return reached, total, ecc


def reached_edges(row_ptr, levels: np.ndarray) -> int:
    """Undirected edges in the reached component: sum of degrees of reached
    vertices / 2 (Graph500-style TEPS numerator on a loop-free, deduplicated
    symmetric CSR)."""
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    return int(deg[levels >= 0].sum() // 2)
