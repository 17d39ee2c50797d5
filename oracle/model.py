"""ORACLE (test infrastructure only): BVSS statistics and the per-level replay of
the frontier-aware queue.

* Compression ratio (Section 3.2): m / (numSlices x sigma), numSlices counting
  only non-empty (unpadded) slices -- the fraction of set bits in the masks.
* Update divergence (Section 3.2.1): for each of the slicesPerThread columns of a
  VSS's 32 x slicesPerThread slice-to-thread matrix, the standard deviation of the
  row ids of its non-padded slices; a VSS's divergence is the mean over its
  non-empty columns; U_div is the mean over all VSSs.  "Standard deviation" is
  read as the population standard deviation.
* Lazy/eager rule (Section 5, discussion of Table 3): lazy vertex updates are
  used when U_div exceeds 25,000.
* Queue replay: a VSS is enqueued for level l exactly when its slice set holds
  a column that entered the frontier at level l-1 (Section 3.1.1: only VSSs with
  a nonzero sigma-bit frontier word are processed).  From a correct level array
  (in the BVSS's vertex order) this gives the exact set of VSSs every level
  processes.
"""
from __future__ import annotations

import numpy as np

from .bvss import BVSS, WARP

LAZY_THRESHOLD = 25_000


def compression_ratio(nnz: int, unpadded_slices: int, sigma: int = 8) -> float:
    return float(nnz) / float(unpadded_slices * sigma) if unpadded_slices else 0.0


def update_divergence(b: BVSS) -> float:
    spt = 32 // b.sigma
    tau = b.tau
    per_vss = []
    for nu in range(b.num_vss):
        cnt = int(b.vss_count[nu])
        cols = []
        for q in range(spt):
            rows = [int(b.row_ids[tau * nu + spt * lane + q])
                    for lane in range(WARP) if q * WARP + lane < cnt]
            if rows:
                cols.append(float(np.std(np.asarray(rows, dtype=np.float64))))
        per_vss.append(sum(cols) / len(cols))
    return float(np.mean(per_vss)) if per_vss else 0.0


def use_lazy(u_div: float) -> bool:
    return u_div > LAZY_THRESHOLD


def active_slice_sets(levels_perm: np.ndarray, sigma: int = 8) -> dict[int, np.ndarray]:
    """level l -> sorted slice sets processed at level l (l >= 1), from a level
    array indexed by the BVSS's vertex ids."""
    lv = np.asarray(levels_perm, dtype=np.int64)
    reached = np.nonzero(lv >= 0)[0]
    out: dict[int, set] = {}
    for c in reached.tolist():
        out.setdefault(int(lv[c]) + 1, set()).add(c // sigma)
    return {l: np.array(sorted(s), dtype=np.int64) for l, s in sorted(out.items())}


def queue_sizes(b: BVSS, levels_perm: np.ndarray) -> list[int]:
    """Number of VSSs processed at levels 1, 2, ..., last (the last one finds
    nothing new and ends the traversal)."""
    act = active_slice_sets(levels_perm, b.sigma)
    rp = np.asarray(b.real_ptrs, dtype=np.int64)
    return [int((rp[s + 1] - rp[s]).sum()) for _, s in sorted(act.items())]
