"""ORACLE (test infrastructure only): the BVSS arrays of Section 3.1, built the
slow, obvious way, one slice set at a time.

Definitions followed (Section 3, "BLEST Data Structure", and Section 3.1):

* A is the adjacency matrix of the TRANSPOSED graph (Section 2): row u of A lists
  the vertices u pulls from, so column c of A is the out-neighbour list of c.
  For the symmetric graphs used here, column c of A is CSR row c.
* Columns are cut into intervals of sigma; interval i covers [sigma*i,
  sigma*(i+1)).  A slice is (row u, sigma-bit mask) for one interval, with mask
  bit j = A[u][sigma*i + j]; only nonzero masks exist.  The slices of interval i
  form slice set i.
* A virtual slice set (VSS) holds at most tau = 32 * slicesPerThread slices, all of
  the same slice set (the two rules of Section 3.1).  slicesPerThread = 32 / sigma.
* realPtrs[s] .. realPtrs[s+1] is the VSS range of slice set s; virtualToReal[v]
  is the slice set of VSS v; rowIds has tau entries per VSS; masks has 32 words
  per VSS, each packing slicesPerThread sigma-bit masks.
* Placement (Section 3.1.2): the slices of a VSS sorted by row id; the k-th goes
  to lane k mod 32, sub-slot floor(k / 32).

Readings of the text (where it is silent or garbled):

* Splitting a slice set into VSSs: consecutive chunks of tau slices in sorted row
  order, so only the last VSS of a slice set is partial (consistent with the
  padding paragraph of Section 3.1.2).
* The masks index printed as masks[(tau x nu) + (k mod 32)][floor(k/32)] has 32
  words per VSS, not tau, so it is read as word 32*nu + (k mod 32), sub-field
  floor(k/32); rowIds follow the same lane/sub-slot rule, one 128-bit group of
  four row ids per lane: rowIds[tau*nu + slicesPerThread*(k mod 32) + floor(k/32)].
* Mask bit j (bit 0 = least significant) is column sigma*s + j; sub-field q of a
  mask word occupies bits [sigma*q, sigma*(q+1)).
* Padding row ids ("random, dummy" in the text) are the row id of the last real
  slice of the VSS; their masks are zero, so they never produce a hit.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

WARP = 32


@dataclass
class BVSS:
    n: int
    sigma: int
    real_ptrs: np.ndarray        # int32[ceil(n/sigma)+1]
    virtual_to_real: np.ndarray  # int32[numVSS]
    row_ids: np.ndarray          # int32[numVSS*tau]
    masks: np.ndarray            # uint32[numVSS*32]
    vss_count: np.ndarray        # int32[numVSS]: real (unpadded) slices in each VSS

    @property
    def tau(self) -> int:
        return WARP * (32 // self.sigma)

    @property
    def num_vss(self) -> int:
        return int(self.real_ptrs[-1])

    @property
    def num_slice_sets(self) -> int:
        return len(self.real_ptrs) - 1


def slice_set(n: int, row_ptr, col_idx, s: int, sigma: int = 8) -> list[tuple[int, int]]:
    """Sorted (row u, mask) slices of slice set s: u ranges over every row with a
    nonzero in columns [sigma*s, sigma*s + sigma); bit j of mask = A[u][sigma*s+j]."""
    rows: dict[int, int] = {}
    for j in range(sigma):
        c = sigma * s + j
        if c >= n:
            break
        for u in col_idx[row_ptr[c]:row_ptr[c + 1]]:
            u = int(u)
            rows[u] = rows.get(u, 0) | (1 << j)
    return sorted(rows.items())


def build(n: int, row_ptr, col_idx, sigma: int = 8) -> BVSS:
    """All four static arrays of Section 3.1 for the (symmetric) CSR graph."""
    if 32 % sigma != 0:
        raise ValueError("sigma must divide 32")
    spt = 32 // sigma
    tau = WARP * spt
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    nss = (n + sigma - 1) // sigma
    per_set = [slice_set(n, rp, ci, s, sigma) for s in range(nss)]
    nvss_per_set = [(len(sl) + tau - 1) // tau for sl in per_set]
    real_ptrs = np.zeros(nss + 1, dtype=np.int64)
    real_ptrs[1:] = np.cumsum(nvss_per_set)
    nvss = int(real_ptrs[-1])
    v2r = np.empty(nvss, dtype=np.int32)
    row_ids = np.zeros(nvss * tau, dtype=np.int64)
    masks = np.zeros(nvss * WARP, dtype=np.uint64)
    count = np.zeros(nvss, dtype=np.int32)
    for s, sl in enumerate(per_set):
        for q in range(nvss_per_set[s]):
            nu = int(real_ptrs[s]) + q
            v2r[nu] = s
            chunk = sl[q * tau:(q + 1) * tau]
            count[nu] = len(chunk)
            for k in range(tau):
                lane, sub = k % WARP, k // WARP
                if k < len(chunk):
                    u, m = chunk[k]
                else:
                    u, m = chunk[-1][0], 0           # padding: last real row, zero mask
                row_ids[tau * nu + spt * lane + sub] = u
                masks[WARP * nu + lane] |= np.uint64(m) << np.uint64(sigma * sub)
    return BVSS(n, sigma, real_ptrs.astype(np.int32), v2r, row_ids.astype(np.int32),
                masks.astype(np.uint32), count)


def vss_slices(b: BVSS, nu: int) -> list[tuple[int, int]]:
    """The real (unpadded) slices of VSS nu in placement order k = 0, 1, ..."""
    spt = 32 // b.sigma
    out = []
    for k in range(int(b.vss_count[nu])):
        lane, sub = k % WARP, k // WARP
        u = int(b.row_ids[b.tau * nu + spt * lane + sub])
        m = (int(b.masks[WARP * nu + lane]) >> (b.sigma * sub)) & ((1 << b.sigma) - 1)
        out.append((u, m))
    return out


def unpadded_slices(b: BVSS) -> int:
    return int(b.vss_count.sum())


def slice_set_stats(n: int, row_ptr, col_idx, sigma: int = 8):
    """Per slice set: number of slices (vectorised restatement used on large
    graphs where ``build`` is too slow).  Returns int64[ceil(n/sigma)]."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    nss = (n + sigma - 1) // sigma
    col_of_entry = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    key = (col_of_entry // sigma) * np.int64(n) + ci        # (slice set, row) pairs
    uniq = np.unique(key)
    return np.bincount(uniq // np.int64(n), minlength=nss).astype(np.int64)


@dataclass
class Compact:
    """The compact layout (one reading of Section 3.1.2 against Table 3, whose
    social-graph rows store far fewer slices than 128 per VSS): slices of a
    slice set are packed four to a group in row order, and only the last
    group of each slice set is padded.  A VSS is up to 32 consecutive groups."""
    goff: np.ndarray       # int32[nss + 1]: first group of each slice set
    rows: np.ndarray       # int32[4 * groups]
    masks: np.ndarray      # uint32[groups]: byte q = mask of sub-slot q

    @property
    def groups(self) -> int:
        return int(self.goff[-1])


def compact(n: int, row_ptr, col_idx, sigma: int = 8) -> Compact:
    """Slice k of slice set s (sorted by row) goes to sub-slot k % 4 of group
    goff[s] + k // 4, goff = exclusive prefix sum of ceil(c_s / 4); padded
    sub-slots repeat the last real row with a zero mask.  Built straight from
    the slice sets, not from the padded arrays."""
    spt = 32 // sigma
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    nss = (n + sigma - 1) // sigma
    per_set = [slice_set(n, rp, ci, s, sigma) for s in range(nss)]
    goff = np.zeros(nss + 1, dtype=np.int64)
    goff[1:] = np.cumsum([(len(sl) + spt - 1) // spt for sl in per_set])
    rows = np.zeros(spt * int(goff[-1]), dtype=np.int64)
    masks = np.zeros(int(goff[-1]), dtype=np.uint64)
    for s, sl in enumerate(per_set):
        ng = int(goff[s + 1] - goff[s])
        for k in range(ng * spt):
            g, sub = int(goff[s]) + k // spt, k % spt
            if k < len(sl):
                u, m = sl[k]
            else:
                u, m = sl[-1][0], 0
            rows[spt * g + sub] = u
            masks[g] |= np.uint64(m) << np.uint64(sigma * sub)
    return Compact(goff.astype(np.int32), rows.astype(np.int32), masks.astype(np.uint32))
