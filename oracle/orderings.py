"""ORACLE (test infrastructure only): the two vertex orderings of Section 3.2, in
pure Python for small graphs.  Every function returns ``new_id`` with
``new_id[old] = position of old vertex in the new order`` (the pi^-1 of
Algorithm 1).

Readings where the paper is silent (the product follows the same ones):

* RCM (Section 3.2.1 names it only by citation): each connected component, taken
  in order of its smallest vertex id, is started from a pseudo-peripheral vertex
  found by the George-Liu iteration from that smallest id (repeat: BFS from x;
  y = a vertex of minimum degree, smallest id on ties, in the last level; move to
  y while its eccentricity is larger).  Cuthill-McKee visits the unvisited
  neighbours of each dequeued vertex in ascending (degree, id).  The
  concatenated order is reversed as a whole.
* JaccardWithWindows (Algorithm 1): pop(Q) takes the smallest remaining id;
  argmax ties go to the smallest id; J is compared as an exact rational
  |N(j) & U| / |N(j) | U|, with 0/0 read as 0; the last window may be shorter
  than w and gets ceil(L/sigma) clusters.
* The pre-pass that Section 3.2 takes from Gorder is replaced by a documented
  stand-in (Gorder itself is a third-party algorithm): a BFS visit order that
  starts each component at the highest-degree unvisited vertex (smallest id on
  ties) and scans neighbours in ascending id.  It groups the neighbours of the
  same hub into the same window, which is what the pre-pass is there for.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

import numpy as np


def _adj(n, row_ptr, col_idx):
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    return [ci[rp[v]:rp[v + 1]].tolist() for v in range(n)]


def _bfs_levels(adj, root):
    lvl = {root: 0}
    order = [root]
    q = deque([root])
    while q:
        u = q.popleft()
        for v in adj[u]:
            if v not in lvl:
                lvl[v] = lvl[u] + 1
                order.append(v)
                q.append(v)
    return lvl


def pseudo_peripheral(adj, start) -> int:
    """George-Liu: from x, take y = min-degree (then min id) vertex of the last BFS
    level; continue from y while its eccentricity grows."""
    x = start
    lx = _bfs_levels(adj, x)
    ex = max(lx.values())
    while True:
        last = [v for v, d in lx.items() if d == ex]
        y = min(last, key=lambda v: (len(adj[v]), v))
        ly = _bfs_levels(adj, y)
        ey = max(ly.values())
        if ey > ex:
            x, lx, ex = y, ly, ey
        else:
            return x


def rcm(n: int, row_ptr, col_idx) -> np.ndarray:
    """Reverse Cuthill-McKee, new_id[old]."""
    adj = _adj(n, row_ptr, col_idx)
    seen = [False] * n
    order = []
    for v0 in range(n):
        if seen[v0]:
            continue
        r = pseudo_peripheral(adj, v0)
        seen[r] = True
        q = deque([r])
        while q:
            u = q.popleft()
            order.append(u)
            nb = sorted((v for v in adj[u] if not seen[v]), key=lambda v: (len(adj[v]), v))
            for v in nb:
                seen[v] = True
                q.append(v)
    new_id = np.empty(n, dtype=np.int32)
    for pos, v in enumerate(order):
        new_id[v] = n - 1 - pos
    return new_id


def hub_bfs_prepass(n: int, row_ptr, col_idx) -> np.ndarray:
    """Stand-in pre-pass: BFS visit order, each component rooted at the
    highest-degree unvisited vertex (smallest id on ties), neighbours in
    ascending id.  new_id[old]."""
    adj = _adj(n, row_ptr, col_idx)
    cand = sorted(range(n), key=lambda v: (-len(adj[v]), v))
    seen = [False] * n
    order = []
    for r in cand:
        if seen[r]:
            continue
        seen[r] = True
        q = deque([r])
        while q:
            u = q.popleft()
            order.append(u)
            for v in sorted(adj[u]):
                if not seen[v]:
                    seen[v] = True
                    q.append(v)
    new_id = np.empty(n, dtype=np.int32)
    for pos, v in enumerate(order):
        new_id[v] = pos
    return new_id


def jaccard_windows(n: int, row_ptr, col_idx, sigma: int = 8, w: int = 1 << 16) -> np.ndarray:
    """Algorithm 1 (JaccardWithWindows) on the graph as labelled, new_id[old].
    N(j) is column j of A, i.e. CSR row j for a symmetric graph."""
    if w % sigma != 0 or w <= 0:
        raise ValueError("w must be a positive multiple of sigma")
    adj = [set(a) for a in _adj(n, row_ptr, col_idx)]
    new_id = np.full(n, -1, dtype=np.int64)
    for s_k in range(0, n, w):
        e_k = min(s_k + w, n)
        Q = list(range(s_k, e_k))            # kept sorted; pop(Q) = smallest id
        L_k = e_k - s_k
        M_k = (L_k + sigma - 1) // sigma
        for ell in range(M_k):
            j_star = Q.pop(0)
            new_id[j_star] = s_k + ell * sigma
            U = set(adj[j_star])
            for r in range(1, sigma):
                if not Q:
                    break
                best, best_j = None, None
                for j in Q:                   # ascending id: strict > keeps the smallest on ties
                    inter = len(adj[j] & U)
                    union = len(adj[j] | U)
                    J = Fraction(inter, union) if union else Fraction(0)
                    if best is None or J > best:
                        best, best_j = J, j
                Q.remove(best_j)
                new_id[best_j] = s_k + ell * sigma + r
                U |= adj[best_j]
    return new_id.astype(np.int32)


def compose(first: np.ndarray, second: np.ndarray) -> np.ndarray:
    """new_id of applying ``first`` then ``second`` (both new_id[old])."""
    return np.asarray(second)[np.asarray(first)]


def gorder(n: int, row_ptr, col_idx, w: int = 5, hub_cap: int = 64) -> np.ndarray:
    """Gorder (Wei, Yu, Lu, Lin, SIGMOD 2016), the pre-pass Section 3.2 names,
    restated from its published definition: a greedy permutation that places
    next the unplaced vertex u with the largest score sum over the last w
    placed vertices v of S(u, v) = S_s(u, v) + S_n(u, v), where S_n counts the
    edges between u and v in both directions (2 for an edge of a symmetric
    graph) and S_s the common neighbours of u and v.  Readings: the first
    vertex has the largest degree; ties go to the smallest id; common
    neighbours of degree above hub_cap are not counted (they say little about
    locality and make the score updates quadratic in their degree).  Written
    out directly -- every step scores every unplaced vertex -- for small n.
    new_id[old]."""
    adj = [set(a) for a in _adj(n, row_ptr, col_idx)]
    deg = [len(a) for a in adj]

    def score(u, v):
        s_n = 2 if v in adj[u] else 0
        s_s = sum(1 for x in adj[u] & adj[v] if deg[x] <= hub_cap)
        return s_n + s_s

    order = []
    placed = [False] * n
    for _ in range(n):
        window = order[-w:]
        best, best_key = -1, -1
        for u in range(n):
            if placed[u]:
                continue
            if not order:
                key = deg[u]          # the first vertex: largest degree
            else:
                key = sum(score(u, v) for v in window)
            if key > best_key:        # strict: ties keep the smallest id
                best, best_key = u, key
        placed[best] = True
        order.append(best)
    new_id = np.empty(n, dtype=np.int64)
    for pos, v in enumerate(order):
        new_id[v] = pos
    return new_id


def gorder_objective(n: int, row_ptr, col_idx, new_id, w: int = 5, hub_cap: int = 64) -> int:
    """Gorder's objective F = sum of S(u, v) over vertex pairs at most w apart
    in the order (S as in gorder)."""
    adj = [set(a) for a in _adj(n, row_ptr, col_idx)]
    deg = [len(a) for a in adj]
    order = [0] * n
    for v in range(n):
        order[int(new_id[v])] = v
    total = 0
    for i in range(n):
        for j in range(i + 1, min(n, i + w + 1)):
            u, v = order[i], order[j]
            total += (2 if v in adj[u] else 0) + sum(1 for x in adj[u] & adj[v] if deg[x] <= hub_cap)
    return total


def compress_order(n: int, row_ptr, col_idx, sigma: int = 8, w: int = 1 << 16, prepass: str = "hub") -> np.ndarray:
    """The compression-oriented ordering: pre-pass (the BFS-from-hubs stand-in,
    or Gorder), then Algorithm 1 on the relabelled graph."""
    p = gorder(n, row_ptr, col_idx) if prepass == "gorder" else hub_bfs_prepass(n, row_ptr, col_idx)
    rp2, ci2 = relabel(n, row_ptr, col_idx, p)
    return compose(p, jaccard_windows(n, rp2, ci2, sigma, w))


def relabel(n: int, row_ptr, col_idx, new_id) -> tuple[np.ndarray, np.ndarray]:
    """CSR of the graph with vertex v renamed new_id[v], rows sorted."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    new_id = np.asarray(new_id, dtype=np.int64)
    old_of = np.empty(n, dtype=np.int64)
    old_of[new_id] = np.arange(n)
    deg = np.diff(rp)[old_of]
    rp2 = np.zeros(n + 1, dtype=np.int64)
    rp2[1:] = np.cumsum(deg)
    ci2 = np.empty(len(ci), dtype=np.int64)
    for v_new in range(n):
        v = old_of[v_new]
        ci2[rp2[v_new]:rp2[v_new + 1]] = np.sort(new_id[ci[rp[v]:rp[v + 1]]])
    return rp2.astype(np.int32), ci2.astype(np.int32)


def bandwidth(n: int, row_ptr, col_idx) -> int:
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    return int(np.abs(rows - ci).max()) if len(ci) else 0


def social_like_degrees(deg) -> bool:
    """Section 3.2.1 classifier on a degree sequence (reading 11).

    Heavy-tail sharing: the ceil(n/100) highest-degree vertices hold more than
    5% of all edge endpoints and the ceil(n/10) highest more than 40%.  "More
    than" is strict and exact: 20 * top1 > total and 5 * top10 > 2 * total.
    Power law (the paper gives no numbers; this reading's band): a least-squares
    line through (log d, log #vertices of degree d), over the degrees d >= 1
    that occur, with at least 5 such points, has slope in [-3.5, -1.5] and
    R^2 >= 0.8.  Social-like = either property."""
    deg = np.asarray(deg, dtype=np.int64)
    n = len(deg)
    total = int(deg.sum())
    if n == 0 or total == 0:
        return False
    srt = np.sort(deg)[::-1]
    k1, k10 = max(1, -(-n // 100)), max(1, -(-n // 10))
    top1, top10 = int(srt[:k1].sum()), int(srt[:k10].sum())
    if 20 * top1 > total and 5 * top10 > 2 * total:
        return True
    ds, cnt = np.unique(deg[deg >= 1], return_counts=True)
    if len(ds) < 5:
        return False
    x, y = np.log(ds.astype(np.float64)), np.log(cnt.astype(np.float64))
    vx = ((x - x.mean()) ** 2).sum()
    vy = ((y - y.mean()) ** 2).sum()
    cxy = ((x - x.mean()) * (y - y.mean())).sum()
    if vx <= 0 or vy <= 0:
        return False
    slope, r2 = cxy / vx, cxy * cxy / (vx * vy)
    return bool(-3.5 <= slope <= -1.5 and r2 >= 0.8)


def is_social_like(n: int, row_ptr, col_idx) -> bool:
    """Section 3.2.1 classifier of a CSR graph: its degree sequence (row
    lengths) through social_like_degrees."""
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    assert len(deg) == n
    return social_like_degrees(deg)
