"""Shared helpers of the GPU parity tests (imported by test_gpu_*.py only)."""
import numpy as np

import oracle
import paper_2512_21967_gb300 as blest
from oracle import bvss as ob
from oracle import orderings as oo
from paper_2512_21967_gb300 import synth

ORDERS = {"none": blest.BLEST_ORDER_NONE, "compress": blest.BLEST_ORDER_COMPRESS,
          "bandwidth": blest.BLEST_ORDER_BANDWIDTH}


def csr(n, edges):
    src = np.array([e[0] for e in edges], np.int32)
    dst = np.array([e[1] for e in edges], np.int32)
    return synth.csr_from_edges(n, src, dst)


def oracle_order(g, order, window=65536):
    if order == blest.BLEST_ORDER_NONE:
        return np.arange(g.n, dtype=np.int32)
    if order == blest.BLEST_ORDER_BANDWIDTH:
        return oo.rcm(g.n, g.row_ptr, g.col_idx)
    if order == blest.BLEST_ORDER_COMPRESS:
        return oo.compress_order(g.n, g.row_ptr, g.col_idx, sigma=8, w=window)
    raise ValueError(order)


def oracle_bvss(g, new_id):
    rp, ci = oo.relabel(g.n, g.row_ptr, g.col_idx, new_id)
    return ob.build(g.n, rp, ci)


def export_bvss(h):
    return {
        "real_ptrs": blest.blest_export(h, blest.BLEST_ARRAY_REAL_PTRS),
        "v2r": blest.blest_export(h, blest.BLEST_ARRAY_VIRTUAL_TO_REAL),
        "row_ids": blest.blest_export(h, blest.BLEST_ARRAY_ROW_IDS),
        "masks": blest.blest_export(h, blest.BLEST_ARRAY_MASKS),
        "vss_count": blest.blest_export(h, blest.BLEST_ARRAY_VSS_COUNT),
        "new_id": blest.blest_export(h, blest.BLEST_ARRAY_NEW_ID),
    }


def assert_bvss_equal(got, b):
    assert np.array_equal(got["real_ptrs"], b.real_ptrs)
    assert np.array_equal(got["v2r"], b.virtual_to_real)
    assert np.array_equal(got["vss_count"], b.vss_count)
    assert np.array_equal(got["masks"], b.masks)
    assert np.array_equal(got["row_ids"], b.row_ids)


def check_levels(g, h, srcs):
    for s in srcs:
        exp = oracle.bfs_levels(g.n, g.row_ptr, g.col_idx, int(s))
        got = blest.blest_bfs(h, int(s))
        assert np.array_equal(got, exp), f"levels differ for source {s}"
