"""Pins for the Section 3.2.1 social-like classifier (reading 11 of the design
notes): hand-built degree sequences sitting exactly on, and one step beside, each
threshold of the heavy-tail rule, the ceil of the top-1% / top-10% counts, and the
slope band and R^2 bound of the power-law rule.  Each expected value below was
worked out by hand from the sequence (the arithmetic is in the comments), not
by calling the classifier.  The product classifier must agree on simple graphs
that realise the same sequences."""
import numpy as np
import pytest

import paper_2512_21967_gb300 as blest
from oracle import orderings as oo
from paper_2512_21967_gb300 import synth


def seq(groups):
    """groups: list of (count, degree)."""
    return np.concatenate([np.full(c, d, np.int64) for c, d in groups])


def hist(counts):
    """counts: {degree: number of vertices}."""
    return seq([(c, d) for d, c in counts.items()])


# (name, degree sequence, social-like?, what it pins)
HEAVY = [
    # n = 1000: k1 = 10, k10 = 100.  100 x 9 + 900 x 1: total 1800; top 10 hold 90 = exactly 5%
    ("top1_exactly_5pct", seq([(100, 9), (900, 1)]), False),
    # 10 x 10 + 90 x 9 + 900 x 1: total 1810; top 10 hold 100 (5.52%), top 100 hold 910 (50.3%)
    ("top1_just_above", seq([(10, 10), (90, 9), (900, 1)]), True),
    # 10 x 15 + 90 x 5 + 900 x 1: total 1500; top 10 hold 150 (10%), top 100 hold 600 = exactly 40%
    ("top10_exactly_40pct", seq([(10, 15), (90, 5), (900, 1)]), False),
    # 10 x 16 + 90 x 5 + 900 x 1: total 1510; top 100 hold 610 (40.4%)
    ("top10_just_above", seq([(10, 16), (90, 5), (900, 1)]), True),
    # n = 1009: k1 = ceil(10.09) = 11, k10 = ceil(100.9) = 101.  101 x 8 + 908 x 1: total 1716;
    # the top 11 hold 88 (5.13%) but the top 10 only 80 (4.66%); the top 101 hold 808 (47.1%)
    ("ceil_top1", seq([(101, 8), (908, 1)]), True),
    # 11 x 29 + 90 x 10 + 907 x 2 + 1 x 1: total 3034; the top 11 hold 319 (10.5%); the top 101
    # hold 1219 (40.18%) but the top 100 only 1209 (39.85%)
    ("ceil_top10", seq([(11, 29), (90, 10), (907, 2), (1, 1)]), True),
]

POWER = [
    # counts 6400 / d^2 at d = 1, 2, 4, 8, 16: log-log slope exactly -2, R^2 = 1.  Not heavy:
    # n = 8525, total 12400, the top 853 hold 3456 (27.9%)
    ("slope_minus_2", hist({1: 6400, 2: 1600, 4: 400, 8: 100, 16: 25}), True),
    # round(10000 d^-e) at d = 1..5 (one degree-1 vertex added where the total was odd); none is
    # heavy (top 1% < 4%, top 10% < 26%); slopes -1.400, -1.600, -3.399, -3.606, R^2 > 0.99999
    ("slope_minus_1.4", hist({1: 10001, 2: 3789, 3: 2148, 4: 1436, 5: 1051}), False),
    ("slope_minus_1.6", hist({1: 10001, 2: 3299, 3: 1724, 4: 1088, 5: 761}), True),
    ("slope_minus_3.4", hist({1: 10001, 2: 947, 3: 239, 4: 90, 5: 42}), True),
    ("slope_minus_3.6", hist({1: 10000, 2: 825, 3: 192, 4: 68, 5: 30}), False),
    # 3600 d^-2 at d = 1..6, odd degrees x f and even ones / f: slope in the band, R^2 0.924
    # (f = 1.5) and 0.693 (f = 3); not heavy
    ("zigzag_r2_0.92", hist({1: 5400, 2: 600, 3: 600, 4: 150, 5: 216, 6: 67}), True),
    ("zigzag_r2_0.69", hist({1: 10800, 2: 300, 3: 1200, 4: 75, 5: 432, 6: 33}), False),
    # four distinct degrees on a perfect d^-2 line: fewer than 5 points, no fit
    ("four_points", hist({1: 1600, 2: 400, 4: 100, 8: 25}), False),
]


def realise(deg):
    """A simple graph with exactly this degree sequence (Havel-Hakimi with
    buckets by remaining degree), as a symmetric CSR."""
    deg = np.asarray(deg, np.int64)
    n, dmax = len(deg), int(deg.max())
    rem = deg.copy()
    buckets = [set() for _ in range(dmax + 1)]
    for v in range(n):
        buckets[rem[v]].add(v)
    src, dst = [], []
    top = dmax
    while True:
        while top > 0 and not buckets[top]:
            top -= 1
        if top == 0:
            break
        v = min(buckets[top])
        buckets[top].discard(v)
        d, rem[v] = int(rem[v]), 0
        buckets[0].add(v)
        picked, b = [], top
        while len(picked) < d:
            while b > 0 and not buckets[b]:
                b -= 1
            assert b > 0, "sequence is not graphical"
            take = sorted(buckets[b])[:d - len(picked)]
            picked.extend(take)
            b -= 1
        for u in picked:
            buckets[rem[u]].discard(u)
            rem[u] -= 1
            buckets[rem[u]].add(u)
            src.append(v)
            dst.append(u)
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    return synth.csr_from_edges(n, src, dst)


@pytest.mark.parametrize("name,deg,social", HEAVY + POWER, ids=[c[0] for c in HEAVY + POWER])
def test_oracle_classifier_pins(name, deg, social):
    assert oo.social_like_degrees(deg) == social
    # the CSR form reads the same sequence from its row lengths
    rp = np.zeros(len(deg) + 1, np.int64)
    rp[1:] = np.cumsum(deg)
    assert oo.is_social_like(len(deg), rp, np.zeros(int(rp[-1]), np.int32)) == social


def test_classifier_is_order_free():
    for _, deg, social in HEAVY + POWER:
        assert oo.social_like_degrees(synth_shuffle(deg)) == social


def synth_shuffle(deg):
    return deg[synth.permutation(len(deg), 7)]


def _mutant(deg, heavy_cmp, k_round, slope_band, r2_min):
    """The classifier with one planted change: the comparisons, the rounding of
    the top counts, the slope band or the R^2 bound."""
    deg = np.asarray(deg, np.int64)
    n, total = len(deg), int(deg.sum())
    srt = np.sort(deg)[::-1]
    k1, k10 = max(1, k_round(n, 100)), max(1, k_round(n, 10))
    if heavy_cmp(20 * int(srt[:k1].sum()), total) and heavy_cmp(5 * int(srt[:k10].sum()), 2 * total):
        return True
    ds, cnt = np.unique(deg[deg >= 1], return_counts=True)
    if len(ds) < 5:
        return False
    x, y = np.log(ds.astype(float)), np.log(cnt.astype(float))
    cxy = ((x - x.mean()) * (y - y.mean())).sum()
    vx, vy = ((x - x.mean()) ** 2).sum(), ((y - y.mean()) ** 2).sum()
    slope, r2 = cxy / vx, cxy * cxy / (vx * vy)
    return bool(slope_band[0] <= slope <= slope_band[1] and r2 >= r2_min)


def test_planted_mistakes_fail_a_pin():
    gt = lambda a, b: a > b
    ge = lambda a, b: a >= b
    ceil = lambda n, d: -(-n // d)
    floor = lambda n, d: n // d
    cases = HEAVY + POWER
    right = dict(heavy_cmp=gt, k_round=ceil, slope_band=(-3.5, -1.5), r2_min=0.8)
    assert all(_mutant(d, **right) == s for _, d, s in cases), "the unmutated rule must pass every pin"
    for change in (dict(heavy_cmp=ge), dict(k_round=floor), dict(slope_band=(1.5, 3.5)),
                   dict(slope_band=(-3.0, -1.5)), dict(slope_band=(-3.5, -2.0)),
                   dict(slope_band=(-4.0, -1.5)), dict(slope_band=(-3.5, -1.0)), dict(r2_min=0.6)):
        mutated = {**right, **change}
        assert any(_mutant(d, **mutated) != s for _, d, s in cases), f"planted {change} passes every pin"


@pytest.mark.parametrize("name,deg,social", HEAVY + POWER, ids=[c[0] for c in HEAVY + POWER])
def test_product_classifier_matches_pins(name, deg, social):
    g = realise(deg)
    assert np.array_equal(np.sort(np.diff(g.row_ptr)), np.sort(deg))
    assert blest.blest_is_social(g.n, g.row_ptr, g.col_idx) == int(social)
