"""Pins of the oracle's communication amounts and transpose-order analysis
against what the paper prints: Table 1, the best-order lists, the worst/best
ratios of Sec. 3.1 and 3.3, the comparison claims of Sec. 4, and the closed
form of the 1-D (slab) method.  CPU only."""

import json
import math
import os

import numpy as np
import pytest

import oracle

with open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed.json")) as _f:
    PAPER = json.load(_f)


def test_table1_counts_by_enumeration():
    t1 = PAPER["table1_order_cases"]
    for M in (2, 3, 4, 5):
        assert oracle.count_orders(M) == t1[str(M)]
    # 6-D is too many to enumerate; the printed value equals (M-1)!^M.
    assert math.factorial(5) ** 6 == t1["6"]


def test_enumerated_orders_are_valid_and_distinct():
    for M in (2, 3, 4):
        orders = oracle.enumerate_orders(M)
        seen = set()
        for o in orders:
            assert list(o[0]) == list(range(M))                  # natural first layout
            assert sorted(o[:, -1].tolist()) == list(range(M))    # every axis transformed once
            for L in o:
                assert sorted(L.tolist()) == list(range(M))
            seen.add(o.tobytes())
        assert len(seen) == len(orders)


def _ratio(N, M, P):
    r = oracle.order_search([N] * M, P, best_cap=1)
    return r["worst"] / r["best"], r


def _pow2(lo, hi):
    return [2 ** k for k in range(1, 40) if lo <= 2 ** k <= hi]


@pytest.mark.parametrize("N", [16, 64])
def test_3d_worst_over_best(N):
    # Reading: process counts are powers of two, as every count the paper
    # names is (Np = N + 1 gives uneven chunks and a larger ratio).
    w = PAPER["worst_over_best"]
    for P in _pow2(2, N):
        assert _ratio(N, 3, P)[0] == w["3d_upto_N"]
    mid = [_ratio(N, 3, P)[0] for P in _pow2(N + 1, N * N)]
    assert round(max(mid), 1) == w["3d_N_to_N2_max"]


def test_3d_best_set_in_1d_regime_is_the_papers_four():
    listed = sorted(PAPER["best_orders_3d"]["orders"])
    for N, P in [(8, 2), (8, 4), (16, 16), (32, 4)]:
        r = oracle.order_search([N] * 3, P)
        assert sorted(r["best_orders"]) == listed
        # 1-D regime: the best amount is the slab method's A_1D = N^3 - N^3 / Np (Sec. 4)
        assert r["best"] == oracle.amount_slab(N, P)


def test_3d_known_discrepancy_in_2d_regime():
    # In the 2-D regime the four listed orders split into two pairs; the
    # prior-work order abc->cab->cba is in the slightly worse pair.
    listed = PAPER["best_orders_3d"]["orders"]
    tot = {o: oracle.comm_volume([8, 8, 8], 16, o)["total"] for o in listed}
    best = oracle.order_search([8, 8, 8], 16)["best"]
    assert tot["abc->acb->bca"] == tot["abc->cba->cab"] == best
    assert tot["abc->acb->cba"] == tot["abc->cab->cba"] > best


def test_fig2_order_awareness_doubles_in_1d_regime():
    f2 = PAPER["fig2_orders"]
    for N, P in [(8, 2), (8, 8), (16, 4), (12, 6)]:
        a = oracle.comm_volume([N] * 3, P, f2["aware"])["total"]
        u = oracle.comm_volume([N] * 3, P, f2["unaware"])["total"]
        assert u == f2["ratio"] * a


def test_4d_worst_over_best_and_best_set():
    w = PAPER["worst_over_best"]
    N = 16
    for P in (2, 4, 16, 64, 128, 256):
        assert _ratio(N, 4, P)[0] == w["4d_upto_N2"]
    upper = [_ratio(N, 4, P)[0] for P in (512, 1024, 2048, 4096)]
    assert max(upper) == w["4d_N2_to_N3_max"]
    listed = sorted(PAPER["best_orders_4d"]["orders"])
    for P in (64, 128, 256):  # 2-D regime: the listed four are exactly the best set
        assert sorted(oracle.order_search([N] * 4, P)["best_orders"]) == listed


def test_5d_worst_over_best_and_96_orders():
    w = PAPER["worst_over_best"]
    N = 8
    for P in (2, 8, 64):
        assert _ratio(N, 5, P)[0] == w["5d_upto_N2"]
    lo, hi = w["5d_N2_to_N3_range"]
    for P in (128, 256, 512):
        assert lo <= round(_ratio(N, 5, P)[0], 1) <= hi
    for P in (1024, 2048, 4096):
        assert round(_ratio(N, 5, P)[0], 1) <= w["5d_N3_to_N4_max"]
    listed = PAPER["best_orders_5d"]["orders"]
    r = oracle.order_search([N] * 5, N ** 3, best_cap=200)
    assert r["n_best"] == PAPER["best_orders_5d"]["count"]
    # Known discrepancy: at Np = N^3 only the last two listed orders are in
    # the 96-order best set; all four are best up to Np = N^2.
    assert listed[2] in r["best_orders"] and listed[3] in r["best_orders"]
    assert listed[0] not in r["best_orders"] and listed[1] not in r["best_orders"]
    for P in (8, 64):
        best = oracle.order_search([N] * 5, P, best_cap=1)["best"]
        assert all(oracle.comm_volume([N] * 5, P, o)["total"] == best for o in listed)


def test_closed_form_best_and_worst_for_cubes():
    # Np dividing N^floor(M/2): best = T (1 - 1/Np) (= A_1D for M = 3),
    # worst = (M - 1) times that (the 2x / 3x / 4x of Sec. 3.1 and 3.3).
    for M, N, Ps in [(3, 6, (2, 3, 6)), (4, 4, (2, 4, 8, 16)), (5, 4, (2, 4, 16))]:
        T = N ** M
        for P in Ps:
            r = oracle.order_search([N] * M, P, best_cap=1)
            assert r["best"] * P == T * (P - 1)
            assert r["worst"] == (M - 1) * r["best"]


def _ours(N, M, P):
    r = oracle.order_search([N] * M, P, best_cap=1)
    return oracle.comm_volume([N] * M, P, r["best_order"])["paper_total"]


def test_comparison_64cubed_vs_pencil_and_volumetric():
    c = PAPER["comparison_64cubed"]
    N = 64
    lo, hi = c["better_than_2d_percent_range"]
    better = {P: 100.0 * (oracle.amount_pencil(N, P) / _ours(N, 3, P) - 1.0) for P in (16, 32, 64)}
    assert round(better[16], 1) == lo
    assert round(better[64], 1) == hi
    assert all(lo <= round(v, 1) <= hi for v in better.values())
    for P in (c["gap_to_2d_zero_from_P"], c["pencil_limit_P"]):
        assert abs(oracle.amount_pencil(N, P) / _ours(N, 3, P) - 1.0) < 2e-3
    # beyond the pencil limit only volumetric decompositions apply
    vs3 = {P: oracle.amount_volumetric(3, N, P) / _ours(N, 3, P)
           for P in [2 ** k for k in range(13, 19)]}
    best_P = max(vs3, key=vs3.get)
    assert best_P == c["vs_3d_max_at_P"]
    assert round(vs3[best_P], 1) == c["vs_3d_max"]


def test_comparison_16_4d():
    c = PAPER["comparison_16_4d_5d"]
    N = 16
    r4 = max(oracle.amount_volumetric(4, N, P) / _ours(N, 4, P) for P in [2 ** k for k in range(1, 17)])
    assert round(r4) == c["vs_4d_max_approx"]


def test_comparison_16_5d_with_listed_orders():
    # 16^5 is too large for the exhaustive search; the paper's listed orders
    # are used as "ours" (they are best up to Np = N^3, see the 5-D test).
    c = PAPER["comparison_16_4d_5d"]
    N = 16
    listed = PAPER["best_orders_5d"]["orders"]
    ratios = {}
    for P in [2 ** k for k in range(4, 13)]:
        ours = min(oracle.comm_volume([N] * 5, P, o)["paper_total"] for o in listed)
        ratios[P] = oracle.amount_volumetric(5, N, P) / ours
    assert round(max(ratios.values()), 1) == c["vs_5d_max"]


def test_split_line_term_only_in_md_regime():
    N = (4, 4, 4)
    for P in range(1, 65):
        for layout in ("abc", "cab", "bca"):
            s = oracle.split_line(N, P, layout)
            if P <= 16:
                assert s == 0
            elif 64 % P == 0:
                assert s == 64 * (P // 16 - 1)  # every line cut into Np / 16 equal pieces
