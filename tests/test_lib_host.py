"""The C-ABI library on the host: it loads, exports every entry point the
header declares, and its planner (box intersection, dynamic-programming
order search) matches the oracle (owner arrays, exhaustive enumeration)
bit for bit.  No GPU: plans are made with MDFFT_PLAN_HOST_ONLY."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1302_6189_gb300 as md

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST = md.MDFFT_PLAN_HOST_ONLY


def test_library_exports_every_declared_symbol():
    with open(os.path.join(ROOT, "include", "mdfft.h")) as f:
        header = f.read()
    declared = set(re.findall(r"\b(mdfft_[a-z_0-9]+)\s*\(", header))
    assert len(declared) >= 15
    lib = ctypes.CDLL(md.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(md.mdfft.SIGNATURES)


def _plan(N, P, order=None):
    return md.mdfft_plan(N, P, order, "c64", HOST)


def _cv(N, P, order):
    h = _plan(N, P, order)
    try:
        return md.mdfft_comm_volume(h, len(N))
    finally:
        md.mdfft_destroy(h)


ORDERS3 = [oracle.format_order(o) for o in oracle.enumerate_orders(3)]


@pytest.mark.parametrize("N", [(4, 5, 6), (8, 8, 8), (6, 3, 10), (16, 4, 9)])
def test_comm_volume_matches_oracle_every_3d_order(N):
    T = int(np.prod(N))
    Ps = sorted({1, 2, 3, N[0], N[0] + 1, N[0] * N[1], N[0] * N[1] + 1, T // 3, T - 1, T})
    for order in ORDERS3:
        for P in Ps:
            got, ref = _cv(N, P, order), oracle.comm_volume(N, P, order)
            for key in ("per_transition", "total", "final_to_natural", "split_line", "paper_total"):
                assert got[key] == ref[key], (order, P, key)


def test_comm_volume_matches_oracle_4d_5d():
    rng = np.random.default_rng(44)
    for M in (4, 5):
        orders = oracle.enumerate_orders(M, cap=5000)
        for _ in range(12):
            N = tuple(int(v) for v in rng.integers(2, 6, size=M))
            T = int(np.prod(N))
            P = int(rng.integers(1, T + 1))
            o = orders[rng.integers(0, len(orders))]
            got, ref = _cv(N, P, o), oracle.comm_volume(N, P, o)
            assert got["per_transition"] == ref["per_transition"]
            assert got["final_to_natural"] == ref["final_to_natural"]
            assert got["split_line"] == ref["split_line"]


def test_regimes_and_closed_forms():
    got = _cv((64, 64, 64), 8192, "abc->acb->bca")
    assert got["regime"] == [3, 3, 3]
    assert got["amount_slab"] == pytest.approx(oracle.amount_slab(64, 8192))
    assert got["amount_pencil"] == pytest.approx(oracle.amount_pencil(64, 8192))
    assert got["amount_volumetric"] == pytest.approx(oracle.amount_volumetric(3, 64, 8192))
    # the 256^3 configuration names P = 16, 256, 4096 as three regimes; f_3D gives 1, 1, 2
    for P, k in ((16, 1), (256, 1), (4096, 2), (131072, 3)):
        assert _cv((256, 256, 256), P, "abc->cab->cba")["regime"][0] == k


@pytest.mark.parametrize("N,P", [((4, 6, 5), 7), ((8, 8, 8), 16), ((3, 4, 2, 5), 11), ((2, 3, 2, 3, 2), 9)])
def test_chunks_match_oracle_in_every_layout(N, P):
    M = len(N)
    h = _plan(N, P)
    try:
        order = md.mdfft_plan_order(h, M)
        for step in range(M + 1):
            L = order[step] if step < M else list(range(M))
            Nl = [N[a] for a in L]
            for pid in range(P):
                assert md.mdfft_chunk(h, step, pid, M) == oracle.chunk(Nl, P, pid)
    finally:
        md.mdfft_destroy(h)


@pytest.mark.parametrize("N,Ps", [((8, 8, 8), (2, 8, 16, 40, 64, 100, 512)),
                                  ((6, 4, 5), (3, 6, 7, 24, 25, 120)),
                                  ((4, 4, 4, 4), (2, 4, 16, 32, 64, 200)),
                                  ((3, 4, 2, 3), (5, 12, 13, 30)),
                                  ((3, 3, 3, 3, 3), (2, 9, 27, 81, 100))])
def test_order_search_matches_exhaustive_oracle(N, Ps):
    for P in Ps:
        ref = oracle.order_search(N, P, best_cap=1)
        best_order, best = md.mdfft_order_search(N, P, 0)
        worst_order, worst = md.mdfft_order_search(N, P, 1)
        assert (best, worst) == (ref["best"], ref["worst"])
        assert best_order == ref["best_order"]      # same tie-break: lexicographically first
        assert worst_order == ref["worst_order"]
        # a plan made without an order uses the best one
        h = _plan(N, P)
        try:
            assert md.mdfft_plan_order(h, len(N)) == ref["best_order"]
        finally:
            md.mdfft_destroy(h)


def test_errors_are_status_codes():
    with pytest.raises(md.MdfftError) as e:
        _plan((8, 8, 8), 16, "acb->cab->cba")
    assert e.value.status == -2
    with pytest.raises(md.MdfftError) as e:
        _plan((8, 8, 8), 16, "abc->cab->cab")
    assert e.value.status == -2
    with pytest.raises(md.MdfftError) as e:
        _plan((2, 2, 2), 9)
    assert e.value.status == -3
    with pytest.raises(md.MdfftError) as e:
        _plan((2, 2, 2), 0)
    assert e.value.status == -3
    with pytest.raises(md.MdfftError) as e:
        md.mdfft_plan((8,), 2, None, "c64", HOST)
    assert e.value.status == -7
    with pytest.raises(md.MdfftError) as e:
        md.mdfft_plan((8, 0, 8), 2, None, "c64", HOST)
    assert e.value.status == -1
    h = _plan((8, 8, 8), 4)
    try:
        with pytest.raises(md.MdfftError) as e:
            md.mdfft_exec(h, 16, 32, -1, 0, 0)        # host-only plans never launch
        assert e.value.status == -1
        with pytest.raises(md.MdfftError):
            md.mdfft_chunk(h, 4, 0, 3)
        with pytest.raises(md.MdfftError):
            md.mdfft_chunk(h, 0, 4, 3)
    finally:
        md.mdfft_destroy(h)


def test_supported_lengths():
    for n in (1, 2, 3, 5, 24, 48, 64, 96, 160, 192, 256, 512, 1024):
        assert md.mdfft_supported_length(n, "c64") and md.mdfft_supported_length(n, "c128")
    for n in (7, 11, 2048, 0, -4):
        assert not md.mdfft_supported_length(n, "c64")


@pytest.mark.parametrize("N,Ps", [((8, 8, 8, 8), (2, 16, 64, 100, 512)), ((4, 4, 4, 4, 4), (2, 16, 64, 200)),
                                  ((3, 4, 2, 3), (5, 12, 30)), ((6, 4, 5), (3, 12, 40))])
def test_balanced_split_heuristic_against_exhaustive(N, Ps):
    # Sec. 3.3's balanced two-part form: equal to the exhaustive optimum in
    # the low regimes for cubes, never below it, always a valid order
    for P in Ps:
        order, total = md.mdfft_order_heuristic(N, P)
        ref = oracle.order_search(N, P, best_cap=1)
        assert total >= ref["best"]
        assert oracle.comm_volume(N, P, order)["total"] == total
        M = len(N)
        assert order[0] == list(range(M)) and sorted(L[-1] for L in order) == list(range(M))
        if len(set(N)) == 1 and P <= N[0] ** (M // 2) and N[0] ** (M // 2) % P == 0:
            assert total == ref["best"]


def test_heuristic_for_six_to_eight_dims():
    # (M-1)!^M orders are too many from M = 6 on (Table 1); in the low regime
    # of a cube the heuristic reaches the closed-form optimum T (1 - 1/P)
    for M, n, Ps in [(6, 4, (2, 4, 16, 64)), (7, 2, (2, 4, 8)), (8, 2, (2, 4, 16))]:
        N = (n,) * M
        T = n ** M
        for P in Ps:
            order, total = md.mdfft_order_heuristic(N, P)
            assert total * P == T * (P - 1)
            assert oracle.comm_volume(N, P, order)["total"] == total
    # without an order, plans of 7-8 dims use it (6 dims: the exact search below)
    for N in [(2, 2, 3, 2, 2, 2, 2), (2,) * 8]:
        h = md.mdfft_plan(N, 4, None, "c64", HOST)
        try:
            assert md.mdfft_plan_order(h, len(N)) == md.mdfft_order_heuristic(N, 4)[0]
        finally:
            md.mdfft_destroy(h)


@pytest.mark.parametrize("N,P,ratio", [((4,) * 6, 4, 1.0), ((4,) * 6, 64, 1.0), ((4,) * 6, 256, 1.325),
                                       ((4,) * 6, 1024, 1.0625), ((2, 3, 4, 2, 3, 4), 50, 1352 / 1187),
                                       ((6, 4, 5, 3, 4, 2), 100, 1.0), ((8,) * 6, 64, 1.0)])
def test_exact_six_dim_search_against_the_heuristic(N, P, ratio):
    # 6 dims: 120^6 = 3e12 orders (Table 1) rule out enumeration, but the
    # dynamic programme over (step, layout, transformed axes) finds the
    # optimum.  Its order's amount is recounted point by point by the oracle
    # (owner arrays, brute force), it is never above the heuristic's, it
    # reaches the closed form T (1 - 1/P) in a cube's low regime, and above
    # the low regimes it shows the heuristic is not optimal (ratio recorded)
    order, total = md.mdfft_order_search(N, P, 0)
    assert oracle.comm_volume(N, P, order)["total"] == total
    horder, htotal = md.mdfft_order_heuristic(N, P)
    assert htotal >= total
    assert htotal == pytest.approx(ratio * total, rel=1e-9)
    M, T = len(N), int(np.prod(N))
    assert order[0] == list(range(M)) and sorted(L[-1] for L in order) == list(range(M))
    if len(set(N)) == 1 and N[0] ** (M // 2) % P == 0:
        assert total * P == T * (P - 1)
    worst_order, worst = md.mdfft_order_search(N, P, 1)
    assert oracle.comm_volume(N, P, worst_order)["total"] == worst >= htotal
    # a 6-D plan without an order takes the exact search's order
    h = md.mdfft_plan(N, P, None, "c64", HOST)
    try:
        assert md.mdfft_plan_order(h, M) == order
    finally:
        md.mdfft_destroy(h)


def test_exact_six_dim_search_refuses_what_it_cannot_afford():
    with pytest.raises(md.MdfftError) as e:
        md.mdfft_order_search((8,) * 6, 4096, 0)
    assert e.value.status == -7  # E_UNSUPPORTED: the heuristic is the way there
    h = md.mdfft_plan((8,) * 6, 4096, None, "c64", HOST)  # plans fall back to the heuristic
    try:
        assert md.mdfft_plan_order(h, 6) == md.mdfft_order_heuristic((8,) * 6, 4096)[0]
    finally:
        md.mdfft_destroy(h)


# ----------------------------------------------------------------------------- comparison methods (Sec. 4)

def _fft_axes(order):
    return [L[-1] for L in oracle.parse_order(order)]


BLOCK_CASES = [((8, 8, 8), "slab", (2, 3, 8)), ((6, 5, 4), "slab", (2, 4, 5)),
               ((8, 8, 8), "pencil", (2, 4, 6, 12, 16, 64)), ((12, 10, 9), "pencil", (6, 9, 30, 90)),
               ((8, 8, 8), "volumetric", (2, 8, 12, 64, 100, 512)), ((6, 5, 4), "volumetric", (6, 30, 60)),
               ((4, 6, 5, 2), "slab", (2, 4)), ((4, 6, 5, 2), "pencil", (4, 12, 24)),
               ((4, 6, 5, 2), "volumetric", (8, 24, 240)), ((3, 4, 2, 2, 3), "volumetric", (6, 36)),
               ((3, 4, 2, 2, 3), "pencil", (6, 12))]


@pytest.mark.parametrize("N,kind,Ps", BLOCK_CASES, ids=lambda v: str(v))
def test_comparison_methods_match_the_oracle(N, kind, Ps):
    M = len(N)
    rng = np.random.default_rng(45)
    orders = oracle.enumerate_orders(M, cap=2000)
    picks = [orders[0]] + [orders[i] for i in rng.choice(len(orders), size=min(4, len(orders) - 1), replace=False)]
    checked = refused = 0
    for o in picks:
        order = oracle.format_order(o)
        for P in Ps:
            try:
                ref = oracle.block_volume(N, P, kind, _fft_axes(order))
            except ValueError:  # a cut with more blocks than points: both sides refuse
                with pytest.raises(md.MdfftError) as e:
                    md.mdfft_plan(N, P, order, "c64", HOST | md.DECOMPOSITIONS[kind])
                assert e.value.status == md.mdfft.MDFFT_E_RANGE
                refused += 1
                continue
            h = md.mdfft_plan(N, P, order, "c64", HOST | md.DECOMPOSITIONS[kind])
            checked += 1
            try:
                got = md.mdfft_comm_volume(h, M)
                for key in ("per_transition", "total", "split_line", "paper_total"):
                    assert got[key] == ref[key], (order, P, key)
                assert got["final_to_natural"] == 0
                assert [md.mdfft_block_grid(h, s, M) for s in range(M)] == ref["q"]
            finally:
                md.mdfft_destroy(h)
    assert checked >= len(Ps)


def test_comparison_method_errors():
    N = (8, 8, 8)
    with pytest.raises(md.MdfftError) as e:
        md.mdfft_plan(N, 16, None, "c64", HOST | md.MDFFT_PLAN_DECOMP_SLAB)  # 16 blocks of 8 points
    assert e.value.status == md.mdfft.MDFFT_E_RANGE
    with pytest.raises(md.MdfftError) as e:
        md.mdfft_plan(N, 4, None, "c64", HOST | md.MDFFT_PLAN_DECOMP_SLAB | md.MDFFT_PLAN_DECOMP_PENCIL)
    assert e.value.status == md.mdfft.MDFFT_E_ARG
    with pytest.raises(md.MdfftError):
        md.mdfft_plan((8, 8), 4, None, "c64", HOST | md.MDFFT_PLAN_DECOMP_PENCIL)  # needs M >= 3
    h = md.mdfft_plan(N, 4, None, "c64", HOST | md.MDFFT_PLAN_DECOMP_PENCIL)
    try:
        with pytest.raises(md.MdfftError):
            md.mdfft_chunk(h, 0, 0, 3)
        with pytest.raises(md.MdfftError):
            md.mdfft_exchange_counts(h, 0, 2)
        with pytest.raises(md.MdfftError):
            md.mdfft_block_grid(h, 3, 3)
    finally:
        md.mdfft_destroy(h)
    h = _plan(N, 4)
    try:
        with pytest.raises(md.MdfftError):
            md.mdfft_block_grid(h, 0, 3)  # row-wise plan
    finally:
        md.mdfft_destroy(h)


def test_comparison_methods_reach_the_closed_forms_at_64_cubed():
    # Fig. 7's setting: every method at the process counts where its closed form is exact
    N = (64, 64, 64)
    for kind, Ps, closed in (("slab", (2, 16, 64), lambda P: oracle.amount_slab(64, P)),
                             ("pencil", (4, 16, 64, 256, 1024, 4096), lambda P: oracle.amount_pencil(64, P)),
                             ("volumetric", (8, 64, 512, 4096, 32768, 262144),
                              lambda P: oracle.amount_volumetric(3, 64, P))):
        for P in Ps:
            h = md.mdfft_plan(N, P, None, "c64", HOST | md.DECOMPOSITIONS[kind])
            try:
                assert md.mdfft_comm_volume(h, 3)["paper_total"] == pytest.approx(closed(P), rel=1e-14), (kind, P)
            finally:
                md.mdfft_destroy(h)


def test_batched_plan_arguments():
    h = md.mdfft_plan_batched((8, 8, 8), 4, None, "c64", HOST, 6)
    try:
        assert md.mdfft_comm_volume(h, 3)["total"] == oracle.order_search((8, 8, 8), 4)["best"]  # per transform
    finally:
        md.mdfft_destroy(h)
    for bad in (0, -1, 1 << 32):
        with pytest.raises(md.MdfftError) as e:
            md.mdfft_plan_batched((256, 256, 256), 4, None, "c64", HOST, bad)
        assert e.value.status == md.mdfft.MDFFT_E_ARG


def test_output_in_the_last_layout_moves_nothing_at_the_end():
    for order in ("abc->acb->bca", "abc->cab->cba"):
        h = md.mdfft_plan((8, 6, 4), 6, order, "c64", HOST | md.MDFFT_PLAN_OUT_LAST_LAYOUT)
        try:
            cv = md.mdfft_comm_volume(h, 3)
        finally:
            md.mdfft_destroy(h)
        ref = oracle.comm_volume((8, 6, 4), 6, order)
        assert cv["final_to_natural"] == 0 and cv["per_transition"] == ref["per_transition"]


def test_wait_selftest_arguments():
    for bad in (0, -5, 10_000_001):
        st, _ = md.mdfft_selftest_wait(0, bad)
        assert st == md.mdfft.MDFFT_E_ARG


def test_tuning_needs_device_plans():
    h = _plan((8, 8, 8), 4)
    try:
        with pytest.raises(md.MdfftError):
            md.mdfft_plan_tuning(h, 3)
    finally:
        md.mdfft_destroy(h)
