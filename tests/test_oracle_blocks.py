"""Pins of the oracle's comparison methods (Sec. 4): slab, pencil and
volumetric decompositions counted point by point.

What fixes them independently of the oracle: the closed forms A_1D, A_2D,
A_3D, A_4D, A_5D of Sec. 4 (exact whenever Np is a k-th power whose root
divides N), hand counts of tiny ragged cases (tests/golden), the process
limits Sec. 4 states (64 processes for the 1-D method and 64 x 64 for the
2-D method on 64^3 points), and the printed comparison figures at 64^3
(60.0 % and 77.8 % over the 2-D method, equality with the 1-D method up to
64 processes)."""

import json
import os

import pytest

import oracle

HERE = os.path.dirname(__file__)
C_B_A = [2, 1, 0]


def _golden():
    with open(os.path.join(HERE, "golden", "block_methods_hand.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: f"{c['kind']}-{'x'.join(map(str, c['N']))}-P{c['P']}")
def test_hand_counted_cases(case):
    r = oracle.block_volume(case["N"], case["P"], case["kind"], case["fft_axes"])
    assert r["per_transition"] == case["per_transition"]
    assert r["split_line"] == case["split_line"]


@pytest.mark.parametrize("N,P", [((8, 8, 8), 2), ((8, 8, 8), 4), ((8, 8, 8), 8), ((12, 8, 6), 4), ((6, 6, 5), 3)])
def test_slab_equals_A1D_when_P_divides_both_cut_axes(N, P):
    T = N[0] * N[1] * N[2]
    r = oracle.block_volume(N, P, "slab", C_B_A)
    assert r["paper_total"] == T - T // P
    if N[0] == N[1] == N[2]:
        assert r["paper_total"] == pytest.approx(oracle.amount_slab(N[0], P), rel=1e-15)


@pytest.mark.parametrize("n,P", [(8, 4), (8, 16), (8, 64), (12, 9), (12, 36), (16, 256)])
def test_pencil_equals_A2D_for_square_grids(n, P):
    r = oracle.block_volume((n, n, n), P, "pencil", C_B_A)
    q = int(round(P ** 0.5))
    assert r["q"][0] == [q, q, 1] and r["q"][1] == [q, 1, q] and r["q"][2] == [1, q, q]
    assert r["split_line"] == [0, 0, 0]
    assert r["paper_total"] == pytest.approx(oracle.amount_pencil(n, P), rel=1e-14)


@pytest.mark.parametrize("M,n,P", [(3, 8, 8), (3, 8, 64), (3, 8, 512), (3, 6, 27), (4, 4, 16), (4, 4, 256),
                                   (5, 4, 32), (5, 4, 1024), (4, 6, 81)])
def test_volumetric_equals_AMD_for_cubic_grids(M, n, P):
    r = oracle.block_volume((n,) * M, P, "volumetric", list(range(M - 1, -1, -1)))
    assert r["total"] == 0  # blocks never move
    assert r["paper_total"] == pytest.approx(oracle.amount_volumetric(M, n, P), rel=1e-14)


def test_process_limits_stated_for_64_cubed():
    # the 1-D method stops at 64 processes, the 2-D method at 64 x 64
    oracle.block_volume((64, 64, 64), 64, "slab", C_B_A)
    with pytest.raises(ValueError):
        oracle.block_volume((64, 64, 64), 128, "slab", C_B_A)
    oracle.block_volume((64, 64, 64), 4096, "pencil", C_B_A)
    with pytest.raises(ValueError):
        oracle.block_volume((64, 64, 64), 8192, "pencil", C_B_A)
    oracle.block_volume((8, 8, 8), 512, "volumetric", C_B_A)


def test_even_split_of_the_process_count():
    # prime factors, largest first, each to the cut with the smallest product
    assert oracle.block_volume((12, 12, 12), 12, "pencil", C_B_A)["q"][0] == [3, 4, 1]
    assert oracle.block_volume((64, 64, 64), 8192, "volumetric", C_B_A)["q"][0] == [32, 16, 16]
    assert oracle.block_volume((64, 64, 64), 8, "pencil", C_B_A)["q"][0] == [4, 2, 1]


def test_rowwise_equals_the_1D_method_up_to_64_processes_at_64_cubed():
    # our method cuts one axis for P <= 64 (P dividing 64) and then moves
    # exactly what the 1-D method moves
    for P in (2, 4, 8, 16, 32, 64):
        best = oracle.order_search((64, 64, 64), P)["best"]
        slab = oracle.block_volume((64, 64, 64), P, "slab", C_B_A)["paper_total"]
        assert best == slab


def test_printed_advantage_over_the_2D_method_at_64_cubed():
    # 60.0 % better at 16 processes and 77.8 % at 64, the end of the range
    for P, ratio in ((16, 1.600), (64, 1.778)):
        best = oracle.order_search((64, 64, 64), P)["best"]
        pencil = oracle.block_volume((64, 64, 64), P, "pencil", C_B_A)["paper_total"]
        assert round(pencil / best, 3) == ratio


def test_steps_in_another_axis_order():
    # the 2-D method with steps c, a, b: the cut of a moves to c, then b's to a
    r = oracle.block_volume((8, 8, 8), 16, "pencil", [2, 0, 1])
    assert r["q"] == [[4, 4, 1], [1, 4, 4], [4, 1, 4]]
    assert r["paper_total"] == pytest.approx(oracle.amount_pencil(8, 16), rel=1e-14)
