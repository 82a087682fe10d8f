"""Pins of the oracle's row-wise index maps (Sec. 3.1-3.2): hand-worked
fixtures, the paper's own 2-D-regime statement, regime boundaries, tiling
invariants and numpy's unravel_index.  CPU only."""

import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _load("index_maps_hand.json")["cases"],
                         ids=lambda c: f"{c['dims']}-P{c['P']}")
def test_hand_worked_chunks(case):
    N, P = case["dims"], case["P"]
    assert oracle.regime(N, P) == case["regime"]
    assert [oracle.fmd(N, P, p) for p in range(P + 1)] == case["starts"]
    for p, (xs, xe, cs, ce) in case["ranks"].items():
        assert oracle.chunk(N, P, int(p)) == (xs, xe, cs, ce)


def test_hand_worked_volumes():
    for case in _load("index_maps_hand.json")["volumes"]["cases"]:
        cv = oracle.comm_volume(case["dims"], case["P"], case["order"])
        assert cv["per_transition"] == case["per_transition"]
        assert cv["final_to_natural"] == case["final_to_natural"]


@pytest.mark.parametrize("N", [(8, 6, 5), (4, 4, 4), (16, 3, 7)])
def test_paper_2d_regime_statement(N):
    # Sec. 3.1: for N1 < Np <= N1 N2, x^s = floor(N1 N2 myid / Np) N3,
    # x^e = floor(N1 N2 (myid+1) / Np) N3 - 1, the chunk runs from
    # (a^s, b^s, 0) to (a^e, b^e, N3 - 1).
    N1, N2, N3 = N
    for P in range(N1 + 1, N1 * N2 + 1):
        assert oracle.regime(N, P) == 2
        for p in range(P):
            xs, xe, cs, ce = oracle.chunk(N, P, p)
            assert xs == (N1 * N2 * p // P) * N3
            assert xe == (N1 * N2 * (p + 1) // P) * N3 - 1
            assert cs[2] == 0 and ce[2] == N3 - 1


@pytest.mark.parametrize("N", [(4, 6, 5), (3, 2, 4, 5), (2, 3, 2, 2, 3)])
def test_regime_boundaries(N):
    pref = np.cumprod(N)
    for k, lead in enumerate(pref, start=1):
        assert oracle.regime(N, int(lead)) == k          # Np = N1..Nk stays in regime k
        if k < len(N):
            assert oracle.regime(N, int(lead) + 1) == k + 1
    assert oracle.regime(N, 1) == 1
    assert oracle.regime(N, int(pref[-1]) + 1) == -1     # Np > T has no decomposition
    assert oracle.regime(N, 0) == -1


@pytest.mark.parametrize("N", [(4, 6, 5), (7, 3, 2), (3, 2, 4, 5), (2, 3, 2, 2, 3), (5, 1, 3)])
def test_chunks_tile_the_grid(N):
    T = int(np.prod(N))
    for P in range(1, T + 1):
        k = oracle.regime(N, P)
        unit = int(np.prod(N[k:]))   # chunks are whole multiples of the trailing dims
        starts = [oracle.fmd(N, P, p) for p in range(P + 1)]
        assert starts[0] == 0 and starts[-1] == T
        sizes = np.diff(starts)
        assert np.all(sizes >= 1)                      # never empty (Np <= T)
        assert np.all(np.array(starts) % unit == 0)
        assert sizes.max() - sizes.min() <= unit       # near-equal division
        for p in (0, P // 2, P - 1):
            xs, xe, cs, ce = oracle.chunk(N, P, p)
            assert (xs, xe) == (starts[p], starts[p + 1] - 1)
            assert cs == [int(v) for v in np.unravel_index(xs, N)]
            assert ce == [int(v) for v in np.unravel_index(xe, N)]


def test_coords_and_linear_match_numpy():
    rng = np.random.default_rng(5)
    for N in [(3, 4, 5), (7, 2, 9, 4), (2, 3, 5, 7, 11)]:
        T = int(np.prod(N))
        for x in rng.integers(0, T, size=50):
            c = oracle.coords(N, int(x))
            assert c == [int(v) for v in np.unravel_index(int(x), N)]
            assert oracle.linear(N, c) == int(x)


def test_owner_arrays_follow_the_layout_row_major_order():
    N = (4, 6, 5)
    T = 120
    for layout in ["abc", "acb", "bac", "bca", "cab", "cba"]:
        L = oracle.parse_layout(layout)
        for P in (1, 3, 4, 7, 24, 25, 60, 120):
            own = oracle.owner_array(N, P, layout)
            seq = np.transpose(own, L).ravel()          # owners in the layout's row-major order
            assert np.all(np.diff(seq) >= 0)
            Nl = [N[a] for a in L]
            counts = np.bincount(seq, minlength=P)
            expect = np.diff([oracle.fmd(Nl, P, p) for p in range(P + 1)])
            assert np.array_equal(counts, expect)
            assert counts.sum() == T


def test_large_products_do_not_overflow():
    # 256^3 at Np = 2^17: N1 N2 N3 * myid reaches about 2^41.
    N = (256, 256, 256)
    P = 131072
    assert oracle.regime(N, P) == 3
    assert oracle.fmd(N, P, P) == 256 ** 3
    assert oracle.fmd(N, P, P - 1) == (256 ** 3 * (P - 1)) // P
    # 2^20-point 1-D dims with a product above 2^63 / 2^20
    big = (1 << 21, 1 << 21, 4)
    assert oracle.fmd(big, 3, 2) == ((1 << 21) * 2 // 3) * (1 << 21) * 4
