"""Pins of the oracle's FFT routes (Sec. 2 of the paper) against things other
than the oracle itself: the naive DFT, numpy.fft, closed-form spectra and
identities of the DFT.  CPU only."""

import itertools

import numpy as np
import pytest

import oracle
import synth_inputs as si

TINY = [(2, 3, 4), (3, 3, 3), (1, 5, 1), (4, 4, 4, 4), (2, 2, 2, 2, 2), (3, 4, 5, 2, 3), (7, 11), (13,)]
MEDIUM = [(24, 48, 20), (16, 16, 16, 16), (6, 10, 12, 5, 9), (32, 32, 32), (17, 19, 3)]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_dft_point_matches_numpy_and_naive():
    rng = np.random.default_rng(3)
    for shape in [(6, 5, 8), (4, 3, 5, 2), (24, 20, 16)]:
        x = si.uniform_complex(shape, 31)
        ref = np.fft.fftn(x)
        for _ in range(6):
            k = tuple(int(rng.integers(0, n)) for n in shape)
            assert abs(oracle.dft_point(x, k) - ref[k]) < 1e-12 * np.abs(ref).max()
            assert abs(oracle.dft_point(x, k, sign=+1) - x.size * np.fft.ifftn(x)[k]) < 1e-12 * np.abs(ref).max()


def test_naive_dft_matches_numpy():
    # numpy's pocketfft is a library routine independent of the oracle.
    for shape in TINY:
        x = si.uniform_complex(shape, 11)
        assert rel_l2(oracle.dft_naive(x), np.fft.fftn(x)) < 1e-13


@pytest.mark.parametrize("shape", TINY)
def test_fftn_matches_naive_dft(shape):
    x = si.uniform_complex(shape, 12)
    assert rel_l2(oracle.fftn(x), oracle.dft_naive(x)) < 1e-13
    assert rel_l2(oracle.fftn(x, sign=+1), oracle.dft_naive(x, sign=+1)) < 1e-13


@pytest.mark.parametrize("shape", MEDIUM)
def test_fftn_matches_numpy(shape):
    x = si.uniform_complex(shape, 13)
    assert rel_l2(oracle.fftn(x), np.fft.fftn(x)) < 1e-14
    # the unnormalised inverse is T times numpy's normalised ifftn
    T = x.size
    assert rel_l2(oracle.fftn(x, sign=+1), T * np.fft.ifftn(x)) < 1e-14


def test_fftn_threads_give_identical_bits():
    x = si.uniform_complex((16, 24, 20), 14)
    assert np.array_equal(oracle.fftn(x, nthreads=1), oracle.fftn(x, nthreads=5))


def test_1d_every_length_up_to_64():
    for n in range(1, 65):
        x = si.uniform_complex((n,), 100 + n)
        assert rel_l2(oracle.fft1d(x), np.fft.fft(x)) < 1e-14, n


def test_delta_input_closed_form():
    # X = delta(j - j0)  ->  Xbar(k) = prod_r exp(-2 pi i j0_r k_r / N_r)
    shape, j0 = (6, 5, 8), (4, 2, 7)
    x = np.zeros(shape, np.complex128)
    x[j0] = 1.0
    expect = np.ones(shape, np.complex128)
    for r, (n, j) in enumerate(zip(shape, j0)):
        k = np.arange(n)
        f = np.exp(-2j * np.pi * ((j * k) % n) / n)
        sl = [None] * len(shape)
        sl[r] = slice(None)
        expect = expect * f[tuple(sl)]
    assert np.max(np.abs(oracle.fftn(x) - expect)) < 1e-14


@pytest.mark.parametrize("shape", [(12, 10, 9), (8, 6, 4, 10), (4, 3, 5, 4, 6)])
def test_plane_wave_spectrum_is_exact_delta(shape):
    k0 = si.plane_wave_k0(shape, 1305)
    x = si.plane_wave(shape, k0)
    y = oracle.fftn(x)
    T = x.size
    expect = np.zeros(shape, np.complex128)
    expect[k0] = T
    assert np.max(np.abs(y - expect)) < 1e-11 * T


def test_parseval_roundtrip_linearity_shift():
    shape = (10, 12, 9)
    x = si.uniform_complex(shape, 15)
    z = si.uniform_complex(shape, 16)
    T = x.size
    X = oracle.fftn(x)
    # Parseval: sum |Xbar|^2 = T sum |X|^2
    assert abs(np.sum(np.abs(X) ** 2) - T * np.sum(np.abs(x) ** 2)) < 1e-12 * T * np.sum(np.abs(x) ** 2)
    # inverse (unnormalised, sign +1) of the forward gives T x
    assert rel_l2(oracle.fftn(X, sign=+1), T * x) < 1e-14
    # linearity
    a, b = 0.3 - 1.2j, -2.0 + 0.5j
    assert rel_l2(oracle.fftn(a * x + b * z), a * X + b * oracle.fftn(z)) < 1e-14
    # shift theorem along every axis
    for axis, s in zip(range(3), (3, 5, 7)):
        n = shape[axis]
        k = np.arange(n)
        ph = np.exp(-2j * np.pi * ((k * s) % n) / n)
        sl = [None] * 3
        sl[axis] = slice(None)
        assert rel_l2(oracle.fftn(np.roll(x, s, axis=axis)), X * ph[tuple(sl)]) < 1e-14


def test_axis_passes_commute():
    # Sec. 2: the M single steps are independent of the axis order.
    x = si.uniform_complex((6, 8, 10), 17)
    y = x
    for axis in (0, 2, 1):
        y = oracle.fft_axis(y, axis)
    assert rel_l2(y, oracle.fftn(x)) < 1e-14


ORDERS3 = [oracle.format_order(o) for o in oracle.enumerate_orders(3)]


@pytest.mark.parametrize("order", ORDERS3)
@pytest.mark.parametrize("P", [1, 3, 4, 7, 12, 40, 60, 120])
def test_fig4_route_equals_plain_route_3d(order, P):
    x = si.uniform_complex((4, 5, 6), 18)
    y, moved, split = oracle.fft_fig4(x, P, order)
    assert rel_l2(y, oracle.fftn(x)) < 1e-14
    cv = oracle.comm_volume((4, 5, 6), P, order)
    # two independent counts inside the oracle: explicit messages vs owner arrays
    assert list(moved[:2]) == cv["per_transition"]
    assert int(moved[2]) == cv["final_to_natural"]
    assert list(split) == cv["split_line"]


@pytest.mark.parametrize("seed", range(6))
def test_fig4_route_equals_plain_route_4d_5d(seed):
    rng = np.random.default_rng(900 + seed)
    for M in (4, 5):
        orders = oracle.enumerate_orders(M, cap=2000)
        o = orders[rng.integers(0, len(orders))]
        shape = tuple(int(v) for v in rng.integers(2, 5, size=M))
        T = int(np.prod(shape))
        P = int(rng.integers(1, T + 1))
        x = si.uniform_complex(shape, 19 + seed)
        y, moved, split = oracle.fft_fig4(x, P, o)
        assert rel_l2(y, oracle.fftn(x)) < 1e-14
        cv = oracle.comm_volume(shape, P, o)
        assert list(moved[: M - 1]) == cv["per_transition"]
        assert list(split) == cv["split_line"]


def test_fig4_rejects_bad_orders():
    x = si.uniform_complex((3, 3, 3), 20)
    with pytest.raises(ValueError):
        oracle.fft_fig4(x, 2, "acb->cab->cba")  # first layout must be natural
    with pytest.raises(ValueError):
        oracle.fft_fig4(x, 2, "abc->acb->bac")  # last axes must all differ (c, b, c)
    with pytest.raises(ValueError):
        oracle.fft_fig4(x, 28, "abc->cab->cba")  # Np > T


def test_every_order_gives_same_spectrum_4d_small():
    x = si.uniform_complex((2, 3, 2, 3), 21)
    ref = oracle.fftn(x)
    for o in itertools.islice(oracle.enumerate_orders(4), 0, 1296, 37):
        y, _, _ = oracle.fft_fig4(x, 5, o)
        assert rel_l2(y, ref) < 1e-14
