"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no FFT or decomposition arithmetic: it only draws the input
arrays (numpy ``default_rng`` = PCG64) so that the CPU oracle and the GPU
library see identical data.  complex64 inputs are the complex128 draws rounded
once, so the two precisions of one seed match.

Workload recipes (shapes and value distributions of the paper's setting: the
paper has no dataset, so these stand in for it):

* uniform: re, im i.i.d. U[-1, 1)                       (32^3, 256^3, 64^4, 24^5)
* gaussian: re, im i.i.d. N(0, 1)                        (512^3 precision study)
* plane wave: exp(+2 pi i sum_r k0_r j_r / N_r), k0 drawn from a seed; its
  forward transform is T at k = k0 and 0 elsewhere    (64^4, 24^5)
* serving mix: Poisson arrivals; 80 % 3-D requests with each axis drawn from
  {48, 64, 96, 128, 160, 192}, 20 % 4-D 32^4
"""

from __future__ import annotations

import numpy as np

SEEDS = {"parity32": 1302, "cube256": 1303, "md_uniform": 1304, "md_plane": 1305,
         "precision512": 1306, "serving": 1307}

SERVING_AXES = (48, 64, 96, 128, 160, 192)


def uniform_complex(shape, seed, dtype=np.complex128):
    """re, im ~ U[-1, 1) from default_rng(seed); complex64 = the rounded draw."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    x = np.empty(shape, np.complex128)
    x.real = rng.uniform(-1.0, 1.0, shape)
    x.imag = rng.uniform(-1.0, 1.0, shape)
    return x.astype(dtype, copy=False)


def gaussian_complex(shape, seed, dtype=np.complex128):
    """re, im ~ N(0, 1) from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    x = np.empty(shape, np.complex128)
    x.real = rng.standard_normal(shape)
    x.imag = rng.standard_normal(shape)
    return x.astype(dtype, copy=False)


def plane_wave_k0(shape, seed):
    rng = np.random.default_rng(seed)
    return tuple(int(rng.integers(0, int(n))) for n in shape)


def plane_wave(shape, k0, dtype=np.complex128):
    """exp(+2 pi i sum_r k0_r j_r / N_r) on the natural grid."""
    shape = tuple(int(s) for s in shape)
    phase = np.zeros(shape, np.float64)
    for r, (n, k) in enumerate(zip(shape, k0)):
        j = np.arange(n, dtype=np.int64)
        frac = ((j * int(k)) % n) / n
        sl = [None] * len(shape)
        sl[r] = slice(None)
        phase = phase + frac[tuple(sl)]
    phase -= np.floor(phase)
    return np.exp(2j * np.pi * phase).astype(dtype, copy=False)


def serving_requests(n, seed, frac_4d=0.2):
    """n request shapes of the serving mix, in arrival order."""
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(int(n)):
        if rng.uniform() < frac_4d:
            shapes.append((32, 32, 32, 32))
        else:
            shapes.append(tuple(int(v) for v in rng.choice(SERVING_AXES, size=3)))
    return shapes


def poisson_arrivals(n, rate_per_s, seed):
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed + 1)
    return np.cumsum(rng.exponential(1.0 / float(rate_per_s), size=int(n)))
