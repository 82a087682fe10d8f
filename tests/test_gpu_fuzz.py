"""Seeded random sweep of the CUDA path against the oracle: shapes of 2 to 5
dims drawn from the supported line lengths, random process counts, orders,
dtypes, batch sizes and output layouts.  Every case runs forward and
normalised inverse; every 4th case also runs counted and checks the amounts
against the oracle's owner arrays."""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TOL = {"c64": 1e-5, "c128": 1e-12}
NP = {"c64": np.complex64, "c128": np.complex128}
LENGTHS = [n for n in range(1, 97) if md.mdfft_supported_length(n, "c64") and md.mdfft_supported_length(n, "c128")]


def _case(i):
    rng = np.random.default_rng(9000 + i)
    M = int(rng.integers(2, 6))
    cap = {2: 96, 3: 64, 4: 24, 5: 12}[M]
    dims = tuple(int(rng.choice([n for n in LENGTHS if n <= cap])) for _ in range(M))
    T = int(np.prod(dims))
    P = int(rng.integers(1, T + 1)) if rng.random() < 0.3 else int(rng.integers(1, min(T, 64) + 1))
    orders = oracle.enumerate_orders(M, cap=5000)
    order = oracle.format_order(orders[int(rng.integers(len(orders)))])
    dt = "c128" if rng.random() < 0.35 else "c64"
    batch = int(rng.choice([1, 1, 2, 3]))
    flags = md.MDFFT_PLAN_OUT_LAST_LAYOUT if rng.random() < 0.25 else 0
    return dims, P, order, dt, batch, flags


@pytest.mark.parametrize("i", range(40))
def test_random_case(i):
    dims, P, order, dt, batch, flags = _case(i)
    M = len(dims)
    xs = [si.uniform_complex(dims, 700 + 17 * i + b) for b in range(batch)]
    x = torch.from_numpy(np.stack([v.astype(NP[dt]) for v in xs])).to(DEV)
    if batch == 1:
        x = x[0]
    last = oracle.parse_order(order)[-1] if flags else list(range(M))
    with md.Plan(dims, P, order, dt, flags, batch=batch) as pl:
        y = pl.exec(x)
        z = pl.exec(x, dir=+1, normalize=True)
        if i % 4 == 0:
            _, counts = pl.exec_counted(x)
            c = counts.cpu().tolist()
        torch.cuda.synchronize()
    ys = [y.cpu().numpy()] if batch == 1 else list(y.cpu().numpy())
    zs = [z.cpu().numpy()] if batch == 1 else list(z.cpu().numpy())
    for b in range(batch):
        ref = np.transpose(oracle.fftn(xs[b]), last)
        refi = np.transpose(oracle.fftn(xs[b], sign=+1), last) / xs[b].size
        err = np.linalg.norm(ys[b] - ref) / max(np.linalg.norm(ref), 1e-300)
        erri = np.linalg.norm(zs[b] - refi) / max(np.linalg.norm(refi), 1e-300)
        assert err < TOL[dt] and erri < TOL[dt], (dims, P, order, dt, batch, flags, err, erri)
    if i % 4 == 0:
        cv = oracle.comm_volume(dims, P, order)
        assert c[: M - 1] == [batch * v for v in cv["per_transition"]]
        assert c[M - 1] == (0 if flags else batch * cv["final_to_natural"])
        assert c[M:] == [batch * v for v in cv["split_line"]]
