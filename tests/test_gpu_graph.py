"""mdfft_exec_graph: the plan's passes replayed from a captured CUDA graph
give exactly mdfft_exec's results, for every cached (in, out, dir,
normalize), after replacement of the least recently used graph and after
autotuning (which drops the captured graphs)."""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("shape,P,order,dt,batch", [((32, 32, 32), 4, "abc->cab->cba", "c128", 1),
                                                   ((32, 32, 32), 4, "abc->cab->cba", "c64", 1),
                                                   ((8, 12, 10, 6), 16, None, "c64", 3)])
def test_graph_replay_equals_direct_launches(shape, P, order, dt, batch):
    npdt = np.complex128 if dt == "c128" else np.complex64
    x = torch.from_numpy(np.stack([si.uniform_complex(shape, 800 + b, npdt) for b in range(batch)])).to(DEV)
    if batch == 1:
        x = x[0]
    with md.Plan(shape, P, order, dt, batch=batch) as pl:
        want_f = pl.exec(x)
        want_i = pl.exec(x, dir=+1, normalize=True)
        out = torch.empty_like(x)
        for _ in range(3):  # first call captures, the next ones replay
            assert torch.equal(pl.exec(x, out, graph=True), want_f)
            assert torch.equal(pl.exec(x, out, dir=+1, normalize=True, graph=True), want_i)
    if batch == 1:
        ref = oracle.fftn(si.uniform_complex(shape, 800))
        err = np.linalg.norm(want_f.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < (1e-12 if dt == "c128" else 1e-5)


def test_graph_cache_replacement_and_autotune():
    shape, P = (16, 24, 20), 8
    xs = [torch.from_numpy(si.uniform_complex(shape, 810 + i, np.complex64)).to(DEV) for i in range(11)]
    with md.Plan(shape, P, None, "c64") as pl:
        want = [pl.exec(x) for x in xs]
        outs = [torch.empty_like(x) for x in xs]
        for rep in range(2):  # 11 (in, out) pairs through a cache of 8
            for x, o, w in zip(xs, outs, want):
                pl.exec(x, o, graph=True)
                assert torch.equal(o, w)
        pl.autotune(xs[0], torch.empty_like(xs[0]), reps=2)
        for x, o, w in zip(xs, outs, want):
            assert torch.equal(pl.exec(x, o, graph=True), w)


def test_graph_argument_errors():
    x = torch.zeros((8, 8, 8), dtype=torch.complex64, device=DEV)
    with md.Plan((8, 8, 8), 4) as pl:
        with pytest.raises(md.MdfftError):
            md.mdfft_exec_graph(pl.handle, x.data_ptr(), x.data_ptr(), -1, 0, 0)  # in == out without INPLACE
        with pytest.raises(md.MdfftError):
            md.mdfft_exec_graph(pl.handle, x.data_ptr(), torch.empty_like(x).data_ptr(), 2, 0, 0)
