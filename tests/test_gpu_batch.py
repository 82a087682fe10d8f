"""Batched plans (mdfft_plan_batched): one launch per pass over the tiles of
every transform of the batch.  Each transform must come out bit-identical to
the same plan run on it alone (same kernel, same tiles, same arithmetic per
line), match the oracle, and counted executions must add the per-transform
amounts."""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TOL = {"c64": 1e-5, "c128": 1e-12}
TDT = {"c64": torch.complex64, "c128": torch.complex128}
NDT = {"c64": np.complex64, "c128": np.complex128}


def _volumes(shape, B, dt, seed):
    return [si.uniform_complex(shape, seed + i, NDT[dt]) for i in range(B)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape,P,order,dt,B", [((32, 48, 20), 12, "abc->cab->bca", "c64", 3),
                                                ((32, 48, 20), 7, "abc->acb->cba", "c128", 2),
                                                ((8, 12, 10, 6), 16, None, "c64", 5),
                                                ((24, 16, 6, 10, 4), 64, None, "c64", 2)])
def test_batch_equals_each_alone(shape, P, order, dt, B):
    vols = _volumes(shape, B, dt, 500)
    x = torch.from_numpy(np.stack(vols)).to(DEV)
    with md.Plan(shape, P, order, dt, batch=B) as pb, md.Plan(shape, P, order, dt) as p1:
        y = pb.exec(x)
        z = pb.exec(y, dir=+1, normalize=True)
        for i in range(B):
            assert torch.equal(y[i], p1.exec(x[i].contiguous()))
        torch.cuda.synchronize()
    for i in range(B):
        ref = oracle.fftn(vols[i].astype(np.complex128))
        assert _rel(y[i].cpu().numpy(), ref) < TOL[dt]
        assert _rel(z[i].cpu().numpy(), vols[i]) < TOL[dt]


def test_counted_batch_adds_the_amounts():
    shape, P, B = (16, 12, 10), 24, 3
    x = torch.from_numpy(np.stack(_volumes(shape, B, "c64", 510))).to(DEV)
    for o in ("abc->acb->bca", "abc->cba->acb"):
        with md.Plan(shape, P, o, "c64", batch=B) as pb:
            _, counts = pb.exec_counted(x)
            got = counts.cpu().tolist()
        ref = oracle.comm_volume(shape, P, o)
        assert got[:2] == [B * v for v in ref["per_transition"]]
        assert got[2] == B * ref["final_to_natural"]
        assert got[3:] == [B * v for v in ref["split_line"]]


def test_batch_in_place_and_host_copies():
    shape, P, B = (20, 16, 12), 8, 3  # odd M: the in-place plan's second workspace
    vols = _volumes(shape, B, "c64", 520)
    x = torch.from_numpy(np.stack(vols)).to(DEV)
    with md.Plan(shape, P, None, "c64", md.MDFFT_PLAN_INPLACE, batch=B) as pb:
        want = pb.exec(x)
        buf = x.clone()
        pb.exec(buf, buf)
        assert torch.equal(buf, want)
        hx = x.cpu().pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        din, dout = torch.empty_like(x), torch.empty_like(x)
        pb.exec_host(hx, hy, din, dout)
        torch.cuda.synchronize()
        assert torch.equal(hy, want.cpu())
        assert pb.workspace_bytes() == 2 * B * int(np.prod(shape)) * 8


def test_batch_autotune_and_persistent_kernel_keep_results():
    shape, P, B = (64, 32, 48), 16, 4
    x = torch.from_numpy(np.stack(_volumes(shape, B, "c64", 530))).to(DEV)
    with md.Plan(shape, P, None, "c64", batch=B) as pb:
        want = pb.exec(x)
        scratch = torch.empty_like(x)
        pb.autotune(x, scratch, reps=2)
        assert torch.equal(pb.exec(x), want)
    with md.Plan(shape, P, None, "c64", md.MDFFT_PLAN_PERSISTENT, batch=B) as pp:
        y = pp.exec(x)
        pp.check()
        assert torch.equal(y, want)


@pytest.mark.parametrize("shape,P,B", [((32, 24, 40), 16, 4), ((8, 12, 10, 6), 12, 3)])
def test_pipelined_host_execution(shape, P, B):
    # copies and passes of neighbouring transforms on three streams: the same
    # results as the device call, forward and normalised inverse, repeatedly
    vols = _volumes(shape, B, "c64", 540)
    x = torch.from_numpy(np.stack(vols)).to(DEV)
    with md.Plan(shape, P, None, "c64", batch=B) as pb:
        want = pb.exec(x)
        back = pb.exec(want, dir=+1, normalize=True)
        hx = x.cpu().pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        hz = torch.empty_like(hx).pin_memory()
        din, dout = torch.empty_like(x), torch.empty_like(x)
        for _ in range(3):
            pb.exec_host(hx, hy, din, dout)
            pb.exec_host(hy, hz, din, dout, dir=+1, normalize=True)
        torch.cuda.synchronize()
        assert torch.equal(hy, want.cpu())
        assert torch.equal(hz, back.cpu())
    for i in range(B):
        assert _rel(hz[i].numpy(), vols[i]) < TOL["c64"]


def test_last_layout_output_through_host_pipeline_and_graph():
    # MDFFT_PLAN_OUT_LAST_LAYOUT with a batch: the pipelined host path and the
    # graph replay give the device call's bytes
    shape, P, B = (24, 32, 20), 12, 3
    x = torch.from_numpy(np.stack(_volumes(shape, B, "c64", 560))).to(DEV)
    with md.Plan(shape, P, None, "c64", md.MDFFT_PLAN_OUT_LAST_LAYOUT, batch=B) as pl:
        want = pl.exec(x)
        assert tuple(want.shape) == pl.out_shape
        hx = x.cpu().pin_memory()
        hy = torch.empty(pl.out_shape, dtype=torch.complex64).pin_memory()
        din = torch.empty_like(x)
        dout = torch.empty(pl.out_shape, dtype=torch.complex64, device=DEV)
        pl.exec_host(hx, hy, din, dout)
        g = torch.empty_like(want)
        pl.exec(x, g, graph=True)
        torch.cuda.synchronize()
        assert torch.equal(hy, want.cpu())
        assert torch.equal(g, want)
        last = pl.order()[-1]
    for i in range(B):
        ref = np.transpose(oracle.fftn(x[i].cpu().numpy().astype(np.complex128)), last)
        assert _rel(want[i].cpu().numpy(), ref) < TOL["c64"]


@pytest.mark.parametrize("shape,P,B", [((8, 6, 10, 4), 16, 3), ((6, 4, 5, 4, 3), 20, 2)])
def test_batched_higher_dims_graph_and_counts(shape, P, B):
    M = len(shape)
    x = torch.from_numpy(np.stack(_volumes(shape, B, "c128", 570))).to(DEV)
    with md.Plan(shape, P, None, "c128", batch=B) as pl:
        want = pl.exec(x)
        assert torch.equal(pl.exec(x, graph=True), want)
        _, counts = pl.exec_counted(x)
        c = counts.cpu().tolist()
        order = pl.order()
    ref = oracle.comm_volume(shape, P, order)
    assert c[: M - 1] == [B * v for v in ref["per_transition"]]
    for i in range(B):
        r = oracle.fftn(x[i].cpu().numpy())
        assert _rel(want[i].cpu().numpy(), r) < TOL["c128"]
