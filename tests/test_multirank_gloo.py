"""The multi-device exchange of the method on two ranks (gloo, world size 2).

The P virtual processes are laid onto G = 2 ranks in contiguous blocks.
 * On CPU ranks: every rank works out from the oracle's f_MD bounds which
   of its points go to which rank at every transpose; the counts must equal
   mdfft_exchange_counts exactly on both ranks, and the cross-device volume
   never exceeds the per-transition amount.
 * On one GPU (marked gpu): two gloo ranks each run their part of the
   transform through libmdfft (mdfft_dist_lines / pack / unpack via
   DistPlan); the only data movement outside the library is gloo's
   all-to-all-v of the packed buffers (through host memory).  The gathered
   spectrum must equal the oracle's.  The ranks' kernels never wait on each
   other: the exchange is on the host."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

CASES = [((8, 6, 4), 4, "abc->acb->bca"), ((8, 6, 4), 6, "abc->cab->cba"),
         ((4, 6, 5, 2), 4, "abcd->abdc->dcab->dcba"), ((16, 12, 10), 16, None)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _layout_strides(L, N):
    st = [0] * len(N)
    s = 1
    for a in reversed(L):
        st[a] = s
        s *= N[a]
    return st


def _region(N, P, L, g, G, fmd):
    Nl = [N[a] for a in L]
    return fmd(Nl, P, g * P // G), fmd(Nl, P, (g + 1) * P // G)


def _counts_worker(rank, world, port, shape, P, order, result_q):
    import oracle
    import paper_1302_6189_gb300 as md

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M = len(shape)
        N = list(shape)
        h = md.mdfft_plan(shape, P, order, "c64", md.MDFFT_PLAN_HOST_ONLY)
        layouts = md.mdfft_plan_order(h, M) + [list(range(M))]
        ok = True
        cross_ok = True
        cv = md.mdfft_comm_volume(h, M)
        for s in range(M):
            L, Ln = layouts[s], layouts[s + 1]
            r0, r1 = _region(N, P, L, rank, world, oracle.fmd)
            coords = np.array(np.unravel_index(np.arange(r0, r1), [N[a] for a in L]))  # in L's axis order
            st_n = _layout_strides(Ln, N)
            dest_idx = sum(coords[i] * st_n[L[i]] for i in range(M))
            send = [0] * world
            for g in range(world):
                a, b = _region(N, P, Ln, g, world, oracle.fmd)
                send[g] = int(np.sum((dest_idx >= a) & (dest_idx < b)))
            counts = md.mdfft_exchange_counts(h, s, world)
            ok &= send == counts[rank]
            got = [None] * world
            dist.all_gather_object(got, send)  # every rank sees the whole matrix
            ok &= got == counts
            if s < M - 1:
                cross_ok &= counts[0][1] + counts[1][0] <= cv["per_transition"][s]
        result_q.put((ok, cross_ok))
        md.mdfft_destroy(h)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("shape,P,order", CASES)
def test_two_rank_counts_match_the_oracle_ownership(shape, P, order):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_counts_worker, args=(r, 2, port, shape, P, order, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[0] for r in results)  # the ranks' realised counts == mdfft_exchange_counts
    assert all(r[1] for r in results)  # cross-device volume <= the per-transition amount


def _data_worker(rank, world, port, shape, P, order, dt, result_q):
    import oracle
    import paper_1302_6189_gb300 as md
    import synth_inputs as si

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        npdt = np.complex128 if dt == "c128" else np.complex64
        x = si.uniform_complex(shape, 77)
        with md.DistPlan(shape, P, world, rank, order, dt) as dp:
            a, b = dp.local_range(0)
            xl = torch.from_numpy(x.astype(npdt).ravel()[a:b].copy()).cuda()
            ex = md.torch_exchange(via_host=True)
            y = dp.run(xl, ex)
            back = dp.run(y, ex, dir=+1, normalize=True)
            torch.cuda.synchronize()
            a1, b1 = dp.local_range(len(shape))
            parts = [None] * world
            dist.all_gather_object(parts, (a1, y.cpu().numpy(), back.cpu().numpy()))
        if rank == 0:
            yy = np.empty(x.size, np.complex128)
            bb = np.empty(x.size, np.complex128)
            for a1, v, w in parts:
                yy[a1:a1 + v.size] = v
                bb[a1:a1 + w.size] = w
            ref = oracle.fftn(x).ravel()
            result_q.put((float(np.linalg.norm(yy - ref) / np.linalg.norm(ref)),
                          float(np.linalg.norm(bb - x.ravel()) / np.linalg.norm(x))))
        else:
            result_q.put(None)
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("shape,P,order", CASES)
def test_two_rank_transform_through_the_library(shape, P, order, dt):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_data_worker, args=(r, 2, port, shape, P, order, dt, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    errs = [r for r in results if r is not None]
    tol = 1e-12 if dt == "c128" else 1e-5
    assert len(errs) == 1 and errs[0][0] < tol and errs[0][1] < 2 * tol, errs


def _bench_worker(rank, world, port, q):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        q.put((rank, bench.max_over_ranks(10.0 + 5.0 * rank, world)))
    finally:
        dist.destroy_process_group()


def test_bench_takes_the_max_time_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 15.0, 1: 15.0}
