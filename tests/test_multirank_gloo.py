"""The multi-device exchange of the method on CPU ranks (gloo, world size 2).

The P virtual processes are laid onto G = 2 ranks in contiguous blocks.  Every
rank holds one contiguous row-major range of the current layout, transforms
its lines locally (numpy, standing in for the pass kernel), and sends every
point to the rank that holds it in the next layout with one all-to-all-v
whose counts come from mdfft_exchange_counts.  The realised send counts must
equal the library's counts exactly, and the gathered spectrum must equal the
oracle's.  No GPU is involved."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

CASES = [((8, 6, 4), 4, "abc->acb->bca"), ((8, 6, 4), 6, "abc->cab->cba"),
         ((4, 6, 5, 2), 4, "abcd->abdc->dcab->dcba")]


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


def _worker(rank, world, port, shape, P, order, result_q):
    import oracle
    import paper_1302_6189_gb300 as md
    import synth_inputs as si

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M = len(shape)
        N = list(shape)
        x = si.uniform_complex(shape, 77)
        h = md.mdfft_plan(shape, P, order, "c64", md.MDFFT_PLAN_HOST_ONLY)
        layouts = md.mdfft_plan_order(h, M) + [list(range(M))]
        ok_counts = True
        r0, r1 = _region(N, P, layouts[0], rank, world, oracle.fmd)
        local = x.ravel()[r0:r1].copy()  # natural layout = layout 0
        for s in range(M):
            L, Ln = layouts[s], layouts[s + 1]
            nf = N[L[-1]]
            local = np.fft.fft(local.reshape(-1, nf), axis=1).ravel()  # lines along L's last axis
            # where every local point goes in the next layout
            Nl = [N[a] for a in L]
            idx = np.arange(r0, r1)
            coords_l = np.array(np.unravel_index(idx, Nl))  # in L's axis order
            st_n = _layout_strides(Ln, N)
            dest_idx = sum(coords_l[i] * st_n[L[i]] for i in range(M))
            bounds = [_region(N, P, Ln, g, world, oracle.fmd) for g in range(world)]
            dest = np.zeros_like(dest_idx)
            for g, (a, b) in enumerate(bounds):
                dest[(dest_idx >= a) & (dest_idx < b)] = g
            counts = md.mdfft_exchange_counts(h, s, world)
            send_counts = [int(np.sum(dest == g)) for g in range(world)]
            ok_counts &= send_counts == counts[rank]
            order_send = np.lexsort((dest_idx, dest))  # by destination rank, then destination index
            send = torch.from_numpy(np.ascontiguousarray(local[order_send]).view(np.float64).copy())
            recv_counts = [counts[g][rank] for g in range(world)]
            recv = torch.empty(2 * sum(recv_counts), dtype=torch.float64)
            dist.all_to_all_single(recv, send, [2 * c for c in recv_counts], [2 * c for c in send_counts])
            # my new region; the source rank of each of its points, in the order they were sent
            n0, n1 = bounds[rank]
            nidx = np.arange(n0, n1)
            Nn = [N[a] for a in Ln]
            coords_n = np.array(np.unravel_index(nidx, Nn))
            st_l = _layout_strides(L, N)
            src_idx = sum(coords_n[i] * st_l[Ln[i]] for i in range(M))
            src = np.zeros_like(src_idx)
            for g in range(world):
                a, b = _region(N, P, L, g, world, oracle.fmd)
                src[(src_idx >= a) & (src_idx < b)] = g
            order_recv = np.lexsort((nidx, src))
            new_local = np.empty(n1 - n0, np.complex128)
            new_local[order_recv] = recv.numpy().view(np.complex128)
            local, r0, r1 = new_local, n0, n1
        parts = [None] * world
        dist.all_gather_object(parts, (r0, local))
        if rank == 0:
            y = np.empty(x.size, np.complex128)
            for a, v in parts:
                y[a:a + v.size] = v
            ref = oracle.fftn(x)
            err = float(np.linalg.norm(y - ref.ravel()) / np.linalg.norm(ref))
            cv = md.mdfft_comm_volume(h, M)
            cross = []
            for s in range(M - 1):
                c = md.mdfft_exchange_counts(h, s, world)
                cross.append(c[0][1] + c[1][0] <= cv["per_transition"][s])
            result_q.put((err, ok_counts, all(cross)))
        else:
            result_q.put((None, ok_counts, True))
        md.mdfft_destroy(h)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("shape,P,order", CASES)
def test_two_rank_exchange_matches_oracle(shape, P, order):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, shape, P, order, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    errs = [r[0] for r in results if r[0] is not None]
    assert len(errs) == 1 and errs[0] < 1e-13
    assert all(r[1] for r in results)  # realised send counts == mdfft_exchange_counts
    assert all(r[2] for r in results)  # cross-device volume <= the per-transition amount


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
