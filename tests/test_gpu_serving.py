"""The continuous-batching server: every result is the same alone (mdfft_exec
of the same shape) and in a mix of shapes, requests join while others are in
flight, and the HBM budget bounds what is admitted."""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def mixed_shapes(n, seed):
    rng = np.random.default_rng(seed)
    axes3 = [16, 24, 32, 48, 64]
    out = []
    for _ in range(n):
        u = rng.uniform()
        if u < 0.15:
            out.append((16, 16, 16, 16))
        elif u < 0.25:
            out.append(tuple(int(v) for v in rng.choice([20, 40, 30, 16], size=3)))  # separate launches
        else:
            out.append(tuple(int(v) for v in rng.choice(axes3, size=3)))
    return out


def alone(shape, x, dir, normalize):
    T = int(np.prod(shape))
    with md.Plan(shape, min(64, T), None, "c64") as plan:
        y = plan.exec(x, dir=dir, normalize=normalize)
        torch.cuda.synchronize()
    return y


def test_mix_equals_alone_and_oracle():
    shapes = mixed_shapes(48, 5)
    rng = np.random.default_rng(6)
    xs = [torch.from_numpy(si.uniform_complex(s, 500 + i, np.complex64)).to(DEV) for i, s in enumerate(shapes)]
    outs = [torch.empty_like(x) for x in xs]
    dirs = [int(rng.choice([-1, 1])) for _ in shapes]
    with md.Server(budget_bytes=1 << 30, max_inflight=16, P=64) as srv:
        srv.set_direct(0)  # every pass through the persistent grouped kernel
        ids = []
        i = 0
        while i < len(shapes):  # arrivals interleaved with steps: requests join mid-flight
            for _ in range(int(rng.integers(1, 4))):
                if i < len(shapes):
                    ids.append(srv.submit(xs[i], outs[i], dir=dirs[i], normalize=dirs[i] == 1))
                    i += 1
            srv.step()
        srv.drain()
        st = srv.stats()
        assert st["completed"] == len(shapes) and st["inflight"] == 0 and st["bytes_in_use"] == 0
        assert st["graph_launches"] >= 1
        for rid in ids:
            done, ms = srv.poll(rid)
            assert done and ms >= 0
            srv.release(rid)
    torch.cuda.synchronize()
    for s, x, y, d in zip(shapes, xs, outs, dirs):
        assert torch.equal(y, alone(s, x, d, d == 1)), s  # same kernels and tiles: identical bits
    for k in range(0, len(shapes), 7):  # and against the oracle
        ref = oracle.fftn(xs[k].cpu().numpy().astype(np.complex128), sign=dirs[k])
        if dirs[k] == 1:
            ref = ref / ref.size
        y = outs[k].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-5


def test_budget_limits_admission():
    shape = (64, 64, 64)
    bytes_req = 3 * 64 ** 3 * 8
    xs = [torch.from_numpy(si.uniform_complex(shape, 600 + i, np.complex64)).to(DEV) for i in range(6)]
    outs = [torch.empty_like(x) for x in xs]
    with md.Server(budget_bytes=2 * bytes_req + 4096, max_inflight=8) as srv:
        for x, y in zip(xs, outs):
            srv.submit(x, y)
        peak = 0
        for _ in range(200000):
            srv.step()
            st = srv.stats()
            assert st["bytes_in_use"] <= st["budget_bytes"]
            peak = max(peak, st["inflight"])
            if st["completed"] == len(xs):
                break
        srv.drain()
        assert peak <= 2
    for x, y in zip(xs, outs):
        assert torch.equal(y, alone(shape, x, -1, False))


def test_single_cta_grid_and_errors():
    shape = (32, 48, 16)
    x = torch.from_numpy(si.uniform_complex(shape, 700, np.complex64)).to(DEV)
    y = torch.empty_like(x)
    with md.Server(budget_bytes=1 << 26, max_inflight=4) as srv:
        srv.set_direct(0)
        srv.set_grid(1)  # one CTA walks every tile
        srv.submit(x, y)
        srv.drain()
        assert srv.stats()["grid_ctas"] == 1
        with pytest.raises(md.MdfftError) as e:
            big = torch.empty((256, 256, 256), dtype=torch.complex64, device=DEV)
            srv.submit(big, big)  # overlapping in/out
        assert e.value.status == -1
        with pytest.raises(md.MdfftError) as e:
            a = torch.empty((256, 256, 256), dtype=torch.complex64, device=DEV)
            b = torch.empty_like(a)
            srv.submit(a, b)  # 3 x 128 MiB > 64 MiB budget
        assert e.value.status == -3
        with pytest.raises(md.MdfftError):
            srv.poll(12345)
    assert torch.equal(y, alone(shape, x, -1, False))


def test_cancel_queued_and_in_flight_requests():
    # budget for two 64^3 requests: the third waits in the queue and is
    # cancelled there; the first is cancelled after its first pass was
    # launched; the others finish exactly as alone, and the budget comes back
    shape = (64, 64, 64)
    bytes_req = 3 * 64 ** 3 * 8
    xs = [torch.from_numpy(si.uniform_complex(shape, 650 + i, np.complex64)).to(DEV) for i in range(4)]
    outs = [torch.empty_like(x) for x in xs]
    with md.Server(budget_bytes=2 * bytes_req + 4096, max_inflight=8) as srv:
        srv.set_depth(1)
        ids = [srv.submit(x, y) for x, y in zip(xs, outs)]
        srv.step()  # admits requests 0 and 1, launches their first pass
        st = srv.stats()
        assert st["inflight"] == 2 and st["queued"] == 2
        srv.cancel(ids[2])  # still queued
        srv.cancel(ids[0])  # in flight: no further passes
        with pytest.raises(md.MdfftError):
            srv.cancel(ids[2])  # already cancelled
        srv.drain()
        st = srv.stats()
        assert st["cancelled"] == 2 and st["completed"] == 2
        assert st["bytes_in_use"] == 0 and st["inflight"] == 0 and st["queued"] == 0
        for i in (0, 2):
            done, ms = srv.poll(ids[i])
            assert done and ms == -1.0
            srv.release(ids[i])
        for i in (1, 3):
            done, ms = srv.poll(ids[i])
            assert done and ms >= 0
            with pytest.raises(md.MdfftError):
                srv.cancel(ids[i])  # finished
    for i in (1, 3):
        assert torch.equal(outs[i], alone(shape, xs[i], -1, False))


@pytest.mark.parametrize("chunk", [1, 16, 64])
def test_tile_dealing_does_not_change_results(chunk):
    shapes = mixed_shapes(12, 640 + chunk)
    xs = [torch.from_numpy(si.uniform_complex(sh, 660 + i, np.complex64)).to(DEV) for i, sh in enumerate(shapes)]
    outs = [torch.empty_like(x) for x in xs]
    with md.Server(budget_bytes=1 << 30, max_inflight=16) as srv:
        srv.set_chunk(chunk)
        for x, y in zip(xs, outs):
            srv.submit(x, y)
        srv.drain()
        with pytest.raises(md.MdfftError):
            srv.set_chunk(0)
    for sh, x, y in zip(shapes, xs, outs):
        assert torch.equal(y, alone(sh, x, -1, False))


def test_serving_bench_lengths_mix_equals_alone_and_oracle():
    # the lengths of the serving benchmark (3-D axes from {48, 64, 96, 128,
    # 160, 192}, 4-D 32^4): every length in every axis position, plus a draw
    # of the benchmark's own request generator, submitted while earlier
    # requests are in flight
    L = si.SERVING_AXES
    shapes = [(L[i], L[(i + 1) % 6], L[(i + 3) % 6]) for i in range(6)] + [(32, 32, 32, 32)]
    shapes += si.serving_requests(24, si.SEEDS["serving"])
    rng = np.random.default_rng(17)
    xs = [torch.from_numpy(si.uniform_complex(s, 1700 + i, np.complex64)).to(DEV) for i, s in enumerate(shapes)]
    outs = [torch.empty_like(x) for x in xs]
    dirs = [int(rng.choice([-1, 1])) for _ in shapes]
    with md.Server(budget_bytes=8 << 30, max_inflight=16, P=64) as srv:
        ids, i = [], 0
        while i < len(shapes):
            for _ in range(int(rng.integers(1, 5))):
                if i < len(shapes):
                    ids.append(srv.submit(xs[i], outs[i], dir=dirs[i], normalize=dirs[i] == 1))
                    i += 1
            srv.step()
        srv.drain()
        assert srv.stats()["completed"] == len(shapes)
        for rid in ids:
            assert srv.poll(rid)[0]
            srv.release(rid)
    torch.cuda.synchronize()
    for s, x, y, d in zip(shapes, xs, outs, dirs):
        assert torch.equal(y, alone(s, x, d, d == 1)), s
    for k in list(range(7)) + list(range(7, len(shapes), 6)):  # every length, and a sample of the draw
        ref = oracle.fftn(xs[k].cpu().numpy().astype(np.complex128), sign=dirs[k], nthreads=8)
        if dirs[k] == 1:
            ref = ref / ref.size
        y = outs[k].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-5, shapes[k]


@pytest.mark.parametrize("direct", [0, 2, 64])
def test_low_load_direct_launches_give_the_same_bits(direct):
    # requests submitted one at a time with the server stepped in between: at
    # low load (nothing queued, at most `direct` requests with passes left)
    # their passes run as plain launches; every result equals mdfft_exec's
    shapes = [(48, 64, 96), (32, 32, 32, 32), (192, 48, 64), (64, 64, 64), (20, 30, 40)]
    xs = [torch.from_numpy(si.uniform_complex(sh, 1800 + i, np.complex64)).to(DEV) for i, sh in enumerate(shapes)]
    outs = [torch.empty_like(x) for x in xs]
    with md.Server(budget_bytes=1 << 30, max_inflight=8) as srv:
        srv.set_direct(direct)
        ids = []
        for x, y in zip(xs, outs):
            ids.append(srv.submit(x, y))
            srv.step()
        srv.drain()
        st = srv.stats()
        assert st["completed"] == len(shapes)
        if direct == 0:
            assert st["direct_requests"] == 0
        else:
            assert st["direct_requests"] >= 1
        with pytest.raises(md.MdfftError):
            srv.set_direct(-1)
    for sh, x, y in zip(shapes, xs, outs):
        assert torch.equal(y, alone(sh, x, -1, False)), sh


@pytest.mark.parametrize("line_kernel", [0, 1])
def test_line_kernel_switch_and_8_byte_aligned_buffers(line_kernel):
    # passes of 16 to 64 points go to the step's one-thread-per-line kernel
    # when it is on and the request's arrays are 16-byte aligned, else to the
    # grouped kernel: every result equals mdfft_exec's either way (requests 1
    # and 3 use arrays that start 8 bytes past a 16-byte boundary)
    shapes = [(32, 32, 32, 32), (48, 64, 24), (16, 64, 48), (24, 24, 24), (64, 96, 32)]
    xs, outs = [], []
    for i, sh in enumerate(shapes):
        T = int(np.prod(sh))
        data = torch.from_numpy(si.uniform_complex(sh, 1900 + i, np.complex64)).to(DEV)
        if i in (1, 3):
            xb = torch.empty(T + 1, dtype=torch.complex64, device=DEV)
            ob = torch.empty(T + 1, dtype=torch.complex64, device=DEV)
            x, y = xb[1:].view(sh), ob[1:].view(sh)
            x.copy_(data)
            assert x.data_ptr() % 16 == 8 and y.data_ptr() % 16 == 8
        else:
            x, y = data, torch.empty_like(data)
        xs.append(x)
        outs.append(y)
    with md.Server(budget_bytes=1 << 30, max_inflight=8) as srv:
        srv.set_direct(0)
        srv.set_line_kernel(line_kernel)
        for x, y in zip(xs, outs):
            srv.submit(x, y)
        srv.drain()
        assert srv.stats()["completed"] == len(shapes)
        with pytest.raises(md.MdfftError):
            srv.set_line_kernel(2)
    for sh, x, y in zip(shapes, xs, outs):
        assert torch.equal(y, alone(sh, x.contiguous(), -1, False)), sh
