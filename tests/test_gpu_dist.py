"""The distributed data plane on G virtual devices of one GPU: every step's
line DFTs, pack and unpack run in libmdfft (mdfft_dist_*); the transport
between the devices is the test's (slices of each send buffer concatenated
into the receivers' buffers, as an all-to-all-v delivers them).  The
gathered spectrum must equal the oracle's, and every group's size the
library's exchange counts."""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = {"c64": 1e-5, "c128": 1e-12}
NP = {"c64": np.complex64, "c128": np.complex128}


def run_virtual(shape, P, order, dt, G, x, dir=-1, normalize=False):
    M = len(shape)
    parts = [md.DistPlan(shape, P, G, g, order, dt) for g in range(G)]
    try:
        h = parts[0].plan.handle
        st = torch.cuda.current_stream().cuda_stream
        flat = torch.from_numpy(np.ascontiguousarray(x.astype(NP[dt])).ravel()).to(DEV)
        local = []
        for g in range(G):
            a, b = parts[g].local_range(0)
            local.append(flat[a:b].clone())
        for s in range(M):
            counts = parts[0].counts(s)
            sends = []
            for g in range(G):
                work = torch.empty_like(local[g])
                md.mdfft_dist_lines(parts[g].plan.handle, s, G, g, local[g].data_ptr(), work.data_ptr(), dir,
                                    int(normalize), st)
                send = torch.empty(sum(counts[g]), dtype=work.dtype, device=DEV)
                md.mdfft_dist_pack(parts[g].plan.handle, s, G, g, work.data_ptr(), send.data_ptr(), st)
                sends.append(send)
            nxt = []
            for hh in range(G):  # the transport: group (g -> hh) of every sender, in sender order
                recv = torch.cat([sends[g][sum(counts[g][:hh]):sum(counts[g][:hh + 1])] for g in range(G)])
                assert recv.numel() == sum(counts[g][hh] for g in range(G))
                a, b = parts[hh].local_range(s + 1)
                out = torch.empty(b - a, dtype=recv.dtype, device=DEV)
                md.mdfft_dist_unpack(parts[hh].plan.handle, s, G, hh, recv.data_ptr(), out.data_ptr(), st)
                nxt.append(out)
            local = nxt
        torch.cuda.synchronize()
        y = torch.cat(local).cpu().numpy().reshape(shape)
        assert h is not None
        return y
    finally:
        for p in parts:
            p.close()


def rel(a, b):
    return float(np.linalg.norm(a.astype(np.complex128) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("shape,P,order,G", [((8, 6, 4), 4, "abc->acb->bca", 2), ((8, 6, 4), 6, "abc->cab->cba", 3),
                                             ((16, 12, 10), 16, None, 4), ((4, 6, 5, 2), 4, "abcd->abdc->dcab->dcba", 2),
                                             ((6, 4, 5, 3, 4), 24, None, 3), ((32, 32, 32), 4, "abc->cab->cba", 1),
                                             ((24, 20, 16, 12), 64, None, 8)])
def test_virtual_devices_match_the_oracle(shape, P, order, G, dt):
    x = si.uniform_complex(shape, 1900 + G)
    y = run_virtual(shape, P, order, dt, G, x)
    assert rel(y, oracle.fftn(x)) <= TOL[dt]
    back = run_virtual(shape, P, order, dt, G, y, dir=+1, normalize=True)
    assert rel(back, x) <= 2 * TOL[dt]


def test_a_line_split_between_devices_is_refused():
    # 4 x 4 x 4 with P = 32: the 3-D regime cuts lines; with G = 32 devices a
    # device boundary falls inside a line of the first layout
    shape = (4, 4, 4)
    with md.DistPlan(shape, 32, 32, 1) as dp:
        x = torch.zeros(64, dtype=torch.complex64, device=DEV)
        with pytest.raises(md.MdfftError) as e:
            md.mdfft_dist_lines(dp.plan.handle, 0, 32, 1, x.data_ptr(), x.data_ptr(), -1, 0, 0)
        assert e.value.status == -7
        with pytest.raises(md.MdfftError):
            md.mdfft_dist_pack(dp.plan.handle, 3, 2, 0, x.data_ptr(), x.data_ptr(), 0)  # step out of range
