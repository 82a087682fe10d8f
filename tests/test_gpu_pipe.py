"""The persistent, bulk-copy (TMA) pipelined pass kernel (MDFFT_PLAN_PERSISTENT)
gives exactly the bits of the default kernels: same tiles, same arithmetic
per line; only how the tiles' input reaches shared memory differs."""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
ORDERS3 = [oracle.format_order(o) for o in oracle.enumerate_orders(3)]


def both(shape, P, order, x, dir=-1, normalize=False):
    outs = []
    for flags in (0, md.MDFFT_PLAN_PERSISTENT):
        with md.Plan(shape, P, order, "c64", flags) as plan:
            outs.append(plan.exec(x, dir=dir, normalize=normalize))
            torch.cuda.synchronize()
            plan.check()
    return outs


@pytest.mark.parametrize("order", ORDERS3)
def test_pipelined_equals_default_every_order(order):
    for shape in [(64, 48, 32), (96, 160, 16), (256, 20, 12), (24, 512, 6)]:
        x = torch.from_numpy(si.uniform_complex(shape, 40, np.complex64)).to(DEV)
        a, b = both(shape, 9, order, x)
        assert torch.equal(a, b), (shape, order)
        a, b = both(shape, 9, order, x, dir=+1, normalize=True)
        assert torch.equal(a, b), (shape, order, "inverse")


def test_pipelined_matches_oracle_and_counts():
    shape = (128, 96, 64)
    x = si.uniform_complex(shape, 41)
    xd = torch.from_numpy(x.astype(np.complex64)).to(DEV)
    ref = oracle.fftn(x, nthreads=8)
    with md.Plan(shape, 100, None, "c64", md.MDFFT_PLAN_PERSISTENT) as plan:
        y, counts = plan.exec_counted(xd)
        torch.cuda.synchronize()
        plan.check()
        cv = plan.comm_volume()
        got = counts.cpu().tolist()
        assert got[:2] == cv["per_transition"] and got[2] == cv["final_to_natural"]
        assert got[3:] == cv["split_line"]
        assert any(d["threads"] > 0 for d in plan.describe())
    yh = y.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(yh - ref) / np.linalg.norm(ref) <= 1e-5


def test_pipelined_full_size_and_many_tiles_per_cta():
    shape = (256, 256, 256)  # 4096 tiles per pass, a few waves of persistent CTAs
    x = torch.from_numpy(si.uniform_complex(shape, si.SEEDS["cube256"], np.complex64)).to(DEV)
    a, b = both(shape, 4096, None, x)
    assert torch.equal(a, b)
    shape4 = (64, 64, 64, 64)
    x4 = torch.from_numpy(si.uniform_complex(shape4, 42, np.complex64)).to(DEV)
    a, b = both(shape4, 64, None, x4)
    assert torch.equal(a, b)


def test_pipelined_needs_16_byte_alignment():
    shape = (32, 32, 32)
    with md.Plan(shape, 4, None, "c64", md.MDFFT_PLAN_PERSISTENT) as plan:
        buf = torch.zeros(2 * 32 ** 3 + 4, dtype=torch.complex64, device=DEV)
        out = torch.zeros(32 ** 3 + 2, dtype=torch.complex64, device=DEV)
        with pytest.raises(md.MdfftError) as e:  # refused on the host before any launch
            md.mdfft_exec(plan.handle, buf.data_ptr() + 8, out.data_ptr(), -1, 0, 0)
        assert e.value.status == -1
