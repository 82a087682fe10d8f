"""Tensor-core dtypes (radix-16 stages as FP16 or BF16 split hi/lo GEMMs with
FP32 accumulation) against the FP64 oracle.

Stated bounds (relative L2 over the result):
  MDFFT_C64_TC_FP16: 1e-5.  hi + lo carries 22 bits of every operand and the
    dropped lo*lo product is below 2^-22, so the stage error is that of FP32
    arithmetic (~1e-7 per stage); 1e-5 is the ceiling.
  MDFFT_C64_TC_BF16: 1e-4.  hi + lo carries 16 bits (BF16 has 8), so each
    radix-16 stage adds ~2^-17 relative error; with up to two radix-16
    stages per pass and three passes the RMS stays near 1e-5; 1e-4 is the
    ceiling.
Lines whose length is not a multiple of 16 run on the FP32 SIMT kernel.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu

TOL = {"c64_tc_fp16": 1e-5, "c64_tc_bf16": 1e-4}
DEV = torch.device("cuda:0")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(shape, P, order, dt, x, dir=-1, normalize=False):
    with md.Plan(shape, P, order, dt) as plan:
        xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).to(DEV)
        y = plan.exec(xd, dir=dir, normalize=normalize)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("dt", ["c64_tc_fp16", "c64_tc_bf16"])
@pytest.mark.parametrize("shape", [(64, 48, 32), (16, 80, 24), (512, 16, 6), (32, 1024, 2), (240, 160, 12),
                                   (96, 96, 96), (16, 16, 16, 16), (32, 48, 16, 8, 4)])
def test_tc_matches_oracle(dt, shape):
    x = si.gaussian_complex(shape, 1306)
    ref = oracle.fftn(x, nthreads=8)
    for order in (None, "worst"):
        o = None
        if order == "worst":
            o, _ = md.mdfft_order_search(shape, 7, 1)
        y = run(shape, 7, o, dt, x)
        e = rel_l2(y, ref)
        assert e <= TOL[dt], (shape, dt, e)
    yi = run(shape, 7, None, dt, x, dir=+1)
    assert rel_l2(yi, oracle.fftn(x, sign=+1, nthreads=8)) <= TOL[dt]


@pytest.mark.parametrize("dt", ["c64_tc_fp16", "c64_tc_bf16"])
def test_tc_round_trip_and_large_values(dt):
    shape = (128, 64, 32)
    x = si.gaussian_complex(shape, 77) * 3e4  # FP16 range needs the per-row scale
    y = run(shape, 16, None, dt, x)
    assert rel_l2(y, oracle.fftn(x, nthreads=8)) <= TOL[dt]
    back = run(shape, 16, None, dt, y, dir=+1, normalize=True)
    assert rel_l2(back, x) <= 2 * TOL[dt]


@pytest.mark.parametrize("dt", ["c64_tc_fp16", "c64_tc_bf16"])
def test_tc_batched_and_last_layout(dt):
    # a batch of three through one launch per pass equals each volume alone,
    # and the last-layout output is the permuted natural one, bit for bit
    shape, P, B = (32, 48, 64), 16, 3
    vols = [si.gaussian_complex(shape, 930 + b) for b in range(B)]
    x = torch.from_numpy(np.stack([v.astype(np.complex64) for v in vols])).to(DEV)
    with md.Plan(shape, P, None, dt, batch=B) as pb, md.Plan(shape, P, None, dt) as p1, \
            md.Plan(shape, P, None, dt, md.MDFFT_PLAN_OUT_LAST_LAYOUT, batch=B) as pl:
        y = pb.exec(x)
        yl = pl.exec(x)
        last = pl.order()[-1]
        for b in range(B):
            assert torch.equal(y[b], p1.exec(x[b].contiguous()))
        assert torch.equal(yl, y.permute(0, *[a + 1 for a in last]).contiguous())
        torch.cuda.synchronize()
    for b in range(B):
        ref = oracle.fftn(vols[b])
        assert rel_l2(y[b].cpu().numpy().astype(np.complex128), ref) < TOL[dt]


@pytest.mark.parametrize("dt", ["c64_tc_fp16", "c64_tc_bf16"])
def test_tc_persistent_passes_counts_and_status(dt):
    # every pass of this shape is a tensor-core pass: persistent (at most one
    # resident wave, several tiles per CTA); count mode adds the oracle's
    # amounts per volume, no bounded wait gives up, and the spectra hold
    shape, P, B = (64, 48, 32), 24, 2
    vols = [si.gaussian_complex(shape, 950 + b) for b in range(B)]
    x = torch.from_numpy(np.stack([v.astype(np.complex64) for v in vols])).to(DEV)
    with md.Plan(shape, P, None, dt, batch=B) as pl:
        passes = pl.describe()
        assert all(p["persistent"] == 1 and 1 <= p["grid"] <= p["ctas"] for p in passes), passes
        _, counts = pl.exec_counted(x)
        y = pl.exec(x)
        back = pl.exec(y, dir=+1, normalize=True)
        torch.cuda.synchronize()
        pl.check()
        c = counts.cpu().tolist()
        order = pl.order()
    ref = oracle.comm_volume(shape, P, order)
    assert c[:2] == [B * v for v in ref["per_transition"]]
    assert c[2] == B * ref["final_to_natural"]
    assert c[3:] == [B * v for v in ref["split_line"]]
    for b in range(B):
        assert rel_l2(y[b].cpu().numpy().astype(np.complex128), oracle.fftn(vols[b])) < TOL[dt]
        assert rel_l2(back[b].cpu().numpy().astype(np.complex128), vols[b]) < 2 * TOL[dt]


def test_tc_plans_need_16_byte_alignment():
    # the tensor-core kernel copies whole lines with bulk copies: refused on
    # the host before any launch
    shape = (32, 48, 16)
    T = 32 * 48 * 16
    with md.Plan(shape, 4, None, "c64_tc_fp16") as plan:
        buf = torch.zeros(T + 2, dtype=torch.complex64, device=DEV)
        out = torch.zeros(T + 2, dtype=torch.complex64, device=DEV)
        with pytest.raises(md.MdfftError) as e:
            md.mdfft_exec(plan.handle, buf.data_ptr() + 8, out.data_ptr(), -1, 0, 0)
        assert e.value.status == -1
        with pytest.raises(md.MdfftError) as e:
            md.mdfft_exec(plan.handle, buf.data_ptr(), out.data_ptr() + 8, -1, 0, 0)
        assert e.value.status == -1
