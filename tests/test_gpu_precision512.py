"""The precision configuration at its full size: 512^3, re/im ~ N(0, 1) from
seed 1306, P = 4096, the planner's best order, forward transform.  Every
output element of every dtype is compared with the FP64 oracle's spectrum of
the same input (the M-D DFT of Sec. 2), not a sample of points.

Bounds (relative L2 over the result; per element against the RMS of the
oracle's spectrum), the ones the other parity tests state:
  complex128 1e-12, complex64 FP32 SIMT 1e-5, tensor-core FP16 hi-lo 1e-5,
  tensor-core BF16 hi-lo 1e-4.
"""

import os

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu

SHAPE = (512, 512, 512)
P = 4096
TOL = {"c64": 1e-5, "c64_tc_fp16": 1e-5, "c64_tc_bf16": 1e-4, "c128": 1e-12}
DEV = torch.device("cuda:0")
NTH = len(os.sched_getaffinity(0))


@pytest.fixture(scope="module")
def case():
    x = si.gaussian_complex(SHAPE, si.SEEDS["precision512"], dtype=np.complex64)
    ref = oracle.fftn(x, nthreads=NTH)  # the complex64 draw, widened: both sides see the same input
    return x, ref


def errors(y, ref):
    """rel-L2, max |y - ref| and RMS of ref, accumulated one slab at a time."""
    num = den = 0.0
    emax = 0.0
    for i in range(0, y.shape[0], 32):
        d = y[i:i + 32].astype(np.complex128) - ref[i:i + 32]
        a = np.abs(d)
        num += float(np.sum(a * a))
        r = np.abs(ref[i:i + 32])
        den += float(np.sum(r * r))
        emax = max(emax, float(a.max()))
    return (num / den) ** 0.5, emax, (den / ref.size) ** 0.5


@pytest.mark.parametrize("dt", ["c64", "c64_tc_fp16", "c64_tc_bf16", "c128"])
def test_512cubed_every_element_against_the_oracle(case, dt):
    x, ref = case
    xd = torch.from_numpy(x).to(DEV)
    if dt == "c128":
        xd = xd.to(torch.complex128)
    with md.Plan(SHAPE, P, None, dt) as plan:
        y = plan.exec(xd)
        torch.cuda.synchronize()
        plan.check()
    del xd
    yh = y.cpu().numpy()
    del y
    e, emax, rms = errors(yh, ref)
    assert e <= TOL[dt], f"{dt}: rel-L2 {e:.3e} > {TOL[dt]}"
    assert emax <= 10 * TOL[dt] * rms, f"{dt}: max error {emax:.3e} vs rms {rms:.3e}"
    print(f"512^3 {dt}: rel-L2 {e:.3e}, max {emax / rms:.3e} x rms")
