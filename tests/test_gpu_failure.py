"""Failure detection without a GPU fault: the bounded device wait used by
the persistent pipelined kernels gives up after its limit when the bytes it
waits for never arrive, the call reports MDFFT_E_TIMEOUT, and the device
stays usable for the next transform."""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    st, us = md.mdfft_selftest_wait(0, 200_000)  # 16 bytes that no copy brings
    assert st == md.mdfft.MDFFT_E_TIMEOUT
    assert 200_000 <= us < 5_000_000
    st, us = md.mdfft_selftest_wait(1, 200_000)  # a plain arrival completes the phase
    assert st == md.mdfft.MDFFT_OK and us < 200_000
    x = si.uniform_complex((16, 24, 20), 901)
    with md.Plan((16, 24, 20), 8, None, "c128") as pl:
        y = pl.exec(torch.from_numpy(x).to(DEV)).cpu().numpy()
        pl.check()
    ref = oracle.fftn(x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-12
