"""The remaining entry points through the binding: per-pass timing, launches
per execution, the server's run loop and clock, and the thread-local error
message that accompanies a status."""

import numpy as np
import pytest
import torch

import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def test_pass_timing_and_launch_count():
    shape = (64, 48, 32)
    x = torch.from_numpy(si.uniform_complex(shape, 970, np.complex64)).to(DEV)
    with md.Plan(shape, 16) as pl:
        assert pl.launches() == 3
        pl.exec(x)
        pl.set_timing(True)
        for _ in range(7):
            pl.exec(x)
        ms, n = pl.pass_times()
        assert n == 7 and len(ms) == 3 and all(0 < v < 100 for v in ms)
        pl.set_timing(False)
        pl.exec(x)
        assert pl.pass_times()[1] == 7  # nothing recorded while off


def test_server_run_loop_and_clock():
    shapes = [(32, 48, 16), (16, 16, 16, 16), (64, 24, 32)]
    xs = [torch.from_numpy(si.uniform_complex(sh, 980 + i, np.complex64)).to(DEV) for i, sh in enumerate(shapes)]
    outs = [torch.empty_like(x) for x in xs]
    with md.Server(budget_bytes=1 << 28, max_inflight=8) as srv:
        srv.set_direct(0)  # batched steps only: one pass of every request per step
        srv.reset_clock()
        ids = [srv.submit(x, y) for x, y in zip(xs, outs)]
        for _ in range(100):
            srv.run(4)
            if all(srv.poll(i)[0] for i in ids):
                break
        srv.drain()
        times = [srv.poll(i)[1] for i in ids]
        assert all(t >= 0 for t in times)
        st = srv.stats()
        assert st["completed"] == 3 and st["steps"] >= 4  # a 4-D request needs four steps
        assert st["direct_requests"] == 0
    with md.Server(budget_bytes=1 << 28, max_inflight=8) as srv:  # default: low load runs them directly
        ids = [srv.submit(x, y) for x, y in zip(xs, outs)]
        srv.drain()
        st = srv.stats()
        assert st["completed"] == 3 and st["steps"] == 1 and st["direct_requests"] == 3
    for sh, x, y in zip(shapes, xs, outs):
        with md.Plan(sh, min(64, int(np.prod(sh)))) as pl:
            assert torch.equal(y, pl.exec(x))


def test_error_status_carries_the_message():
    with pytest.raises(md.MdfftError) as e:
        md.Plan((8, 8, 7), 4)  # 7 is not a built line length
    assert e.value.status == md.mdfft.MDFFT_E_UNSUPPORTED
    assert "line length 7" in str(e.value)


def test_fp64_rate_probe_measures_a_plausible_rate():
    # the complex128 roofline's denominator: a positive multiply-add rate well
    # below the FP32 class (GB300's FP64 rate is a small fraction of it)
    out = torch.empty(152 * 256, dtype=torch.float64, device=DEV)
    st = torch.cuda.current_stream(DEV).cuda_stream
    tf = md.mdfft_fp64_rate_probe(out.data_ptr(), 152, 256, st)
    assert 0.05 < tf < 20.0, tf
    assert torch.isfinite(out).all()
    with pytest.raises(md.MdfftError) as e:
        md.mdfft_fp64_rate_probe(out.data_ptr(), 0, 256, st)
    assert e.value.status == -1
    with pytest.raises(md.MdfftError):
        md.mdfft_fp64_rate_probe(0, 1, 1, st)
