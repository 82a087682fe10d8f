"""mdfft_exec_noalloc: the entry point for callers that cannot let a library
allocate GPU memory (their device memory belongs to their own allocator or
pool, or they cannot afford the synchronisation cudaMalloc/cudaFree may
cause).  Its scratch is a static device array, so two calls in a row must not
depend on what the previous call left there.

This file is collected last on purpose: it must pass alone in a fresh process
and after every other test."""

import numpy as np
import pytest
import torch

import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-12}  # the parity tolerances of the other GPU tests
NP = {"c64": np.complex64, "c128": np.complex128}
DEV = torch.device("cuda:0")


def rel_l2(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


CASES = [((64, 48, 40), "abc->cab->cba", "c64", 1),
         ((24, 20, 16, 12), "abcd->abdc->dcab->dcba", "c128", 2)]


def test_noalloc_matches_planned_exec_two_calls_in_a_row():
    stream = torch.cuda.current_stream(DEV).cuda_stream
    xs, outs = [], []
    for shape, order, dt, seed in CASES:
        x = torch.from_numpy(si.uniform_complex(shape, 400 + seed, NP[dt])).to(DEV)
        y = torch.empty_like(x)
        xs.append(x)
        outs.append(y)
    # two calls back to back on one stream: the second reuses the scratch the first left
    for (shape, order, dt, _), x, y in zip(CASES, xs, outs):
        md.mdfft_exec_noalloc(shape, order, dt, x.data_ptr(), y.data_ptr(), -1, 0, stream)
    torch.cuda.synchronize(DEV)
    for (shape, order, dt, _), x, y in zip(CASES, xs, outs):
        with md.Plan(shape, 4, order, dt) as plan:
            ref = plan.exec(x)
            torch.cuda.synchronize(DEV)
        assert rel_l2(y, ref) <= TOL[dt], (shape, dt)
    # and the inverse, normalised, brings the first input back
    shape, order, dt, _ = CASES[0]
    back = torch.empty_like(xs[0])
    md.mdfft_exec_noalloc(shape, order, dt, outs[0].data_ptr(), back.data_ptr(), +1, 1, stream)
    torch.cuda.synchronize(DEV)
    assert rel_l2(back, xs[0]) <= TOL[dt]


def test_noalloc_rejects_arrays_beyond_its_scratch():
    shape = (256, 256, 256)  # 128 MiB of complex64, over the 64 MiB scratch
    x = torch.empty(8, dtype=torch.complex64, device=DEV)
    y = torch.empty(8, dtype=torch.complex64, device=DEV)
    with pytest.raises(md.MdfftError) as e:  # refused before any launch: nothing is read or written
        md.mdfft_exec_noalloc(shape, "abc->cab->cba", "c64", x.data_ptr(), y.data_ptr(), -1, 0, 0)
    assert e.value.status == md.mdfft.MDFFT_E_UNSUPPORTED
    assert "MDFFT_NOALLOC_MAX_ARRAY_BYTES" in str(e.value)
    with pytest.raises(md.MdfftError) as e:
        md.mdfft_exec_noalloc((8, 8, 8), None, "c64", x.data_ptr(), x.data_ptr(), -1, 0, 0)
    assert e.value.status == md.mdfft.MDFFT_E_ARG


def test_noalloc_allocates_no_device_memory():
    # after one warm-up call (kernels loaded, the scratch address looked up),
    # further calls change neither torch's allocator nor the device's free memory
    shape, order, dt, seed = CASES[0]
    stream = torch.cuda.current_stream(DEV).cuda_stream
    x = torch.from_numpy(si.uniform_complex(shape, 420, NP[dt])).to(DEV)
    y = torch.empty_like(x)
    md.mdfft_exec_noalloc(shape, order, dt, x.data_ptr(), y.data_ptr(), -1, 0, stream)
    torch.cuda.synchronize(DEV)
    first = y.clone()
    torch.cuda.synchronize(DEV)
    torch_before = torch.cuda.memory_allocated(DEV)
    free_before = torch.cuda.mem_get_info(DEV)[0]
    for _ in range(4):
        md.mdfft_exec_noalloc(shape, order, dt, x.data_ptr(), y.data_ptr(), -1, 0, stream)
    torch.cuda.synchronize(DEV)
    assert torch.cuda.memory_allocated(DEV) == torch_before
    assert torch.cuda.mem_get_info(DEV)[0] == free_before
    assert torch.equal(y, first)  # the same bits on every call
