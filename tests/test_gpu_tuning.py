"""Stored launch choices: a plan's tuning (after autotuning) survives a JSON
round trip and, given to a fresh plan of the same problem, reproduces its
launch shapes and its results bit for bit; invalid tunings are refused
without changing the plan."""

import json

import numpy as np
import pytest
import torch

import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("shape,P,dt,batch", [((64, 48, 32), 16, "c64", 2), ((24, 20, 16, 12), 64, "c64", 1),
                                             ((32, 40, 24), 8, "c128", 1)])
def test_tuning_round_trip(shape, P, dt, batch):
    npdt = np.complex128 if dt == "c128" else np.complex64
    x = torch.from_numpy(np.stack([si.uniform_complex(shape, 950 + b, npdt) for b in range(batch)])).to(DEV)
    if batch == 1:
        x = x[0]
    with md.Plan(shape, P, None, dt, batch=batch) as a:
        a.autotune(x, torch.empty_like(x), reps=3)
        stored = json.dumps(a.tuning())
        want = a.exec(x)
        shapes = [{k: d[k] for k in ("threads", "tile_g", "tile_h", "ctas", "grid")} for d in a.describe()]
    with md.Plan(shape, P, None, dt, batch=batch) as b:
        b.set_tuning(json.loads(stored))
        assert [{k: d[k] for k in ("threads", "tile_g", "tile_h", "ctas", "grid")} for d in b.describe()] == shapes
        assert torch.equal(b.exec(x), want)
        assert torch.equal(b.exec(x, graph=True), want)


def test_invalid_tuning_is_refused_whole():
    shape = (64, 48, 32)
    x = torch.from_numpy(si.uniform_complex(shape, 960, np.complex64)).to(DEV)
    with md.Plan(shape, 16) as pl:
        before = pl.tuning()
        want = pl.exec(x)
        bad = [dict(t) for t in before]
        bad[-1]["tile_g"] = 4096  # larger than the kernel's lines
        with pytest.raises(md.MdfftError):
            pl.set_tuning(bad)
        bad = [dict(t) for t in before]
        bad[0]["variant"] = "thr256"  # valid on its own (32 has fixed-CTA variants) ...
        bad[1]["tile_h"] = 0  # ... but the second pass's tile is not, so nothing is applied
        with pytest.raises(md.MdfftError):
            pl.set_tuning(bad)
        assert pl.tuning() == before  # nothing applied
        assert torch.equal(pl.exec(x), want)


@pytest.mark.parametrize("shape,P,dt", [((24, 24, 24, 24), 64, "c64"), ((48, 24, 48), 16, "c64"),
                                        ((64, 32, 256), 16, "c64"), ((512, 12, 96), 16, "c64"),
                                        ((64, 48, 256), 16, "c64_tc_fp16"), ((512, 16, 8), 16, "c64_tc_bf16")])
def test_every_tuning_variant_gives_the_default_bits(shape, P, dt):
    # each kernel variant the autotuner may choose for these lengths (fixed
    # 192 / 384 / 256 / 512-thread CTAs; 128-thread tensor-core CTAs), set on
    # every pass where it is built, reproduces the default plan's spectrum
    x = torch.from_numpy(si.uniform_complex(shape, 970, np.complex64)).to(DEV)
    with md.Plan(shape, P, None, dt) as pl:
        want = pl.exec(x)
        want_counts = pl.exec_counted(x)[1].cpu().tolist()
        base = pl.tuning()
        pl_default_radix = [d["radix"] for d in pl.describe()]
        tried = 0
        for v in md.mdfft.TUNING_VARIANTS[1:]:
            if v.startswith("pipe"):
                continue
            for s in range(len(shape)):
                for order in (0, 1):
                    t = [dict(d) for d in base]
                    t[s]["variant"], t[s]["tile_g"], t[s]["tile_h"], t[s]["tile_order"] = v, 1, 1, order
                    try:
                        pl.set_tuning(t)
                    except md.MdfftError:
                        continue  # not built for this length, or no input-chunk order for this kernel
                    d = pl.describe()[s]
                    assert d["tile_order"] == order
                    tried += 1
                    y = pl.exec(x)
                    # every variant's count mode counts the same moved and split-line points
                    assert pl.exec_counted(x)[1].cpu().tolist() == want_counts, (v, s, d)
                    if "radix_alt" in v:  # another radix split: the same spectrum up to rounding
                        assert d["radix"] != pl_default_radix[s]
                        assert rel_l2(y, want) <= 1e-6, (v, s, d)
                    else:
                        assert torch.equal(y, want), (v, s, d)
        pl.set_tuning(base)
        assert torch.equal(pl.exec(x), want)  # the default radix plan's twiddles are back
        assert tried >= 1
        y = torch.empty_like(x)
        pl.autotune(x, y, reps=2)
        got = pl.exec(x)
        if any("radix_alt" in t["variant"] for t in pl.tuning()):
            assert rel_l2(got, want) <= 1e-6
        else:
            assert torch.equal(got, want)


def rel_l2(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_input_chunk_tile_order_gives_cta_t_chunk_t():
    # 64^3, P = 256 (the 2-D regime of layout abc: a chunk is 16 lines along b);
    # pass 0 in input-chunk tile order with 16 x 1 tiles has exactly P tiles,
    # tile t holding the lines of chunk t, and the same spectrum bit for bit
    shape, P = (64, 64, 64), 256
    x = torch.from_numpy(si.uniform_complex(shape, 975, np.complex64)).to(DEV)
    with md.Plan(shape, P, "abc->acb->bca") as pl:
        want = pl.exec(x)
        t = pl.tuning()
        t[0].update(variant="default", tile_g=16, tile_h=1, tile_order=1)
        pl.set_tuning(t)
        d = pl.describe()[0]
        assert d["tile_order"] == 1 and d["store_axis"] == 1 and d["ctas"] == P
        for pid in (0, 1, 77, P - 1):
            xs, xe, _, _ = md.mdfft_chunk(pl.handle, 0, pid, 3)
            # tile pid: lines (a = pid // 4, b = 16 (pid % 4) ... + 15), 64 points each
            assert xs == ((pid // 4) * 64 + 16 * (pid % 4)) * 64 and xe == xs + 16 * 64 - 1
        assert torch.equal(pl.exec(x), want)


def test_radix_search_is_opt_in_and_stays_within_the_bound():
    # with MDFFT_PLAN_TUNE_RADIX the autotuner may switch a pass to another
    # radix split (rounding changes only): the spectrum still meets the FP32
    # bound against the oracle, and the tuning records the plan per pass
    import oracle
    shape = (256, 64, 96)
    xh = si.uniform_complex(shape, 980)
    x = torch.from_numpy(xh.astype(np.complex64)).to(DEV)
    with md.Plan(shape, 16, None, "c64", md.MDFFT_PLAN_TUNE_RADIX) as pl:
        pl.autotune(x, torch.empty_like(x), reps=2)
        y = pl.exec(x).cpu().numpy().astype(np.complex128)
        passes = pl.describe()
    ref = oracle.fftn(xh, nthreads=8)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-5
    for d in passes:
        assert int(np.prod(d["radix"])) == d["line_length"]
        assert all(v in (2, 3, 4, 5, 8, 16) for v in d["radix"])
