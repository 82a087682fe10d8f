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
                                        ((64, 48, 256), 16, "c64_tc_fp16"), ((512, 16, 8), 16, "c64_tc_bf16")])
def test_every_tuning_variant_gives_the_default_bits(shape, P, dt):
    # each kernel variant the autotuner may choose for these lengths (fixed
    # 192 / 384 / 256 / 512-thread CTAs; 128-thread tensor-core CTAs), set on
    # every pass where it is built, reproduces the default plan's spectrum
    x = torch.from_numpy(si.uniform_complex(shape, 970, np.complex64)).to(DEV)
    with md.Plan(shape, P, None, dt) as pl:
        want = pl.exec(x)
        base = pl.tuning()
        tried = 0
        for v in md.mdfft.TUNING_VARIANTS[1:]:
            if v.startswith("pipe"):
                continue
            for s in range(len(shape)):
                t = [dict(d) for d in base]
                t[s]["variant"], t[s]["tile_g"], t[s]["tile_h"] = v, 1, 1
                try:
                    pl.set_tuning(t)
                except md.MdfftError:
                    continue  # not built for this length
                d = pl.describe()[s]
                tried += 1
                assert torch.equal(pl.exec(x), want), (v, s, d)
        pl.set_tuning(base)
        assert tried >= 1
        y = torch.empty_like(x)
        pl.autotune(x, y, reps=2)
        assert torch.equal(pl.exec(x), want)
