"""The ring-of-slots pass kernel (a persistent CTA streaming its tiles
through S shared-memory slots filled by 16-byte asynchronous copies, with a
cap of resident CTAs per SM) and the one-thread-per-line kernel (every radix
stage on a line held in registers) compute exactly what the default pass
kernel computes: the same radix plan and butterflies in the same order.
Checked bit for bit on every length it is built for, on ragged tiles,
batches, the per-volume host path, the normalised inverse and count mode;
the spectrum is also checked against the oracle."""

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
RING = [v for v in md.mdfft.TUNING_VARIANTS if v.startswith("ring") or v.startswith("line")]


def ring_tuning(pl, variant, tile, base=None):
    """`base` (default: the plan's current tuning) with `variant` and `tile` on
    every pass whose length has it; the plan is left at `base`."""
    base = pl.tuning() if base is None else base
    chosen = [dict(d) for d in base]
    hit = []
    for s in range(len(base)):
        t = [dict(d) for d in base]
        t[s].update(variant=variant, tile_g=tile[0], tile_h=tile[1], tile_order=0)
        try:
            pl.set_tuning(t)
        except md.MdfftError:
            continue
        chosen[s] = t[s]
        hit.append(s)
    pl.set_tuning(base)
    return chosen, hit


@pytest.mark.parametrize("shape,P,batch", [((24, 20, 48), 16, 2), ((16, 32, 64, 6), 64, 1), ((96, 128, 10), 8, 1),
                                           ((256, 24, 12), 32, 2), ((64, 64, 30), 64, 1),
                                           ((24, 24, 24, 24), 64, 2), ((64, 64, 32, 16), 64, 1)])
def test_ring_variants_give_the_default_bits(shape, P, batch):
    x = torch.from_numpy(np.stack([si.uniform_complex(shape, 990 + b, np.complex64) for b in range(batch)])).to(DEV)
    if batch == 1:
        x = x[0]
    with md.Plan(shape, P, None, "c64", batch=batch) as pl:
        want = pl.exec(x)
        want_inv = pl.exec(want, dir=1, normalize=True)
        want_counts = pl.exec_counted(x)[1].cpu().tolist()
        default = pl.tuning()
        tried, walks = 0, 0.0
        for v in RING:
            for tile in ((8, 8), (5, 3), (16, 4), (24, 5)):
                # the variant on every pass it is built for, the default kernel elsewhere
                chosen, hit = ring_tuning(pl, v, tile, default)
                if not hit:
                    continue
                ref = want
                if "radix_alt" in v:  # compare with the non-ring kernel of the same radix plan
                    # (tiles never change results: 1 x 1 fits every kernel)
                    alt = [dict(d, variant="radix_alt", tile_g=1, tile_h=1, tile_order=0) if s in hit else d
                           for s, d in enumerate(chosen)]
                    pl.set_tuning(alt)
                    ref = pl.exec(x)
                pl.set_tuning(chosen)
                d = pl.describe()
                for s in hit:
                    if v.startswith("line"):
                        assert d[s]["persistent"] == 0 and d[s]["threads"] == (64 if v == "line2w" else 128), (v, s)
                        continue
                    assert d[s]["persistent"] in (2, 3) and d[s]["grid"] <= d[s]["ctas"], (v, s, d[s])
                    walks = max(walks, d[s]["ctas"] / d[s]["grid"])
                tried += 1
                assert torch.equal(pl.exec(x), ref), (v, tile, hit)
                assert torch.equal(pl.exec(x, graph=True), ref), (v, tile, hit)
                assert pl.exec_counted(x)[1].cpu().tolist() == want_counts, (v, tile, hit)
                if "radix_alt" not in v:
                    assert torch.equal(pl.exec(want, dir=1, normalize=True), want_inv), (v, tile, hit)
                    if batch > 1:  # volume by volume on the plan's streams (one volume per launch)
                        xh = x.cpu().pin_memory()
                        oh = torch.empty_like(xh).pin_memory()
                        pl.exec_host(xh, oh, torch.empty_like(x), torch.empty_like(x))
                        torch.cuda.synchronize(DEV)
                        assert torch.equal(oh, want.cpu()), (v, tile, hit)
        assert tried >= 1
        if shape in ((24, 24, 24, 24), (64, 64, 32, 16)):
            assert walks >= 3, walks  # CTAs walk several tiles: every slot and meta entry is reused


def test_ring_24_cubed_four_dims_against_the_oracle():
    # 24^4 with every pass on the three-CTA ring kernel: element-wise against
    # the FP64 oracle (the tolerance of the FP32 path in the parity tests)
    shape = (24, 24, 24, 24)
    x = si.uniform_complex(shape, 995, np.complex64)
    with md.Plan(shape, 64, None, "c64") as pl:
        chosen, hit = ring_tuning(pl, "ring2x3", (8, 8))
        assert hit == [0, 1, 2, 3]
        pl.set_tuning(chosen)
        got = pl.exec(torch.from_numpy(x).to(DEV)).cpu().numpy().astype(np.complex128)
    want = oracle.fftn(x, -1, nthreads=8)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-5, err


@pytest.mark.parametrize("shape,P,variant", [((24, 24, 24, 24), 64, "line"), ((16, 48, 32, 8), 16, "line"),
                                             ((64, 60, 40), 8, "line"), ((64, 64, 32, 8), 64, "line2t"),
                                             ((32, 64, 20), 16, "line2t_radix_alt")])
def test_line_kernel_on_every_pass_against_the_oracle(shape, P, variant):
    # every pass whose length has the one-thread-per-line (or two-threads-per-
    # line) kernel runs it, with the default tiles; element-wise against the
    # FP64 oracle, forward and normalised inverse
    x = si.uniform_complex(shape, 996, np.complex64)
    with md.Plan(shape, P, None, "c64") as pl:
        base = pl.tuning()
        chosen, hit = ring_tuning(pl, variant, (base[0]["tile_g"], base[0]["tile_h"]))
        if not hit:
            chosen, hit = ring_tuning(pl, variant, (8, 4))
        assert hit
        pl.set_tuning(chosen)
        xd = torch.from_numpy(x).to(DEV)
        got = pl.exec(xd)
        back = pl.exec(got, dir=1, normalize=True).cpu().numpy()
        got = got.cpu().numpy().astype(np.complex128)
    want = oracle.fftn(x, -1, nthreads=8)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-5, err
    assert np.abs(back - x).max() < 1e-5
