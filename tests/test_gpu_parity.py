"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (relative L2 over the whole result, and per element against the
RMS of the reference):
  complex128 (FP64): 1e-12, the bound the build is held to;
  complex64 (FP32):  1e-5, the stated ceiling.  A radix-r Cooley-Tukey FFT
    with correctly rounded twiddles has an RMS relative error of order
    u * sqrt(log2 T) (u = 2^-24 = 6e-8); at T = 2^27 that is about 3e-7, so
    1e-5 leaves a margin of 30 while still catching a wrong twiddle or index
    (those give errors of order 1).
Integer results (communication counts) must match exactly.
"""

import os

import numpy as np
import pytest
import torch

import oracle
import paper_1302_6189_gb300 as md
import synth_inputs as si

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-12}
NP = {"c64": np.complex64, "c128": np.complex128}
NTH = os.cpu_count() or 4
DEV = torch.device("cuda:0")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check(y, ref, dt, what=""):
    y = y.astype(np.complex128)
    e = rel_l2(y, ref)
    assert e <= TOL[dt], f"{what} rel-L2 {e:.3e} > {TOL[dt]}"
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    emax = float(np.max(np.abs(y - ref)))
    assert emax <= 10 * TOL[dt] * rms, f"{what} max error {emax:.3e} vs rms {rms:.3e}"
    return e


def run(shape, P, order, dt, x, dir=-1, normalize=False):
    with md.Plan(shape, P, order, dt) as plan:
        xd = torch.from_numpy(np.ascontiguousarray(x.astype(NP[dt]))).to(DEV)
        y = plan.exec(xd, dir=dir, normalize=normalize)
        torch.cuda.synchronize()
        return y.cpu().numpy(), plan.order()


ORDERS3 = [oracle.format_order(o) for o in oracle.enumerate_orders(3)]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", ORDERS3)
def test_every_3d_order_small(dt, order):
    # several tiles and ragged last tiles along every axis
    for shape in [(20, 24, 12), (40, 6, 30), (16, 10, 48)]:
        x = si.uniform_complex(shape, 50)
        ref = oracle.fftn(x)
        y, _ = run(shape, 7, order, dt, x)
        check(y, ref, dt, f"{shape} {order}")
        yi, _ = run(shape, 7, order, dt, x, dir=+1)
        check(yi, oracle.fftn(x, sign=+1), dt, f"inverse {shape} {order}")


def test_parity_config_32cubed_c128():
    # 3-D complex128 32^3, P = 4, the prior-work order, forward + inverse
    shape = (32, 32, 32)
    x = si.uniform_complex(shape, si.SEEDS["parity32"])
    y, _ = run(shape, 4, "abc->cab->cba", "c128", x)
    check(y, oracle.fftn(x), "c128")
    back, _ = run(shape, 4, "abc->cab->cba", "c128", y, dir=+1, normalize=True)
    check(back, x, "c128", "round trip")


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("seed", range(4))
def test_random_4d_5d_orders(dt, seed):
    rng = np.random.default_rng(700 + seed)
    lengths = [1, 2, 3, 4, 5, 6, 8, 10, 12, 15, 16, 20, 24, 30, 32]
    for M in (4, 5):
        orders = oracle.enumerate_orders(M, cap=20000)
        o = orders[rng.integers(0, len(orders))]
        shape = tuple(int(rng.choice(lengths)) for _ in range(M))
        while int(np.prod(shape)) > 400000:
            shape = tuple(int(rng.choice(lengths[:10])) for _ in range(M))
        T = int(np.prod(shape))
        x = si.uniform_complex(shape, 60 + seed)
        y, _ = run(shape, int(rng.integers(1, T + 1)), o, dt, x)
        check(y, oracle.fftn(x, nthreads=NTH), dt, f"{shape} {oracle.format_order(o)}")


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_long_and_mixed_radix_lines(dt):
    for shape in [(1024, 6, 4), (4, 960, 5), (3, 8, 768), (640, 2, 12), (480, 10, 3), (384, 320, 2),
                  (240, 160, 6), (120, 96, 10), (80, 60, 40), (1, 512, 1), (5, 1, 1)]:
        x = si.uniform_complex(shape, 70)
        y, _ = run(shape, 3, None, dt, x)
        check(y, oracle.fftn(x, nthreads=NTH), dt, str(shape))


def test_plane_waves_have_exact_spectra():
    for shape in [(64, 16, 24, 32), (24, 24, 24, 24, 24)]:
        k0 = si.plane_wave_k0(shape, si.SEEDS["md_plane"])
        x = si.plane_wave(shape, k0)
        T = x.size
        for dt in ("c64", "c128"):
            y, _ = run(shape, 64, None, dt, x)
            expect = np.zeros(shape, np.complex128)
            expect[k0] = T
            err = float(np.max(np.abs(y.astype(np.complex128) - expect)))
            assert err <= 10 * TOL[dt] * T, (shape, dt, err)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_inverse_normalised_round_trip(dt):
    shape = (48, 40, 12)
    x = si.uniform_complex(shape, 80)
    with md.Plan(shape, 16, "abc->acb->bca", dt) as plan:
        xd = torch.from_numpy(x.astype(NP[dt])).to(DEV)
        y = plan.exec(xd)
        back = plan.exec(y, dir=+1, normalize=True)
        torch.cuda.synchronize()
        check(back.cpu().numpy(), x, dt, "round trip")
        assert torch.equal(xd, torch.from_numpy(x.astype(NP[dt])).to(DEV))  # input untouched


@pytest.mark.parametrize("shape,order", [((12, 20, 16), "abc->cab->cba"), ((6, 8, 10, 4), "abcd->abdc->dcab->dcba")])
def test_in_place(shape, order):
    x = si.uniform_complex(shape, 81)
    ref = oracle.fftn(x)
    with md.Plan(shape, 5, order, "c64", md.MDFFT_PLAN_INPLACE) as plan:
        xd = torch.from_numpy(x.astype(np.complex64)).to(DEV)
        plan.exec(xd, out=xd)
        torch.cuda.synchronize()
        check(xd.cpu().numpy(), ref, "c64", "in place")


def test_exec_argument_errors():
    shape = (8, 8, 8)
    with md.Plan(shape, 4, None, "c64") as plan:
        x = torch.zeros(shape, dtype=torch.complex64, device=DEV)
        y = torch.zeros(2 * 512 + 2, dtype=torch.complex64, device=DEV)
        h = plan.handle
        with pytest.raises(md.MdfftError) as e:
            md.mdfft_exec(h, x.data_ptr(), x.data_ptr(), -1, 0, 0)  # in place without the flag
        assert e.value.status == -1
        with pytest.raises(md.MdfftError):
            md.mdfft_exec(h, y.data_ptr(), y.data_ptr() + 8 * 3, -1, 0, 0)  # partial overlap
        with pytest.raises(md.MdfftError):
            md.mdfft_exec(h, y.data_ptr() + 4, y.data_ptr() + 8 * 600, -1, 0, 0)  # misaligned
        with pytest.raises(md.MdfftError):
            md.mdfft_exec(h, x.data_ptr(), y.data_ptr(), -1, 1, 0)  # normalise a forward
        with pytest.raises(md.MdfftError):
            md.mdfft_exec(h, x.data_ptr(), y.data_ptr(), 2, 0, 0)
        with pytest.raises(md.MdfftError):
            md.mdfft_exec(h, 0, y.data_ptr(), -1, 0, 0)


# ------------------------------------------------------------------ count mode

@pytest.mark.parametrize("shape,Ps", [((8, 8, 8), (1, 4, 8, 16, 40, 64, 100, 512)),
                                      ((6, 10, 4), (3, 7, 60, 61, 240)),
                                      ((4, 6, 5, 3), (2, 5, 24, 100, 360)),
                                      ((3, 4, 2, 5, 2), (7, 24, 100, 240))])
def test_device_counts_match_oracle_bit_exact(shape, Ps):
    M = len(shape)
    orders = oracle.enumerate_orders(M, cap=3000)
    rng = np.random.default_rng(11)
    x = si.uniform_complex(shape, 90)
    ref_y = oracle.fftn(x)
    for P in Ps:
        for idx in rng.choice(len(orders), size=min(len(orders), 8), replace=False):
            o = orders[idx]
            with md.Plan(shape, P, o, "c64") as plan:
                y, counts = plan.exec_counted(torch.from_numpy(x.astype(np.complex64)).to(DEV))
                torch.cuda.synchronize()
                got = counts.cpu().tolist()
                cv = oracle.comm_volume(shape, P, o)
                lib = plan.comm_volume()
            assert got[: M - 1] == cv["per_transition"] == lib["per_transition"]
            assert got[M - 1] == cv["final_to_natural"] == lib["final_to_natural"]
            assert got[M:] == cv["split_line"] == lib["split_line"]
            check(y.cpu().numpy(), ref_y, "c64", "counted")


@pytest.mark.parametrize("shape,kind,Ps", [((8, 12, 10), "slab", (3, 8)), ((8, 12, 10), "pencil", (6, 16, 40)),
                                           ((8, 12, 10), "volumetric", (12, 60, 960)),
                                           ((6, 8, 4, 5), "pencil", (4, 12)), ((6, 8, 4, 5), "volumetric", (24, 120)),
                                           ((64, 64, 64), "pencil", (16, 4096)),
                                           ((64, 64, 64), "volumetric", (8192, 262144))])
def test_device_counts_of_the_comparison_methods(shape, kind, Ps):
    # the Sec. 4 methods through the same passes: counts equal the oracle's
    # point-by-point ones, the spectrum is bit-identical to the row-wise plan's
    M = len(shape)
    orders = oracle.enumerate_orders(M, cap=3000)
    rng = np.random.default_rng(12)
    x = torch.from_numpy(si.uniform_complex(shape, 91).astype(np.complex64)).to(DEV)
    for P in Ps:
        for idx in rng.choice(len(orders), size=min(len(orders), 4), replace=False):
            o = orders[idx]
            axes = [L[-1] for L in o]
            try:
                ref = oracle.block_volume(shape, P, kind, axes)
            except ValueError:
                continue  # this order moves a cut onto an axis with fewer points
            with md.Plan(shape, P, o, "c64", md.DECOMPOSITIONS[kind]) as plan, md.Plan(shape, P, o, "c64") as rw:
                y, counts = plan.exec_counted(x)
                y_rw = rw.exec(x)
                torch.cuda.synchronize()
                got = counts.cpu().tolist()
            assert got[: M - 1] == ref["per_transition"], (kind, P, o)
            assert got[M - 1] == 0
            assert got[M:] == ref["split_line"], (kind, P, o)
            assert torch.equal(y, y_rw)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("shape,P,orders", [((20, 24, 12), 7, ORDERS3), ((8, 12, 10, 6), 16, None),
                                            ((6, 5, 8, 4, 3), 12, None)])
def test_output_in_the_last_layout(dt, shape, P, orders):
    # MDFFT_PLAN_OUT_LAST_LAYOUT: the spectrum stays in layout L_M (the last
    # pass stores whole lines); it is the natural-order result with the axes
    # permuted into L_M, bit for bit, forward and normalised inverse
    M = len(shape)
    if orders is None:
        orders = [oracle.format_order(o) for o in oracle.enumerate_orders(M, cap=400)[::97]]
    x = si.uniform_complex(shape, 57)
    xd = torch.from_numpy(np.ascontiguousarray(x.astype(NP[dt]))).to(DEV)
    ref = oracle.fftn(x)
    for order in orders:
        last = oracle.parse_order(order)[-1]
        with md.Plan(shape, P, order, dt, md.MDFFT_PLAN_OUT_LAST_LAYOUT) as pl, md.Plan(shape, P, order, dt) as pn:
            assert pl.out_shape == tuple(shape[a] for a in last)
            y = pl.exec(xd)
            assert torch.equal(y, pn.exec(xd).permute(*last).contiguous())
            yi = pl.exec(xd, dir=+1, normalize=True)
            assert torch.equal(yi, pn.exec(xd, dir=+1, normalize=True).permute(*last).contiguous())
            _, counts = pl.exec_counted(xd)
            assert counts[M - 1].item() == 0 and pl.comm_volume()["final_to_natural"] == 0
            assert counts[: M - 1].cpu().tolist() == pn.comm_volume()["per_transition"]
        check(y.cpu().numpy(), np.transpose(ref, last), dt, f"{shape} {order}")


def test_output_in_the_last_layout_batched_and_persistent():
    shape, P, B = (32, 48, 64), 12, 3
    x = torch.from_numpy(np.stack([si.uniform_complex(shape, 58 + i, np.complex64) for i in range(B)])).to(DEV)
    with md.Plan(shape, P, None, "c64", batch=B) as pn:
        want = pn.exec(x)
        last = pn.order()[-1]
    for flags in (md.MDFFT_PLAN_OUT_LAST_LAYOUT, md.MDFFT_PLAN_OUT_LAST_LAYOUT | md.MDFFT_PLAN_PERSISTENT):
        with md.Plan(shape, P, None, "c64", flags, batch=B) as pl:
            y = pl.exec(x)
            pl.check()
            assert torch.equal(y, want.permute(0, *[a + 1 for a in last]).contiguous())


# ------------------------------------------------------------------ full-size configurations

_REF = {}


def _ref(key, x):
    if key not in _REF:
        _REF[key] = oracle.fftn(x, nthreads=NTH)
    return _REF[key]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("P", [16, 256, 4096])
def test_256cubed_best_and_worst_orders(dt, P):
    shape = (256, 256, 256)
    x = si.uniform_complex(shape, si.SEEDS["cube256"])
    ref = _ref("cube256", x)
    best, _ = md.mdfft_order_search(shape, P, 0)
    worst, _ = md.mdfft_order_search(shape, P, 1)
    for o in (best, worst):
        y, _ = run(shape, P, o, dt, x)
        check(y, ref, dt, f"256^3 P={P} {md.format_order(o, 3)}")


def test_256cubed_every_order_c64():
    shape = (256, 256, 256)
    x = si.uniform_complex(shape, si.SEEDS["cube256"])
    ref = _ref("cube256", x)
    xd = torch.from_numpy(x.astype(np.complex64)).to(DEV)
    for o in ORDERS3:
        with md.Plan(shape, 4096, o, "c64") as plan:
            y = plan.exec(xd)
            back = plan.exec(y, dir=+1, normalize=True)
            torch.cuda.synchronize()
            check(y.cpu().numpy(), ref, "c64", o)
            check(back.cpu().numpy(), x, "c64", "round trip " + o)


def test_256cubed_counts_every_regime():
    # P = 131072 puts every layout in the 3-D regime (split lines)
    shape = (256, 256, 256)
    x = torch.zeros(shape, dtype=torch.complex64, device=DEV)
    for P in (16, 256, 4096, 131072):
        for o in ("abc->cab->cba", "abc->acb->bca"):
            with md.Plan(shape, P, o, "c64") as plan:
                _, counts = plan.exec_counted(x)
                got = counts.cpu().tolist()
                lib = plan.comm_volume()
            assert got[:2] == lib["per_transition"] and got[2] == lib["final_to_natural"]
            assert got[3:] == lib["split_line"]
    ref = oracle.comm_volume(shape, 131072, "abc->acb->bca")
    assert ref["per_transition"] == got[:2] and ref["split_line"] == got[3:]


@pytest.mark.parametrize("shape,P", [((64, 64, 64, 64), 64), ((64, 64, 64, 64), 1024),
                                     ((24, 24, 24, 24, 24), 64), ((24, 24, 24, 24, 24), 1024)])
def test_4d_5d_configs_best_and_worst(shape, P):
    x = si.uniform_complex(shape, si.SEEDS["md_uniform"])
    ref = _ref(("md", shape), x)
    for want in (0, 1):
        o, _ = md.mdfft_order_search(shape, P, want)
        y, _ = run(shape, P, o, "c64", x)
        check(y, ref, "c64", f"{shape} P={P}")


def test_autotune_keeps_results_bit_identical():
    for shape, dt in [((256, 128, 64), "c64"), ((96, 48, 160), "c64"), ((64, 32, 48), "c128")]:
        x = torch.from_numpy(si.uniform_complex(shape, 95, NP[dt])).to(DEV)
        with md.Plan(shape, 16, None, dt) as plan:
            before = plan.exec(x)
            scratch = torch.empty_like(x)
            ms0, ms1 = plan.autotune(x, scratch, reps=3)
            assert all(b <= a * 1.05 + 1e-3 for a, b in zip(ms0, ms1))  # never picks a slower configuration
            after = plan.exec(x)
            torch.cuda.synchronize()
            if any("radix_alt" in t["variant"] for t in plan.tuning()):  # another radix split: rounding only
                check(after.cpu().numpy(), oracle.fftn(x.cpu().numpy().astype(np.complex128)), dt, str(shape))
            else:
                assert torch.equal(before, after), shape
            for d in plan.describe():
                assert d["tile_g"] * d["tile_h"] * (d["threads"] // max(1, d["threads"])) >= 1


def test_pattern_probe_moves_the_data_of_a_pass():
    # the probe kernel writes the input, untransformed, into the next layout
    shape = (64, 48, 32)
    x = torch.from_numpy(si.uniform_complex(shape, 97, np.complex64)).to(DEV)
    out = torch.empty_like(x)
    with md.Plan(shape, 4, "abc->acb->bca", "c64") as plan:
        ms = plan.pattern_probe(0, x, out, reps=2)
        torch.cuda.synchronize()
    assert ms > 0
    # pass 0 goes from layout abc to acb: element (a, b, c) lands at (a, c, b)
    got = out.cpu().numpy().reshape(64, 32, 48)
    assert np.array_equal(got, np.transpose(x.cpu().numpy(), (0, 2, 1)))


@pytest.mark.parametrize("shape,P", [((64, 48, 32), 4), ((24, 20, 24, 24), 64), ((40, 64, 30), 16)])
def test_movement_probe_moves_what_the_pattern_probe_moves(shape, P):
    # the ring-structured probe (persistent CTAs, 2 or 3 slots, a CTA cap per
    # SM) writes exactly the pattern probe's output, every pass it is built for
    x = torch.from_numpy(si.uniform_complex(shape, 96, np.complex64)).to(DEV)
    with md.Plan(shape, P, None, "c64") as plan:
        probed = 0
        for s in range(len(shape)):
            want = torch.zeros_like(x)
            try:
                plan.pattern_probe(s, x, want, reps=1)
            except md.MdfftError:
                continue
            for slots, per_sm in ((2, 3), (3, 2), (2, 1)):
                got = torch.zeros_like(x)
                try:
                    ms = plan.movement_probe(s, x, got, slots, per_sm, reps=2)
                except md.MdfftError as e:
                    assert e.status == -7, e  # E_UNSUPPORTED: no ring build for this length
                    break
                assert ms > 0
                assert torch.equal(got, want), (s, slots, per_sm)
                probed += 1
        assert probed >= 3
        with pytest.raises(md.MdfftError):
            plan.movement_probe(0, x, torch.empty_like(x), 4, 2)
        with pytest.raises(md.MdfftError):
            plan.movement_probe(0, x, torch.empty_like(x), 2, 0)


@pytest.mark.parametrize("shape", [(4, 2, 3, 2, 4, 2), (2, 2, 3, 2, 2, 2, 5), (2, 3, 2, 2, 2, 2, 2, 4)])
def test_six_to_eight_dims_with_the_heuristic_order(shape):
    x = si.uniform_complex(shape, 98)
    for dt in ("c64", "c128"):
        y, _ = run(shape, 5, None, dt, x)
        check(y, oracle.fftn(x), dt, str(shape))
        yi, _ = run(shape, 5, None, dt, x, dir=+1, normalize=True)
        check(yi * 1.0, oracle.fftn(x, sign=+1) / x.size, dt, "inverse " + str(shape))


@pytest.mark.parametrize("shape,P,B", [((256, 256, 256), 4096, 8), ((64, 64, 64, 64), 64, 4), ((24, 24, 24, 24, 24), 64, 4)])
def test_benchmark_launch_configurations_against_the_oracle(shape, P, B):
    # the launches the benchmark times: a batched plan of B volumes, autotuned
    # with radix splits allowed (kernel variant, tiles, tile order, radix plan
    # per pass); the first and the last volume of the batch, every element,
    # against the oracle, and the normalised inverse back to the input
    vols = [si.uniform_complex(shape, 1303 + i) for i in (0, B - 1)]
    x = torch.empty((B,) + shape, dtype=torch.complex64, device=DEV)
    for i in range(B):
        src = vols[0] if i == 0 else vols[1] if i == B - 1 else si.uniform_complex(shape, 1303 + i)
        x[i].copy_(torch.from_numpy(src.astype(np.complex64)))
    with md.Plan(shape, P, None, "c64", md.MDFFT_PLAN_TUNE_RADIX, batch=B) as plan:
        plan.autotune(x, torch.empty_like(x), reps=2)
        y = plan.exec(x)
        back = plan.exec(y, dir=+1, normalize=True)
        torch.cuda.synchronize()
        for i, v in ((0, vols[0]), (B - 1, vols[1])):
            check(y[i].cpu().numpy(), oracle.fftn(v, nthreads=NTH), "c64", f"{shape} volume {i}")
            check(back[i].cpu().numpy(), v, "c64", f"{shape} round trip {i}")
