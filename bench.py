#!/usr/bin/env python
"""Throughput benchmark of the row-wise decomposed M-D FFT on GB300.

Workload (one "step"): forward + normalised inverse 3-D complex64 FFT of a
batch of B = 8 distinct 256x256x256 volumes (seeded U[-1,1) re/im), P = 4096
virtual processes, the planner's best transpose order.  Every volume is
128 MiB, larger than the 126 MB L2, and the step walks through 8 of them, so
no L2 flush is needed between steps.

value = algorithmic bytes / device time, the algorithmic bytes of one
transform being 2 * M * T * 8 (M fused passes, each reading and writing the
array once; the transposes are inside the passes).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (under torchrun) every rank runs an independent replica on
its own GPU (the path has no exchange step on one node's GPUs here); rank 0
prints the line with the max time over ranks.  --impl reference times the CPU
FP64 oracle on the host cores instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "M-D FFT GB/s & % HBM peak vs plain; served FFT/s, p50/p99 at stated error"
SHAPE = (256, 256, 256)
P_DEFAULT = 4096
PROFILE = os.path.join(ROOT, "profiles", "fft_pass_256cubed_c64.md")
# everything the profiled kernels are compiled from: every CUDA source and
# header of the library (the autotuner may pick any variant), and the build
# script that holds the nvcc flags
_CSRC = os.path.join(ROOT, "paper_1302_6189_gb300", "csrc")
KERNEL_SOURCES = sorted(os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith((".cu", ".cuh", ".h"))) + \
                 [os.path.join(ROOT, "paper_1302_6189_gb300", "build.py")]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--P", type=int, default=P_DEFAULT)
    ap.add_argument("--no-extra", action="store_true", help="skip the per-order / complex128 table")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--profile-case", action="store_true",
                    help="one warm-up and one profiled forward transform of a batch of 256^3 volumes "
                         "(3 + 3 pass launches), for ncu captures")
    ap.add_argument("--profile-batch", type=int, default=8, help="volumes per launch in --profile-case")
    ap.add_argument("--profile-dtype", default="c64", choices=["c64", "c128", "c64_tc_fp16", "c64_tc_bf16"])
    ap.add_argument("--profile-shape", default="256,256,256", help="grid of --profile-case, e.g. 64,64,64,64")
    ap.add_argument("--profile-tuning", default=None,
                    help="--profile-case applies this tuning record (JSON: one entry for every pass, or a list)")
    ap.add_argument("--profile-tune", action="store_true",
                    help="--profile-case autotunes the plan first (radix splits included), as the bench's studies do")
    ap.add_argument("--serving-only", type=int, default=0, metavar="REQUESTS",
                    help="run only the serving study with this many requests and print it")
    ap.add_argument("--serving-budget-gb", type=float, default=40.0)
    return ap.parse_args()


PROFILE_C128 = os.path.join(ROOT, "profiles", "fft_pass_256cubed_c128.md")


def fp64_peak(dev):
    """The device's FP64 multiply-add rate in TFLOP/s, measured by the
    library's probe kernel (CUDA events; 8 waves of 256-thread CTAs)."""
    import torch

    from paper_1302_6189_gb300 import mdfft_fp64_rate_probe
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ctas = sms * 8 * 8
    out = torch.empty(ctas * 256, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    return max(mdfft_fp64_rate_probe(out.data_ptr(), ctas, 4096, stream) for _ in range(3))


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_values(path=PROFILE):
    """The `key: value` lines (traffic_bytes_*, dp_*) of a committed ncu
    summary, if it was taken on the current kernel sources (else {})."""
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return {}
    kv = {}
    for line in text.splitlines():
        t = line.strip()
        if ":" in t and t.startswith(("traffic_bytes", "kernel_source_sha256", "dp_")):
            k, v = t.split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.pop("kernel_source_sha256", None) != kernel_hash():
        return {}
    out = {}
    for k, v in kv.items():
        try:
            out[k] = int(float(v))
        except ValueError:
            pass
    return out


def profile_traffic(path=PROFILE, key="traffic_bytes_per_launch"):
    """DRAM bytes per launch from a committed ncu summary taken on the current
    kernel sources (else None)."""
    return profile_values(path).get(key)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "20", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        sm = []
        smax = None
        power = []
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                power.append(float(r[3]))
            except ValueError:
                continue
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world):
    """Max of a per-rank time over all ranks (NCCL: on the device; gloo: on the host)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_bytes(shape, elem):
    T = 1
    for n in shape:
        T *= n
    return 2 * len(shape) * T * elem, T


# ---------------------------------------------------------------------------- CPU oracle

def oracle_fwd_inv_seconds(shape, reps, nthreads):
    """Wall time of `reps` forward + inverse FP64 oracle transforms of one volume."""
    import numpy as np

    import oracle
    import synth_inputs as si
    x = si.uniform_complex(shape, si.SEEDS["cube256"])
    y = np.empty_like(x)
    times = []
    for _ in range(reps):
        np.copyto(y, x)
        t0 = time.perf_counter()
        oracle.fftn_inplace(y, -1, nthreads)
        oracle.fftn_inplace(y, +1, nthreads)
        times.append(time.perf_counter() - t0)
    return times


def cpu_model():
    try:  # lscpu names Arm cores too (its "Model name"); /proc/cpuinfo only has their part number there
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_spectrum(x, nthreads):
    """The FP64 oracle's forward transform of the host array x, and its wall
    time: the checker the GPU results of the bench are stated against (this
    and cpu_baseline are the only places the bench runs the oracle)."""
    import numpy as np

    import oracle
    y = np.array(x, dtype=np.complex128, order="C")
    t0 = time.perf_counter()
    oracle.fftn_inplace(y, -1, nthreads)
    return y, time.perf_counter() - t0


def errors_vs(y, ref):
    """rel-L2 of y against ref and the largest element error over ref's RMS
    (accumulated slab by slab along the first axis)."""
    import numpy as np
    num = den = emax = 0.0
    for i in range(0, y.shape[0], 32):
        d = np.abs(y[i:i + 32].astype(np.complex128) - ref[i:i + 32])
        r = np.abs(ref[i:i + 32])
        num += float(np.sum(d * d))
        den += float(np.sum(r * r))
        emax = max(emax, float(d.max()))
    rms = (den / ref.size) ** 0.5
    return {"rel_l2": (num / den) ** 0.5, "max_err_over_rms": emax / rms}


def cpu_baseline(shape, elem, fwd0=None):
    """The oracle timed on the host cores (forward + inverse of one volume);
    with fwd0 (the GPU forward spectrum of volume 0 of the bench workload) also
    the error of that result against the oracle's."""
    nthreads = len(os.sched_getaffinity(0))
    # about 20 s of CPU work: one forward + inverse takes ~0.25 s on 16 cores
    reps = max(2, min(12, int(round(80 / max(1, nthreads)))))
    times = oracle_fwd_inv_seconds(shape, reps, nthreads)
    per_step, _ = algorithmic_bytes(shape, elem)
    gbs = 2 * per_step * reps / sum(times) / 1e9
    out = {"value": round(gbs, 3), "unit": "GB/s", "cores": nthreads, "kind": "oracle",
           "sample": f"{reps} x (forward + inverse) of one {'x'.join(map(str, shape))} volume, FP64 oracle "
                     f"(complex128) on {nthreads} host threads; bytes counted as for the complex64 GPU path",
           "seconds": round(sum(times), 3), "cpu": cpu_model()}
    if fwd0 is not None:
        import numpy as np

        import synth_inputs as si
        x = si.uniform_complex(shape, si.SEEDS["cube256"]).astype(np.complex64)  # the GPU's input, widened
        ref, _ = oracle_spectrum(x, nthreads)
        out["forward_vs_oracle_volume0"] = errors_vs(fwd0, ref)
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nthreads = len(os.sched_getaffinity(0))
    per_transform, _ = algorithmic_bytes(SHAPE, 8)
    # warm-up and timed steps; one step = forward + inverse of one volume (a
    # bounded sample of the 8-volume step of the GPU arm)
    oracle_fwd_inv_seconds(SHAPE, max(0, args.warmup), nthreads) if args.warmup else None
    times = oracle_fwd_inv_seconds(SHAPE, args.steps, nthreads)
    total = sum(times)
    gbs = 2 * per_transform * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "3-D FFT 256x256x256 forward+inverse, oracle sample of 1 volume per step",
                       "P": args.P, "parallelism": "host threads"},
            "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": nthreads, "kind": "oracle",
                             "sample": "one 256^3 volume forward + inverse per step (FP64)"},
            "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU arm

def host_link_gbs(h_in, d_in, h_out, d_out, reps=3):
    """Copy-engine bandwidth between pinned host memory and the GPU: each
    direction alone and both at once (two streams), over the bench's buffers."""
    import torch

    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    cur = torch.cuda.current_stream()
    nbytes = h_in.numel() * h_in.element_size()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        for _ in range(reps):
            fn()
        b.record(cur)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def both():
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            d_in.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    h2d = timed(lambda: d_in.copy_(h_in, non_blocking=True))
    d2h = timed(lambda: h_out.copy_(d_out, non_blocking=True))
    conc = timed(both)
    return {"h2d_gbs": round(nbytes / (h2d * 1e-3) / 1e9, 1), "d2h_gbs": round(nbytes / (d2h * 1e-3) / 1e9, 1),
            "concurrent_gbs": round(2 * nbytes / (conc * 1e-3) / 1e9, 1)}


def run_ours(args):
    import numpy as np
    import torch

    import synth_inputs as si
    from paper_1302_6189_gb300 import MDFFT_PLAN_TUNE_RADIX, Plan, format_order, mdfft_order_search

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    shape, B, P = SHAPE, args.batch, args.P
    elem = 8
    per_transform, T = algorithmic_bytes(shape, elem)
    order, total_amount = mdfft_order_search(shape, P, 0)
    # one batched plan: every pass is one launch over the tiles of all B volumes
    # (the autotuner may also pick another radix split of the line length)
    plan = Plan(shape, P, order, "c64", MDFFT_PLAN_TUNE_RADIX, batch=B)
    comm = plan.comm_volume()

    xs = torch.empty((B,) + shape, dtype=torch.complex64, device=dev)
    for i in range(B):
        xs[i].copy_(torch.from_numpy(si.uniform_complex(shape, si.SEEDS["cube256"] + i, np.complex64)))
    ys = torch.empty_like(xs)
    zs = torch.empty_like(xs)
    stream = torch.cuda.current_stream(dev)
    nvtx = torch.cuda.nvtx
    nvtx.range_push("autotune")
    tune_before, tune_after = plan.autotune(xs, ys, reps=5)
    nvtx.range_pop()
    tuned = [{k: d[k] for k in ("threads", "tile_g", "tile_h", "ctas", "radix", "tile_order")} for d in plan.describe()]

    def step():
        plan.exec(xs, ys, dir=-1)
        plan.exec(ys, zs, dir=+1, normalize=True)

    nvtx.range_push("warmup")
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    nvtx.range_pop()
    err = float((torch.linalg.vector_norm(zs[0] - xs[0]) / torch.linalg.vector_norm(xs[0])).item())
    fwd0 = ys[0].cpu().numpy()  # forward spectrum of volume 0 (checked against the oracle in the CPU leg)
    # forward error of volume 0 against the complex128 GPU path of the same order
    with Plan(shape, P, order, "c128") as p128:
        ref = p128.exec(xs[0].to(torch.complex128))
        fwd_err = float((torch.linalg.vector_norm(ys[0].to(torch.complex128) - ref) / torch.linalg.vector_norm(ref)).item())
        del ref

    clocks = ClockSampler(local)
    plan.set_timing(True)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    nvtx.range_push("timed")
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    nvtx.range_pop()
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    pass_ms, n_timed = plan.pass_times()
    plan.set_timing(False)
    ms_max = max_over_ranks(ms, world)

    bytes_per_step = 2 * B * per_transform
    value = world * args.steps * bytes_per_step / (ms_max * 1e-3) / 1e9
    peak, peak_kind = peaks()
    launch_bytes = 2 * B * T * elem  # one pass: read and write the B arrays once
    avg_launch_ms = sum(pass_ms) / len(pass_ms)
    achieved = launch_bytes / (avg_launch_ms * 1e-3) / 1e9
    traffic = profile_traffic()
    # the bound the redistribution's access pattern puts on a pass: the same
    # loads and transposed stores without the butterflies
    pattern_ms = [plan.pattern_probe(s_, xs, ys, reps=5) for s_ in range(3)]
    pattern_gbs = launch_bytes / (sum(pattern_ms) / len(pattern_ms) * 1e-3) / 1e9

    # end to end: host (pinned) buffers through mdfft_exec_host, copies inside the timed region
    hx = xs.cpu().pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    hz = torch.empty_like(hx).pin_memory()
    din, dout = torch.empty_like(xs), torch.empty_like(xs)

    def e2e_step():
        plan.exec_host(hx, hy, din, dout, dir=-1)
        plan.exec_host(hy, hz, din, dout, dir=+1, normalize=True)

    e2e_step()
    torch.cuda.synchronize(dev)
    e_steps = max(1, min(args.steps, 5))
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    e2e_value = world * e_steps * bytes_per_step / (e_ms * 1e-3) / 1e9
    e2e_err = float((torch.linalg.vector_norm(hz[0] - hx[0]) / torch.linalg.vector_norm(hx[0])).item())
    host_bytes = 4 * B * T * elem  # per step: two inputs in, two results out
    link = host_link_gbs(hx, din, hy, dout)
    link["frac_of_concurrent"] = round(host_bytes / (e_ms / e_steps * 1e-3) / 1e9 / link["concurrent_gbs"], 3)

    extra = None
    if not args.no_extra and world == 1:  # single-GPU studies: not repeated on every rank of a replica run
        extra = extra_table(dev, xs, P, with_oracle=not args.no_cpu)

    if rank != 0:
        barrier(world)
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_baseline(shape, elem, fwd0)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "pct_hbm_peak": round(100.0 * value / world / peak, 1),
        "nominal_gflops": round(world * args.steps * 2 * B * 5.0 * T * math.log2(T) / (ms_max * 1e-3) / 1e9, 1),
        "forward_rel_l2_vs_c128": fwd_err,
        "config": {"workload": "3-D complex64 FFT 256x256x256, forward + normalised inverse, batch of "
                               f"{B} distinct volumes per step",
                   "P": P, "order": format_order(order, 3), "regimes": comm["regime"],
                   "comm_points_total": comm["total"], "l2": "inputs larger than L2 (8 x 128 MiB per step)",
                   "parallelism": f"replicas x{world}", "input": "U[-1,1) re/im, seeds 1303..1310",
                   "roundtrip_rel_l2": err, "autotune_ms_per_pass": {"default": [round(v, 5) for v in tune_before],
                                                                      "chosen": [round(v, 5) for v in tune_after]},
                   "passes": tuned},
        "roofline": {"kernel": "fft_pass_kernel<float,256>", "bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "algorithmic_bytes_per_launch": launch_bytes,
                     "avg_launch_ms": round(avg_launch_ms, 5), "launches_timed": n_timed * 3,
                     "pattern_bound_gbs": round(pattern_gbs, 1), "frac_of_pattern": round(achieved / pattern_gbs, 4),
                     "pass_ms": [round(v, 5) for v in pass_ms],
                     # ncu DRAM bytes of the M passes over the bytes of one full-array read + write
                     "full_array_passes_per_transform": None if traffic is None else
                     round(len(shape) * traffic / launch_bytes, 3)},
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 2), "unit": "GB/s", "h2d_bytes_per_step": 2 * B * T * elem,
                "d2h_bytes_per_step": 2 * B * T * elem, "steps": e_steps, "roundtrip_rel_l2": e2e_err,
                "api": "mdfft_exec_host", "host_link": link},
        "clocks": clk,
        "gpu_launches": args.steps * 2 * plan.launches(),
        "kernel_source_sha256": kernel_hash(),
    }
    if extra is not None:
        line["extra"] = extra
    print(json.dumps(line), flush=True)
    barrier(world)


def _orders3():
    out = []
    import itertools
    for p2 in itertools.permutations(range(3)):
        for p3 in itertools.permutations(range(3)):
            if len({2, p2[2], p3[2]}) == 3:
                out.append([[0, 1, 2], list(p2), list(p3)])
    return out


def extra_table(dev, x, P, with_oracle=True):
    """GB/s of every 3-D transpose order (complex64) and of the best order in
    complex128, a batch of 256^3 volumes (x: [B, 256, 256, 256]) per launch,
    forward transforms, 10 timed reps each."""
    import torch

    from paper_1302_6189_gb300 import Plan, format_order, mdfft_order_search

    B = x.shape[0]
    per_transform, T = algorithmic_bytes(SHAPE, 8)
    per_transform *= B
    res = {"orders_c64_gbs": {}, "note": f"forward only, 10 reps, the same {B} volumes per launch"}
    y = torch.empty_like(x)
    for o in _orders3():
        with Plan(SHAPE, P, o, "c64", batch=B) as pl:
            for _ in range(3):
                pl.exec(x, y)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(10):
                pl.exec(x, y)
            b.record()
            torch.cuda.synchronize(dev)
            res["orders_c64_gbs"][format_order(o, 3)] = round(10 * per_transform / (a.elapsed_time(b) * 1e-3) / 1e9, 1)
    x128 = x.to(torch.complex128)
    y128 = torch.empty_like(x128)
    best, _ = mdfft_order_search(SHAPE, P, 0)
    with Plan(SHAPE, P, best, "c128", batch=B) as pl:
        for _ in range(2):
            pl.exec(x128, y128)
        pl.set_timing(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(5):
            pl.exec(x128, y128)
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / 5
        pass_ms, _ = pl.pass_times()
    flops = 5.0 * T * 24 * B  # nominal 5 T log2 T per volume
    fp64_tflops = flops / (ms * 1e-3) / 1e12
    peak64 = fp64_peak(dev)
    # FP64 operations the pass kernel executes, counted by ncu (multiply-adds
    # x 2 + adds + multiplies per launch of one volume), if that count was
    # taken on the current kernel sources
    prof = profile_values(PROFILE_C128)
    counted, inst = prof.get("dp_flops_per_launch"), prof.get("dp_inst_per_launch")
    avg_pass_ms = sum(pass_ms) / len(pass_ms)
    counted_tflops = None if counted is None else B * counted / (avg_pass_ms * 1e-3) / 1e12
    # the FP64 pipe issues one instruction per slot whatever its kind: its
    # busy fraction is the instruction rate over the multiply-add rate
    issue_frac = None if inst is None else B * inst / (avg_pass_ms * 1e-3) / (peak64 * 1e12 / 2)
    res["c128"] = {"gbs": round(2 * per_transform / (ms * 1e-3) / 1e9, 1), "ms_per_transform": round(ms / B, 4),
                   "nominal_tflops_fp64": round(fp64_tflops, 3),
                   "pass_ms": [round(v, 4) for v in pass_ms],
                   # FP64-bound: the executed FP64 operations per second against the measured FP64 rate
                   "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": round(peak64, 3),
                                "peak_kind": "measured (mdfft_fp64_rate_probe: independent multiply-add chains)",
                                "achieved": None if counted_tflops is None else round(counted_tflops, 3),
                                "frac": None if counted_tflops is None else round(counted_tflops / peak64, 3),
                                "dp_flops_per_launch_per_volume": counted,
                                "fp64_instructions_per_launch_per_volume": inst,
                                "fp64_issue_frac": None if issue_frac is None else round(issue_frac, 3),
                                "achieved_nominal_5TlogT": round(fp64_tflops, 3),
                                "frac_nominal_work": round(fp64_tflops / peak64, 3)}}
    res["chunk_tile_order"] = chunk_order_study(dev, x, P)
    res["distributed_256cubed"] = dist_study(dev, x[0], P)
    res["small_32cubed_c128"] = small_study(dev)
    res["precision_512cubed"] = precision_study(dev, with_oracle)
    res["md_4d_5d"] = md_study(dev)
    res["decompositions"] = decomposition_study(dev)
    res["serving"] = serving_study(dev)
    return res


def chunk_order_study(dev, x, P, reps=10):
    """The bench workload's forward passes in the two tile orders: tiles along
    the output's fastest axis (default) and input-chunk order with one f_MD
    chunk per tile (16 x 1 lines: CTA t owns chunk t of the input layout),
    GB/s per pass, same kernel."""
    import torch

    from paper_1302_6189_gb300 import Plan, mdfft_order_search

    B = x.shape[0]
    _, T = algorithmic_bytes(SHAPE, 8)
    order, _ = mdfft_order_search(SHAPE, P, 0)
    y = torch.empty_like(x)
    out = {"note": f"{B} volumes per launch, forward, {reps} reps, default kernel for both"}
    with Plan(SHAPE, P, order, "c64", batch=B) as pl:
        want = pl.exec(x).clone()
        base = pl.tuning()
        for name, tuning in (("output_runs", base),
                             ("input_chunk_per_cta", [dict(t, tile_g=16, tile_h=1, tile_order=1) for t in base])):
            pl.set_tuning(tuning)
            for _ in range(2):
                pl.exec(x, y)
            pl.set_timing(True)
            for _ in range(reps):
                pl.exec(x, y)
            torch.cuda.synchronize(dev)
            pass_ms, _ = pl.pass_times()
            pl.set_timing(False)
            out[name] = {"gbs_per_pass": [round(2 * B * T * 8 / (m * 1e-3) / 1e9, 1) for m in pass_ms],
                         "ctas": [d["ctas"] for d in pl.describe()], "store_axis": [d["store_axis"] for d in pl.describe()],
                         "same_bits": bool(torch.equal(y, want))}
        pl.set_tuning(base)
    return out


def dist_study(dev, x0, P, reps=5):
    """The data plane of the distributed setting on one GPU: 256^3 complex64,
    P = 4096, the P processes on G = 2 and 8 virtual devices.  Per order (best
    and worst), the points that would cross devices per transform (the
    off-diagonal exchange counts, what a network would carry) beside the
    order's amount; and, for the best order, the device time of the library's
    line DFTs, pack and unpack per transform summed over the devices (the
    transport between them, a copy here, is not timed)."""
    import torch

    from paper_1302_6189_gb300 import (DistPlan, mdfft_dist_lines, mdfft_dist_pack, mdfft_dist_unpack,
                                       mdfft_order_search, format_order)

    _, T = algorithmic_bytes(SHAPE, 8)
    out = {"note": "cross-device points from mdfft_exchange_counts; times: CUDA events, library kernels only"}
    flat = x0.reshape(-1)
    for G in (2, 8):
        row = {}
        for want in (0, 1):
            order, amount = mdfft_order_search(SHAPE, P, want)
            parts = [DistPlan(SHAPE, P, G, g, order) for g in range(G)]
            try:
                cross = 0
                for s_ in range(3):
                    c = parts[0].counts(s_)
                    cross += sum(c[a][b] for a in range(G) for b in range(G) if a != b)
                entry = {"order": format_order(order, 3), "amount": amount, "cross_device_points": cross}
                if want == 0:
                    st = torch.cuda.current_stream(dev).cuda_stream
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                    t = {"lines": 0.0, "pack": 0.0, "unpack": 0.0}
                    for _ in range(reps):
                        local = []
                        for g in range(G):
                            a, b = parts[g].local_range(0)
                            local.append(flat[a:b].clone())
                        for s_ in range(3):
                            c = parts[0].counts(s_)
                            work = [torch.empty_like(v) for v in local]
                            sends = [torch.empty(sum(c[g]), dtype=x0.dtype, device=dev) for g in range(G)]
                            ev[0].record()
                            for g in range(G):
                                mdfft_dist_lines(parts[g].plan.handle, s_, G, g, local[g].data_ptr(), work[g].data_ptr(),
                                                 -1, 0, st)
                            ev[1].record()
                            for g in range(G):
                                mdfft_dist_pack(parts[g].plan.handle, s_, G, g, work[g].data_ptr(), sends[g].data_ptr(), st)
                            ev[2].record()
                            recvs = [torch.cat([sends[g][sum(c[g][:h]):sum(c[g][:h + 1])] for g in range(G)])
                                     for h in range(G)]
                            nxt = []
                            for h in range(G):
                                a, b = parts[h].local_range(s_ + 1)
                                nxt.append(torch.empty(b - a, dtype=x0.dtype, device=dev))
                            ev[3].record()
                            for h in range(G):
                                mdfft_dist_unpack(parts[h].plan.handle, s_, G, h, recvs[h].data_ptr(), nxt[h].data_ptr(), st)
                            end = torch.cuda.Event(enable_timing=True)
                            end.record()
                            torch.cuda.synchronize(dev)
                            t["lines"] += ev[0].elapsed_time(ev[1])
                            t["pack"] += ev[1].elapsed_time(ev[2])
                            t["unpack"] += ev[3].elapsed_time(end)
                            local = nxt
                    per = {k: v / reps for k, v in t.items()}
                    entry["ms_per_transform"] = {k: round(v, 4) for k, v in per.items()}
                    # each kernel reads and writes the whole array once per step (3 steps)
                    entry["gbs"] = {k: round(3 * 2 * T * 8 / (v * 1e-3) / 1e9, 1) for k, v in per.items()}
                row["best" if want == 0 else "worst"] = entry
            finally:
                for p_ in parts:
                    p_.close()
        row["worst_over_best_cross_device"] = round(row["worst"]["cross_device_points"] /
                                                    max(1, row["best"]["cross_device_points"]), 3)
        out[f"G={G}"] = row
    return out


def small_study(dev, reps=2000):
    """The 32^3 complex128 configuration (P = 4, order abc->cab->cba), forward
    + normalised inverse per call pair: microseconds per pair with the M pass
    launches issued one by one (mdfft_exec) and replayed from a captured
    CUDA graph (mdfft_exec_graph)."""
    import numpy as np
    import torch

    import synth_inputs as si
    from paper_1302_6189_gb300 import Plan

    shape = (32, 32, 32)
    x = torch.from_numpy(si.uniform_complex(shape, si.SEEDS["parity32"], np.complex128)).to(dev)
    y, z = torch.empty_like(x), torch.empty_like(x)
    out = {}
    with Plan(shape, 4, "abc->cab->cba", "c128") as pl:
        for graph in (False, True):
            for _ in range(20):
                pl.exec(x, y, graph=graph)
                pl.exec(y, z, dir=+1, normalize=True, graph=graph)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                pl.exec(x, y, graph=graph)
                pl.exec(y, z, dir=+1, normalize=True, graph=graph)
            b.record()
            torch.cuda.synchronize(dev)
            out["graph_us" if graph else "direct_us"] = round(a.elapsed_time(b) * 1e3 / reps, 2)
        err = float((torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x)).item())
    out["roundtrip_rel_l2"] = err
    out["note"] = "forward + normalised inverse, 6 pass launches or 2 graph launches per pair"
    return out


def md_study(dev, reps=10):
    """64^4 and 24^5 complex64 (U[-1,1) re/im), P in {64, 1024}, best and
    worst orders: forward GB/s of a batched plan (4 volumes per launch, about
    512 MiB per array) after autotuning, and the mean time of each pass."""
    import numpy as np
    import torch

    import synth_inputs as si
    from paper_1302_6189_gb300 import MDFFT_PLAN_TUNE_RADIX, Plan, format_order, mdfft_order_search

    out = {}
    for shape in ((64, 64, 64, 64), (24, 24, 24, 24, 24)):
        B = 4
        M, T = len(shape), int(np.prod(shape))
        x = torch.empty((B,) + shape, dtype=torch.complex64, device=dev)
        for i in range(B):
            x[i].copy_(torch.from_numpy(si.uniform_complex(shape, si.SEEDS["md_uniform"] + i, np.complex64)))
        y = torch.empty_like(x)
        for P in (64, 1024):
            for want in (0, 1):
                order, amount = mdfft_order_search(shape, P, want)
                with Plan(shape, P, order, "c64", MDFFT_PLAN_TUNE_RADIX, batch=B) as pl:
                    pl.autotune(x, y, reps=3)
                    # the bound the passes' access pattern sets: the same loads and
                    # transposed stores without the butterflies (the chosen tiles)
                    pattern_ms = [pl.pattern_probe(s_, x, y, reps=5) for s_ in range(M)]
                    # and the same movement with S - 1 tiles' loads in flight per CTA
                    # (persistent CTAs streaming tiles through a ring of slots)
                    movement_ms = [movement_bound_ms(pl, s_, x, y) for s_ in range(M)]
                    tuning = [dict(t, radix=d["radix"]) for t, d in zip(pl.tuning(), pl.describe())]
                    for _ in range(3):
                        pl.exec(x, y)
                    pl.set_timing(True)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    for _ in range(reps):
                        pl.exec(x, y)
                    b.record()
                    torch.cuda.synchronize(dev)
                    ms = a.elapsed_time(b) / reps
                    pass_ms, _ = pl.pass_times()
                name = f"{'x'.join(map(str, shape))} P={P} {'worst' if want else 'best'}"
                out[name] = {"order": format_order(order, M), "comm_points": amount,
                             "gbs": round(2 * M * T * 8 * B / (ms * 1e-3) / 1e9, 1),
                             "pass_ms": [round(v, 4) for v in pass_ms], "tuning": tuning,
                             "pattern_bound_gbs": [round(2 * B * T * 8 / (v * 1e-3) / 1e9, 1) for v in pattern_ms],
                             "movement_bound_gbs": [round(2 * B * T * 8 / (v * 1e-3) / 1e9, 1) if v else None
                                                    for v in movement_ms],
                             "probe_note": "the probes move a pass's data the way the default kernel (pattern) "
                                           "or the ring kernel (movement) does, with the pass's tiles where they "
                                           "fit that kernel's CTA, else its default tiling; they bound those "
                                           "kernels, not the one- or two-threads-per-line ones",
                             "roofline": pass_roofline(2 * B * T * 8, pass_ms, MD_PROFILES.get(name))}
    return out


# ncu summaries of the 4-D / 5-D configurations' launches (4 volumes, autotuned plan)
MD_PROFILES = {"64x64x64x64 P=64 best": os.path.join(ROOT, "profiles", "fft_pass_64x4_c64.md"),
               "24x24x24x24x24 P=64 best": os.path.join(ROOT, "profiles", "fft_pass_24x5_c64.md")}


def movement_bound_ms(pl, s, x, y):
    """The fastest ring-structured data movement of pass s (mdfft_movement_probe:
    2 slots at 3 CTAs per SM, 3 slots at 2), or None where no ring probe is built."""
    from paper_1302_6189_gb300 import MdfftError
    best = None
    for slots, per_sm in ((2, 3), (3, 2)):
        try:
            ms = pl.movement_probe(s, x, y, slots, per_sm, reps=5)
        except MdfftError:
            return None
        best = ms if best is None else min(best, ms)
    return best


def pass_roofline(launch_bytes, pass_ms, profile=None, volumes=1):
    """HBM roofline of every pass of a configuration: algorithmic bytes of a
    launch (read + write of the array) over its CUDA-event time, the fraction
    of the measured copy peak, and, when a committed ncu summary of the same
    kernels holds the DRAM traffic of each pass (`volumes` per launch of the
    summary), that traffic per launch over the algorithmic bytes."""
    peak, kind = peaks()
    ach = [launch_bytes / (t * 1e-3) / 1e9 for t in pass_ms]
    r = {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_kind": kind,
         "algorithmic_bytes_per_launch": launch_bytes,
         "achieved_per_pass": [round(a, 1) for a in ach], "frac_per_pass": [round(a / peak, 4) for a in ach],
         "frac": round(launch_bytes * len(pass_ms) / (sum(pass_ms) * 1e-3) / 1e9 / peak, 4)}
    if profile:
        vals = profile_values(profile)
        tr = [vals.get(f"traffic_bytes_pass_{s_}") for s_ in range(len(pass_ms))]
        if all(t is not None for t in tr):
            r["traffic_per_pass"] = [t * volumes for t in tr]
            r["traffic_over_algorithmic"] = [round(t * volumes / launch_bytes, 3) for t in tr]
    return r


def decomposition_study(dev):
    """Amounts of communication (points) counted on the device by the pass
    kernels for the row-wise method (best order) and the comparison methods
    of Sec. 4 run through the same passes, beside the closed forms: 64^3 as
    in Fig. 7, 16^4 and 16^5 as in Fig. 8."""
    import torch

    from paper_1302_6189_gb300 import DECOMPOSITIONS, MdfftError, Plan

    cases = {(64, 64, 64): (4, 16, 64, 256, 1024, 4096, 8192, 32768, 262144),
             (16, 16, 16, 16): (16, 256, 4096, 65536), (16,) * 5: (32, 1024, 4096, 32768)}
    out = {}
    for shape, Ps in cases.items():
        M = len(shape)
        x = torch.zeros(shape, dtype=torch.complex64, device=dev)
        rows = []
        for P in Ps:
            row = {"P": P}
            for kind, flag in DECOMPOSITIONS.items():
                try:
                    with Plan(shape, P, None, "c64", flag) as pl:
                        _, c = pl.exec_counted(x)
                        c = c.cpu().tolist()
                        cv = pl.comm_volume()
                except MdfftError:
                    row[kind] = None  # the method cannot use P processes on this grid
                    continue
                row[kind] = int(sum(c[: M - 1]) + sum(c[M:]))
                row["A_1D"] = cv["amount_slab"]
                row["A_2D"] = cv["amount_pencil"] if M == 3 else None
                row["A_MD"] = cv["amount_volumetric"]
            for kind in ("slab", "pencil", "volumetric"):
                if row.get(kind):
                    row[f"{kind}_over_rowwise"] = round(row[kind] / row["rowwise"], 3)
            rows.append(row)
        out["x".join(map(str, shape))] = rows
    return out


PRECISION_PROFILES = {"c64": os.path.join(ROOT, "profiles", "fft_pass_512cubed_c64.md"),
                      "c64_tc_fp16": os.path.join(ROOT, "profiles", "fft_pass_512cubed_tc_fp16.md")}
PRECISION_BOUNDS = {"c64": 1e-5, "c64_tc_fp16": 1e-5, "c64_tc_bf16": 1e-4, "c128": 1e-12}


def precision_study(dev, with_oracle=True):
    """512^3, N(0,1) re/im (seed 1306), P = 4096, the planner's best order:
    forward transform of the FP32 SIMT path, the tensor-core FP16 / BF16
    hi-lo paths and the FP64 path, each plan autotuned (kernel variant and
    tiles; results bit-identical to the default launch).  Throughput (bytes of the M passes) and,
    with_oracle, every output element against the FP64 oracle's spectrum of
    the same input: rel-L2 and the largest element error over the RMS, beside
    the stated bound."""
    import numpy as np
    import torch

    import synth_inputs as si
    from paper_1302_6189_gb300 import Plan, format_order, mdfft_order_search

    shape = (512, 512, 512)
    per_transform, T = algorithmic_bytes(shape, 8)
    xh = si.gaussian_complex(shape, si.SEEDS["precision512"], np.complex64)
    x = torch.from_numpy(xh).to(dev)
    order, _ = mdfft_order_search(shape, 4096, 0)
    out = {"order": format_order(order, 3), "reference": "FP64 oracle (CPU), every element" if with_oracle
           else "none (run without the CPU oracle)", "dtypes": {}}
    ref = None
    if with_oracle:
        ref, secs = oracle_spectrum(xh, len(os.sched_getaffinity(0)))
        out["oracle_seconds"] = round(secs, 3)
    for dt in ("c64", "c64_tc_fp16", "c64_tc_bf16", "c128"):
        xin = x.to(torch.complex128) if dt == "c128" else x
        y = torch.empty_like(xin)
        with Plan(shape, 4096, order, dt) as pl:
            pl.autotune(xin, y, reps=3)
            pattern_ms = [pl.pattern_probe(s_, xin, y, reps=3) for s_ in range(3)] if dt == "c64" else None
            tuning = pl.tuning()
            for _ in range(2):
                pl.exec(xin, y)
            pl.set_timing(True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(5):
                pl.exec(xin, y)
            b.record()
            torch.cuda.synchronize(dev)
            pl.check()
            ms = a.elapsed_time(b) / 5
            pass_ms, _ = pl.pass_times()
        elem = 16 if dt == "c128" else 8
        row = {"gbs": round(per_transform * elem / 8 / (ms * 1e-3) / 1e9, 1), "ms": round(ms, 4),
               "pass_ms": [round(v, 4) for v in pass_ms], "bound_rel_l2": PRECISION_BOUNDS[dt],
               "tuning": [t["variant"] for t in tuning]}
        if dt != "c128":  # the complex128 path is FP64-bound (see extra.c128)
            row["roofline"] = pass_roofline(2 * T * elem, pass_ms, PRECISION_PROFILES.get(dt))
        if pattern_ms:
            row["pattern_bound_gbs"] = [round(2 * T * 8 / (v * 1e-3) / 1e9, 1) for v in pattern_ms]
        if ref is not None:
            row.update(errors_vs(y.cpu().numpy(), ref))
            row["within_bound"] = row["rel_l2"] <= PRECISION_BOUNDS[dt]
        out["dtypes"][dt] = row
        del xin, y
    return out


def profile_case(args):
    """Two forward transforms of a batch of volumes with the planner's best
    order (M + M pass launches: a warm-up, then the profiled ones, inside the
    NVTX range "profiled"); with --profile-tune the plan is autotuned first."""
    import numpy as np
    import torch

    import synth_inputs as si
    from paper_1302_6189_gb300 import MDFFT_PLAN_TUNE_RADIX, Plan

    torch.cuda.set_device(0)
    shape = tuple(int(v) for v in args.profile_shape.split(","))
    npdt = np.complex128 if args.profile_dtype == "c128" else np.complex64
    B = args.profile_batch
    x = torch.empty((B,) + shape if B > 1 else shape, dtype=torch.from_numpy(np.zeros(1, npdt)).dtype,
                    device="cuda")
    for i in range(B):
        (x[i] if B > 1 else x).copy_(torch.from_numpy(si.uniform_complex(shape, si.SEEDS["cube256"] + i, npdt)))
    flags = MDFFT_PLAN_TUNE_RADIX if args.profile_tune and args.profile_dtype == "c64" else 0
    with Plan(shape, args.P, None, args.profile_dtype, flags, batch=B) as plan:
        y = torch.empty_like(x)
        if args.profile_tune:
            plan.autotune(x, y, reps=3)
        if args.profile_tuning:
            t = json.loads(args.profile_tuning)
            plan.set_tuning([dict(e) for e in t] if isinstance(t, list) else [dict(t) for _ in shape])
        plan.exec(x, y)  # warm-up: launches 1..M (after any autotuning)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        plan.exec(x, y)  # profiled: the next M launches
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        plan.check()
        print(json.dumps({"profile_case": f"{B} x {'x'.join(map(str, shape))} {args.profile_dtype} forward",
                          "order": plan.order_str(), "tuning": plan.tuning(), "passes": plan.describe()}))


def serving_study(dev, n=2000, budget=40e9):
    """2000 Poisson arrivals: 80 % 3-D requests with axes from {48..192}, 20 %
    32^4, complex64 forward, 40 GB HBM admission budget.  The batched server
    (one graph launch of one persistent kernel per step) against plain
    per-request mdfft_exec launches of the same kernels, at arrival rates
    0.5, 0.8 and 1.0 times the server's saturated throughput X.  Latency is
    arrival (host clock) to completion (CUDA event), both from one zero."""
    import numpy as np
    import torch

    import synth_inputs as si
    from paper_1302_6189_gb300 import Plan, Server

    shapes = si.serving_requests(n, si.SEEDS["serving"])
    distinct = sorted(set(shapes))
    gen = torch.Generator(device=dev)
    inputs = {}
    for k, shp in enumerate(distinct):
        gen.manual_seed(si.SEEDS["serving"] * 1000 + k)
        re = torch.rand(shp, generator=gen, device=dev) * 2 - 1
        im = torch.rand(shp, generator=gen, device=dev) * 2 - 1
        inputs[shp] = torch.complex(re, im)
    outs = [torch.empty(shp, dtype=torch.complex64, device=dev) for shp in shapes]
    bytes_per = [2 * len(shp) * int(np.prod(shp)) * 8 for shp in shapes]
    stream = torch.cuda.current_stream(dev)

    def run_server(srv, arrivals):
        srv.reset_clock()
        t0 = time.perf_counter()
        ids, i = [], 0
        while i < n:
            now = time.perf_counter() - t0
            while i < n and arrivals[i] <= now:
                ids.append(srv.submit(inputs[shapes[i]], outs[i]))
                i += 1
            srv.run(4)  # up to one step per pass of a 4-D request
        srv.drain()
        done = []
        for rid in ids:
            ok, ms = srv.poll(rid)
            done.append(ms / 1e3)
            srv.release(rid)
        return np.array(done)

    plans = {shp: Plan(shp, 64, None, "c64") for shp in distinct}

    def run_plain(arrivals):
        torch.cuda.synchronize(dev)
        t0ev = torch.cuda.Event(enable_timing=True)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        t0ev.record(stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        i = 0
        while i < n:
            now = time.perf_counter() - t0
            while i < n and arrivals[i] <= now:
                plans[shapes[i]].exec(inputs[shapes[i]], outs[i])
                evs[i].record(stream)
                i += 1
        torch.cuda.synchronize(dev)
        return np.array([t0ev.elapsed_time(e) / 1e3 for e in evs])

    def summary(arrivals, done):
        lat = (done - arrivals) * 1e3
        span = float(done.max() - arrivals.min())
        return {"fft_per_s": round(n / span, 1), "gbs": round(sum(bytes_per) / span / 1e9, 1),
                "p50_ms": round(float(np.percentile(lat, 50)), 4), "p99_ms": round(float(np.percentile(lat, 99)), 4)}

    zero = np.zeros(n)
    with Server(int(budget), max_inflight=512, P=64) as srv:
        for _ in range(2):  # plans, graphs and clocks warm
            run_server(srv, zero)
        # autotune the persistent grid (whole multiples of the SM count) and the
        # number of steps in flight, on the saturated load (the tiles dealt to a
        # CTA at a time stay at the default maximum of 4: larger chunks raise the
        # saturated rate a little but double the latency at 0.8 X)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        best = None
        for per_sm in (2, 4):
            for depth in (1, 2, 4):
                srv.set_grid(sms * per_sm)
                srv.set_depth(depth)
                t = float(run_server(srv, zero).max())
                if best is None or t < best[0]:
                    best = (t, per_sm, depth, 4)
        srv.set_grid(sms * best[1])
        srv.set_depth(best[2])
        sat = run_server(srv, zero)
        X = n / float(sat.max())
        run_plain(zero)
        plain_sat = run_plain(zero)
        out = {"requests": n, "budget_gb": budget / 1e9, "grid_ctas_per_sm": best[1], "depth": best[2],
               "chunk_tiles": best[3], "direct_max_requests": 4,
               "saturated": {"batched": summary(zero, sat), "plain": summary(zero, plain_sat)}, "poisson": {}}
        for frac in (0.5, 0.8, 1.0):
            arrivals = si.poisson_arrivals(n, frac * X, si.SEEDS["serving"])
            arrivals = arrivals - arrivals[0]
            d0 = srv.stats()["direct_requests"]
            b = summary(arrivals, run_server(srv, arrivals))
            b["direct_requests"] = srv.stats()["direct_requests"] - d0
            p = summary(arrivals, run_plain(arrivals))
            out["poisson"][f"{frac:.1f}X"] = {"rate_per_s": round(frac * X, 1), "batched": b, "plain": p}
        out["server_stats"] = srv.stats()
    for pl in plans.values():
        pl.close()
    out["results"] = "identical kernels and tiles in both arms (tests: bit-equal to mdfft_exec)"
    return out


def main():
    args = parse_args()
    if args.profile_case:
        profile_case(args)
        return
    if args.serving_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"serving": serving_study(torch.device("cuda", 0), n=args.serving_only,
                                                   budget=args.serving_budget_gb * 1e9)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
