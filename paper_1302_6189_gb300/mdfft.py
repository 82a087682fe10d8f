"""Thin ctypes binding of libmdfft (include/mdfft.h).

Argument marshalling only: every function here converts Python arguments to
the C types of the function of the same name and raises ``MdfftError`` on a
non-zero status.  All computation happens in the library (host planner and
sm_103a kernels).  ``Plan`` is a convenience wrapper that passes torch CUDA
tensors' data pointers and the current CUDA stream.

The library must have been built (``__graft_entry__.build()``); importing this
module without it raises ImportError -- there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libmdfft.so")
AXES = "abcdefgh"
MAX_DIMS = 8

MDFFT_OK, MDFFT_E_ARG, MDFFT_E_ORDER, MDFFT_E_RANGE = 0, -1, -2, -3
MDFFT_E_NOMEM, MDFFT_E_CUDA, MDFFT_E_TIMEOUT, MDFFT_E_UNSUPPORTED = -4, -5, -6, -7
MDFFT_C64, MDFFT_C128, MDFFT_C64_TC_FP16, MDFFT_C64_TC_BF16 = 0, 1, 2, 3
MDFFT_PLAN_HOST_ONLY, MDFFT_PLAN_INPLACE, MDFFT_PLAN_PERSISTENT = 0x1, 0x2, 0x4
MDFFT_PLAN_DECOMP_SLAB, MDFFT_PLAN_DECOMP_PENCIL, MDFFT_PLAN_DECOMP_VOLUMETRIC = 0x10, 0x20, 0x40
MDFFT_PLAN_OUT_NATURAL, MDFFT_PLAN_OUT_LAST_LAYOUT = 0x0, 0x80
MDFFT_PLAN_TUNE_RADIX = 0x100
DECOMPOSITIONS = {"rowwise": 0, "slab": MDFFT_PLAN_DECOMP_SLAB, "pencil": MDFFT_PLAN_DECOMP_PENCIL,
                  "volumetric": MDFFT_PLAN_DECOMP_VOLUMETRIC}
DTYPES = {"c64": MDFFT_C64, "c128": MDFFT_C128, "c64_tc_fp16": MDFFT_C64_TC_FP16,
          "c64_tc_bf16": MDFFT_C64_TC_BF16}
STATUS_NAMES = {0: "OK", -1: "E_ARG", -2: "E_ORDER", -3: "E_RANGE", -4: "E_NOMEM", -5: "E_CUDA",
                -6: "E_TIMEOUT", -7: "E_UNSUPPORTED"}

i64, c_int, c_void_p, c_size_t = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
P_ = ctypes.POINTER


class MdfftComm(ctypes.Structure):
    _fields_ = [("per_transition", i64 * MAX_DIMS), ("total", i64), ("final_to_natural", i64),
                ("split_line", i64 * MAX_DIMS), ("paper_total", i64), ("regime", c_int * MAX_DIMS),
                ("amount_slab", ctypes.c_double), ("amount_pencil", ctypes.c_double),
                ("amount_volumetric", ctypes.c_double)]


class MdfftPassInfo(ctypes.Structure):
    _fields_ = [("line_length", i64), ("tile_g", c_int), ("tile_h", c_int), ("threads", c_int),
                ("smem_bytes", c_int), ("ctas", i64), ("fft_axis", c_int), ("store_axis", c_int),
                ("grid", i64), ("persistent", c_int), ("stages", c_int), ("radix", c_int * 12),
                ("tile_order", c_int)]


class MdfftServerStats(ctypes.Structure):
    _fields_ = [("submitted", i64), ("admitted", i64), ("completed", i64), ("steps", i64),
                ("graph_launches", i64), ("kernel_launches", i64), ("inflight", i64), ("queued", i64),
                ("bytes_in_use", c_size_t), ("budget_bytes", c_size_t), ("grid_ctas", c_int),
                ("cancelled", i64), ("direct_requests", i64)]


SIGNATURES = {
    "mdfft_plan": (c_int, [P_(c_void_p), c_int, P_(i64), i64, P_(c_int), c_int, ctypes.c_uint]),
    "mdfft_plan_batched": (c_int, [P_(c_void_p), c_int, P_(i64), i64, P_(c_int), c_int, ctypes.c_uint, i64]),
    "mdfft_exec": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "mdfft_exec_graph": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "mdfft_selftest_wait": (c_int, [c_int, i64, P_(i64)]),
    "mdfft_plan_tuning": (c_int, [c_void_p, P_(ctypes.c_int32), c_int]),
    "mdfft_plan_set_tuning": (c_int, [c_void_p, P_(ctypes.c_int32), c_int]),
    "mdfft_exec_counted": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "mdfft_comm_volume": (c_int, [c_void_p, P_(MdfftComm)]),
    "mdfft_chunk": (c_int, [c_void_p, c_int, i64, P_(i64), P_(i64), P_(i64), P_(i64)]),
    "mdfft_plan_order": (c_int, [c_void_p, P_(c_int)]),
    "mdfft_exchange_counts": (c_int, [c_void_p, c_int, c_int, P_(i64)]),
    "mdfft_block_grid": (c_int, [c_void_p, c_int, P_(i64)]),
    "mdfft_order_search": (c_int, [c_int, P_(i64), i64, c_int, P_(c_int), P_(i64)]),
    "mdfft_order_heuristic": (c_int, [c_int, P_(i64), i64, P_(c_int), P_(i64)]),
    "mdfft_pass_timing": (c_int, [c_void_p, c_int]),
    "mdfft_pass_times": (c_int, [c_void_p, P_(ctypes.c_float), c_int, P_(c_int)]),
    "mdfft_exec_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "mdfft_pass_describe": (c_int, [c_void_p, c_int, P_(MdfftPassInfo)]),
    "mdfft_plan_autotune": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, P_(ctypes.c_float),
                                    P_(ctypes.c_float)]),
    "mdfft_workspace_size": (c_int, [c_void_p, P_(c_size_t)]),
    "mdfft_plan_check": (c_int, [c_void_p]),
    "mdfft_pattern_probe": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p, P_(ctypes.c_float)]),
    "mdfft_movement_probe": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_int, c_void_p,
                                     P_(ctypes.c_float)]),
    "mdfft_launches_per_exec": (c_int, [c_void_p, P_(c_int)]),
    "mdfft_fp64_rate_probe": (c_int, [c_void_p, c_int, i64, c_void_p, P_(ctypes.c_double)]),
    "mdfft_dist_local_range": (c_int, [c_void_p, c_int, c_int, c_int, P_(i64), P_(i64)]),
    "mdfft_dist_lines": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "mdfft_dist_pack": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "mdfft_dist_unpack": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "mdfft_supported_length": (c_int, [i64, c_int]),
    "mdfft_destroy": (c_int, [c_void_p]),
    "mdfft_exec_noalloc": (c_int, [c_int, P_(i64), P_(c_int), c_int, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "mdfft_last_error": (ctypes.c_char_p, []),
    "mdfft_server_create": (c_int, [P_(c_void_p), c_size_t, c_int, i64, c_void_p]),
    "mdfft_server_submit": (c_int, [c_void_p, c_int, P_(i64), c_void_p, c_void_p, c_int, c_int, P_(i64)]),
    "mdfft_server_step": (c_int, [c_void_p, P_(c_int)]),
    "mdfft_server_run": (c_int, [c_void_p, c_int, P_(c_int)]),
    "mdfft_server_poll": (c_int, [c_void_p, i64, P_(c_int), P_(ctypes.c_double)]),
    "mdfft_server_release": (c_int, [c_void_p, i64]),
    "mdfft_server_cancel": (c_int, [c_void_p, i64]),
    "mdfft_server_drain": (c_int, [c_void_p]),
    "mdfft_server_reset_clock": (c_int, [c_void_p]),
    "mdfft_server_set_grid": (c_int, [c_void_p, c_int]),
    "mdfft_server_set_depth": (c_int, [c_void_p, c_int]),
    "mdfft_server_set_chunk": (c_int, [c_void_p, c_int]),
    "mdfft_server_set_direct": (c_int, [c_void_p, c_int]),
    "mdfft_server_set_line_kernel": (c_int, [c_void_p, c_int]),
    "mdfft_server_get_stats": (c_int, [c_void_p, P_(MdfftServerStats)]),
    "mdfft_server_destroy": (c_int, [c_void_p]),
}


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is not built; run __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(_LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    return lib


_lib = _load()
LIB_PATH = _LIB_PATH


class MdfftError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.mdfft_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def _check(st, where):
    if st != MDFFT_OK:
        raise MdfftError(st, where)


def parse_order(order, M):
    """'abc->cab->cba' or [[0,1,2],...] -> flat list of M*M axis ids."""
    if isinstance(order, str):
        layouts = [p.strip() for p in order.replace("→", "->").split("->")]
        flat = [AXES.index(ch) for L in layouts for ch in L]
    else:
        flat = [int(a) for L in order for a in L]
    if len(flat) != M * M:
        raise ValueError(f"order must have {M} layouts of {M} axes")
    return flat


def format_order(order, M):
    flat = parse_order(order, M)
    return "->".join("".join(AXES[a] for a in flat[s * M:(s + 1) * M]) for s in range(M))


def _dims(N):
    return (i64 * len(N))(*[int(n) for n in N]), len(N)


# ------------------------------------------------------------------- C entry points

def mdfft_plan(N, P, order=None, dtype=MDFFT_C64, flags=0):
    dims, M = _dims(N)
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    oarr = None if order is None else (c_int * (M * M))(*parse_order(order, M))
    h = c_void_p()
    _check(_lib.mdfft_plan(ctypes.byref(h), M, dims, int(P), oarr, dt, int(flags)), "mdfft_plan")
    return h


def mdfft_plan_batched(N, P, order=None, dtype=MDFFT_C64, flags=0, batch=1):
    dims, M = _dims(N)
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    oarr = None if order is None else (c_int * (M * M))(*parse_order(order, M))
    h = c_void_p()
    _check(_lib.mdfft_plan_batched(ctypes.byref(h), M, dims, int(P), oarr, dt, int(flags), int(batch)),
           "mdfft_plan_batched")
    return h


def mdfft_exec(plan, in_ptr, out_ptr, dir=-1, normalize=0, stream=0):
    _check(_lib.mdfft_exec(plan, c_void_p(in_ptr), c_void_p(out_ptr), int(dir), int(normalize),
                           c_void_p(stream)), "mdfft_exec")


def mdfft_exec_graph(plan, in_ptr, out_ptr, dir=-1, normalize=0, stream=0):
    _check(_lib.mdfft_exec_graph(plan, c_void_p(in_ptr), c_void_p(out_ptr), int(dir), int(normalize),
                                 c_void_p(stream)), "mdfft_exec_graph")


def mdfft_selftest_wait(arrive, limit_us):
    """Returns (status, microseconds waited); status MDFFT_E_TIMEOUT when the wait gave up."""
    waited = i64()
    st = _lib.mdfft_selftest_wait(int(arrive), int(limit_us), ctypes.byref(waited))
    return st, waited.value


TUNING_VARIANTS = ("default", "thr256", "thr512", "pipe1", "pipe2", "tc128", "thr192", "thr384", "radix_alt", "occ6", "tcg", "tcg_direct", "pf2", "pf4",
                   "pf2_radix_alt", "pf4_radix_alt", "shfl256", "ring2x3", "ring3x2", "ring2x4", "ring2x2",
                   "ring2x3_radix_alt", "ring3x2_radix_alt", "line", "line2w", "line_radix_alt", "line2t", "line2t_radix_alt")


def mdfft_plan_tuning(plan, M):
    """[{"variant": ..., "tile_g": ..., "tile_h": ..., "tile_order": ...} per pass] (JSON-friendly)."""
    arr = (ctypes.c_int32 * (4 * M))()
    _check(_lib.mdfft_plan_tuning(plan, arr, 4 * M), "mdfft_plan_tuning")
    return [{"variant": TUNING_VARIANTS[arr[4 * s]], "tile_g": arr[4 * s + 1], "tile_h": arr[4 * s + 2],
             "tile_order": arr[4 * s + 3]} for s in range(M)]


def mdfft_plan_set_tuning(plan, tuning):
    vals = []
    for t in tuning:
        vals += [TUNING_VARIANTS.index(t["variant"]), int(t["tile_g"]), int(t["tile_h"]), int(t.get("tile_order", 0))]
    arr = (ctypes.c_int32 * len(vals))(*vals)
    _check(_lib.mdfft_plan_set_tuning(plan, arr, len(vals)), "mdfft_plan_set_tuning")


def mdfft_exec_counted(plan, in_ptr, out_ptr, dir, normalize, stream, counts_ptr):
    _check(_lib.mdfft_exec_counted(plan, c_void_p(in_ptr), c_void_p(out_ptr), int(dir), int(normalize),
                                   c_void_p(stream), c_void_p(counts_ptr)), "mdfft_exec_counted")


def mdfft_comm_volume(plan, M):
    c = MdfftComm()
    _check(_lib.mdfft_comm_volume(plan, ctypes.byref(c)), "mdfft_comm_volume")
    return {"per_transition": list(c.per_transition[: M - 1]), "total": c.total,
            "final_to_natural": c.final_to_natural, "split_line": list(c.split_line[:M]),
            "paper_total": c.paper_total, "regime": list(c.regime[:M]),
            "amount_slab": c.amount_slab, "amount_pencil": c.amount_pencil,
            "amount_volumetric": c.amount_volumetric}


def mdfft_chunk(plan, step, pid, M):
    xs, xe = i64(), i64()
    cs, ce = (i64 * M)(), (i64 * M)()
    _check(_lib.mdfft_chunk(plan, int(step), int(pid), ctypes.byref(xs), ctypes.byref(xe), cs, ce),
           "mdfft_chunk")
    return xs.value, xe.value, list(cs), list(ce)


def mdfft_exchange_counts(plan, step, G):
    arr = (i64 * (G * G))()
    _check(_lib.mdfft_exchange_counts(plan, int(step), int(G), arr), "mdfft_exchange_counts")
    return [list(arr[g * G:(g + 1) * G]) for g in range(G)]


def mdfft_block_grid(plan, step, M):
    arr = (i64 * M)()
    _check(_lib.mdfft_block_grid(plan, int(step), arr), "mdfft_block_grid")
    return list(arr)


def mdfft_plan_order(plan, M):
    arr = (c_int * (M * M))()
    _check(_lib.mdfft_plan_order(plan, arr), "mdfft_plan_order")
    return [list(arr[s * M:(s + 1) * M]) for s in range(M)]


def mdfft_order_search(N, P, want_worst=0):
    dims, M = _dims(N)
    arr = (c_int * (M * M))()
    tot = i64()
    _check(_lib.mdfft_order_search(M, dims, int(P), int(want_worst), arr, ctypes.byref(tot)),
           "mdfft_order_search")
    return [list(arr[s * M:(s + 1) * M]) for s in range(M)], tot.value


def mdfft_order_heuristic(N, P):
    dims, M = _dims(N)
    arr = (c_int * (M * M))()
    tot = i64()
    _check(_lib.mdfft_order_heuristic(M, dims, int(P), arr, ctypes.byref(tot)), "mdfft_order_heuristic")
    return [list(arr[s * M:(s + 1) * M]) for s in range(M)], tot.value


def mdfft_pass_timing(plan, enable):
    _check(_lib.mdfft_pass_timing(plan, int(enable)), "mdfft_pass_timing")


def mdfft_pass_times(plan, M):
    """(mean ms per pass, number of executions averaged)."""
    arr = (ctypes.c_float * M)()
    n = c_int()
    _check(_lib.mdfft_pass_times(plan, arr, M, ctypes.byref(n)), "mdfft_pass_times")
    return list(arr), n.value


def mdfft_exec_host(plan, in_host_ptr, out_host_ptr, dev_in_ptr, dev_out_ptr, dir=-1, normalize=0, stream=0):
    _check(_lib.mdfft_exec_host(plan, c_void_p(in_host_ptr), c_void_p(out_host_ptr), c_void_p(dev_in_ptr),
                                c_void_p(dev_out_ptr), int(dir), int(normalize), c_void_p(stream)),
           "mdfft_exec_host")


def mdfft_pass_describe(plan, s):
    info = MdfftPassInfo()
    _check(_lib.mdfft_pass_describe(plan, int(s), ctypes.byref(info)), "mdfft_pass_describe")
    d = {f: getattr(info, f) for f, _ in MdfftPassInfo._fields_ if f != "radix"}
    d["radix"] = [info.radix[i] for i in range(info.stages)]
    return d


def mdfft_plan_autotune(plan, in_ptr, out_ptr, reps, stream, M):
    before, after = (ctypes.c_float * M)(), (ctypes.c_float * M)()
    _check(_lib.mdfft_plan_autotune(plan, c_void_p(in_ptr), c_void_p(out_ptr), int(reps), c_void_p(stream),
                                    before, after), "mdfft_plan_autotune")
    return list(before), list(after)


def mdfft_movement_probe(plan, s, slots, per_sm, in_ptr, out_ptr, reps, stream):
    ms = ctypes.c_float()
    _check(_lib.mdfft_movement_probe(plan, int(s), int(slots), int(per_sm), c_void_p(in_ptr), c_void_p(out_ptr),
                                     int(reps), c_void_p(stream), ctypes.byref(ms)), "mdfft_movement_probe")
    return ms.value


def mdfft_pattern_probe(plan, s, in_ptr, out_ptr, reps, stream):
    ms = ctypes.c_float()
    _check(_lib.mdfft_pattern_probe(plan, int(s), c_void_p(in_ptr), c_void_p(out_ptr), int(reps), c_void_p(stream),
                                    ctypes.byref(ms)), "mdfft_pattern_probe")
    return ms.value


def mdfft_fp64_rate_probe(out_ptr, ctas, iters, stream):
    """Measured FP64 multiply-add rate of the device, TFLOP/s (out_ptr: ctas x 256 doubles)."""
    tf = ctypes.c_double()
    _check(_lib.mdfft_fp64_rate_probe(c_void_p(out_ptr), int(ctas), int(iters), c_void_p(stream),
                                      ctypes.byref(tf)), "mdfft_fp64_rate_probe")
    return tf.value


def mdfft_dist_local_range(plan, step, G, g):
    x0, x1 = i64(), i64()
    _check(_lib.mdfft_dist_local_range(plan, int(step), int(G), int(g), ctypes.byref(x0), ctypes.byref(x1)),
           "mdfft_dist_local_range")
    return x0.value, x1.value


def mdfft_dist_lines(plan, step, G, g, in_ptr, out_ptr, dir, normalize, stream):
    _check(_lib.mdfft_dist_lines(plan, int(step), int(G), int(g), c_void_p(in_ptr), c_void_p(out_ptr), int(dir),
                                 int(normalize), c_void_p(stream)), "mdfft_dist_lines")


def mdfft_dist_pack(plan, step, G, g, local_ptr, send_ptr, stream):
    _check(_lib.mdfft_dist_pack(plan, int(step), int(G), int(g), c_void_p(local_ptr), c_void_p(send_ptr),
                                c_void_p(stream)), "mdfft_dist_pack")


def mdfft_dist_unpack(plan, step, G, h, recv_ptr, local_ptr, stream):
    _check(_lib.mdfft_dist_unpack(plan, int(step), int(G), int(h), c_void_p(recv_ptr), c_void_p(local_ptr),
                                  c_void_p(stream)), "mdfft_dist_unpack")


def mdfft_plan_check(plan):
    _check(_lib.mdfft_plan_check(plan), "mdfft_plan_check")


def mdfft_workspace_size(plan):
    n = c_size_t()
    _check(_lib.mdfft_workspace_size(plan, ctypes.byref(n)), "mdfft_workspace_size")
    return n.value


def mdfft_launches_per_exec(plan):
    n = c_int()
    _check(_lib.mdfft_launches_per_exec(plan, ctypes.byref(n)), "mdfft_launches_per_exec")
    return n.value


def mdfft_supported_length(n, dtype=MDFFT_C64):
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return bool(_lib.mdfft_supported_length(int(n), dt))


def mdfft_destroy(plan):
    _check(_lib.mdfft_destroy(plan), "mdfft_destroy")


def mdfft_exec_noalloc(N, order, dtype, in_ptr, out_ptr, dir=-1, normalize=0, stream=0):
    """The transform without any device allocation (scratch is a static device array)."""
    dims, M = _dims(N)
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    oarr = None if order is None else (c_int * (M * M))(*parse_order(order, M))
    _check(_lib.mdfft_exec_noalloc(M, dims, oarr, dt, c_void_p(in_ptr), c_void_p(out_ptr), int(dir),
                                   int(normalize), c_void_p(stream)), "mdfft_exec_noalloc")


def mdfft_server_create(budget_bytes, max_inflight, P=64, stream=0):
    h = c_void_p()
    _check(_lib.mdfft_server_create(ctypes.byref(h), int(budget_bytes), int(max_inflight), int(P),
                                    c_void_p(stream)), "mdfft_server_create")
    return h


def mdfft_server_submit(server, N, in_ptr, out_ptr, dir=-1, normalize=0):
    dims, M = _dims(N)
    rid = i64()
    _check(_lib.mdfft_server_submit(server, M, dims, c_void_p(in_ptr), c_void_p(out_ptr), int(dir), int(normalize),
                                    ctypes.byref(rid)), "mdfft_server_submit")
    return rid.value


def mdfft_server_step(server):
    launched = c_int()
    _check(_lib.mdfft_server_step(server, ctypes.byref(launched)), "mdfft_server_step")
    return bool(launched.value)


def mdfft_server_run(server, max_steps):
    n = c_int()
    _check(_lib.mdfft_server_run(server, int(max_steps), ctypes.byref(n)), "mdfft_server_run")
    return n.value


def mdfft_server_poll(server, request_id):
    done, ms = c_int(), ctypes.c_double()
    _check(_lib.mdfft_server_poll(server, int(request_id), ctypes.byref(done), ctypes.byref(ms)),
           "mdfft_server_poll")
    return bool(done.value), ms.value


def mdfft_server_release(server, request_id):
    _check(_lib.mdfft_server_release(server, int(request_id)), "mdfft_server_release")


def mdfft_server_cancel(server, request_id):
    _check(_lib.mdfft_server_cancel(server, int(request_id)), "mdfft_server_cancel")


def mdfft_server_drain(server):
    _check(_lib.mdfft_server_drain(server), "mdfft_server_drain")


def mdfft_server_reset_clock(server):
    _check(_lib.mdfft_server_reset_clock(server), "mdfft_server_reset_clock")


def mdfft_server_set_grid(server, ctas):
    _check(_lib.mdfft_server_set_grid(server, int(ctas)), "mdfft_server_set_grid")


def mdfft_server_set_chunk(server, chunk):
    _check(_lib.mdfft_server_set_chunk(server, int(chunk)), "mdfft_server_set_chunk")


def mdfft_server_set_depth(server, depth):
    _check(_lib.mdfft_server_set_depth(server, int(depth)), "mdfft_server_set_depth")


def mdfft_server_set_direct(server, max_requests):
    _check(_lib.mdfft_server_set_direct(server, int(max_requests)), "mdfft_server_set_direct")


def mdfft_server_set_line_kernel(server, enable):
    _check(_lib.mdfft_server_set_line_kernel(server, int(enable)), "mdfft_server_set_line_kernel")


def mdfft_server_get_stats(server):
    st = MdfftServerStats()
    _check(_lib.mdfft_server_get_stats(server, ctypes.byref(st)), "mdfft_server_get_stats")
    return {f: getattr(st, f) for f, _ in MdfftServerStats._fields_}


def mdfft_server_destroy(server):
    _check(_lib.mdfft_server_destroy(server), "mdfft_server_destroy")


def mdfft_last_error():
    return _lib.mdfft_last_error().decode(errors="replace")


# ------------------------------------------------------------------- torch convenience

_TORCH_DTYPE = {MDFFT_C64: "complex64", MDFFT_C128: "complex128",
                MDFFT_C64_TC_FP16: "complex64", MDFFT_C64_TC_BF16: "complex64"}


class Plan:
    """A plan bound to torch CUDA tensors: ``Plan(shape, P, order, dtype)``.
    With batch > 1 every tensor has shape (batch,) + shape: that many
    independent transforms per execution."""

    def __init__(self, shape, P, order=None, dtype="c64", flags=0, batch=1):
        self.M = len(tuple(shape))
        self.P = int(P)
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.flags = int(flags)
        self.batch = int(batch)
        dims = tuple(int(n) for n in shape)
        self.handle = mdfft_plan_batched(dims, P, order, self.dtype, flags, self.batch)
        self.shape = dims if self.batch == 1 else (self.batch,) + dims
        # MDFFT_PLAN_OUT_LAST_LAYOUT: the output's dims are in the last layout's axis order
        out_dims = dims
        if self.flags & MDFFT_PLAN_OUT_LAST_LAYOUT:
            out_dims = tuple(dims[a] for a in mdfft_plan_order(self.handle, self.M)[-1])
        self.out_shape = out_dims if self.batch == 1 else (self.batch,) + out_dims

    def _stream(self, stream):
        import torch
        s = torch.cuda.current_stream() if stream is None else stream
        return s.cuda_stream

    def _check_tensor(self, t, name, shape=None, cuda=True):
        import torch
        want = getattr(torch, _TORCH_DTYPE[self.dtype])
        shape = self.shape if shape is None else shape
        if not (t.is_cuda == cuda and t.dtype == want and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError(f"{name} must be a contiguous {'CUDA' if cuda else 'host'} {want} tensor of shape {shape}")

    def _out(self, x, out):
        import torch
        if out is None:
            out = torch.empty(self.out_shape, dtype=x.dtype, device=x.device)
        self._check_tensor(out, "out", self.out_shape)
        return out

    def exec(self, x, out=None, dir=-1, normalize=False, stream=None, graph=False):
        """graph=True replays the passes from a CUDA graph captured for these arrays (mdfft_exec_graph)."""
        self._check_tensor(x, "input")
        out = self._out(x, out)
        run = mdfft_exec_graph if graph else mdfft_exec
        run(self.handle, x.data_ptr(), out.data_ptr(), dir, int(bool(normalize)), self._stream(stream))
        return out

    def exec_counted(self, x, out=None, dir=-1, normalize=False, stream=None):
        """Returns (out, counts): counts is an int64 CUDA tensor of 2*M entries."""
        import torch
        self._check_tensor(x, "input")
        out = self._out(x, out)
        counts = torch.empty(2 * self.M, dtype=torch.int64, device=x.device)
        mdfft_exec_counted(self.handle, x.data_ptr(), out.data_ptr(), dir, int(bool(normalize)),
                           self._stream(stream), counts.data_ptr())
        return out, counts

    def comm_volume(self):
        return mdfft_comm_volume(self.handle, self.M)

    def block_grid(self, step):
        """Blocks per natural axis in a step (plans with an MDFFT_PLAN_DECOMP_* flag)."""
        return mdfft_block_grid(self.handle, step, self.M)

    def order(self):
        return mdfft_plan_order(self.handle, self.M)

    def order_str(self):
        return format_order(self.order(), self.M)

    def chunk(self, step, pid):
        return mdfft_chunk(self.handle, step, pid, self.M)

    def describe(self):
        return [mdfft_pass_describe(self.handle, s) for s in range(self.M)]

    def set_timing(self, enable=True):
        mdfft_pass_timing(self.handle, enable)

    def pass_times(self):
        """(mean ms per pass over the recorded executions, how many)."""
        return mdfft_pass_times(self.handle, self.M)

    def exec_host(self, x_host, out_host, dev_in, dev_out, dir=-1, normalize=False, stream=None):
        """End to end on host tensors (pinned for async copies) via caller device buffers."""
        self._check_tensor(dev_in, "dev_in")
        self._check_tensor(dev_out, "dev_out", self.out_shape)
        self._check_tensor(x_host, "x_host", cuda=False)
        self._check_tensor(out_host, "out_host", self.out_shape, cuda=False)
        mdfft_exec_host(self.handle, x_host.data_ptr(), out_host.data_ptr(), dev_in.data_ptr(),
                        dev_out.data_ptr(), dir, int(bool(normalize)), self._stream(stream))
        return out_host

    def autotune(self, x, scratch, reps=10, stream=None):
        """Pick the fastest kernel variant and tile shape per pass; returns
        (ms per pass before, after).  x is only read; scratch is overwritten."""
        self._check_tensor(x, "input")
        self._check_tensor(scratch, "scratch", self.out_shape)
        return mdfft_plan_autotune(self.handle, x.data_ptr(), scratch.data_ptr(), reps, self._stream(stream), self.M)

    def pattern_probe(self, s, x, scratch, reps=10, stream=None):
        """ms per launch of a kernel that moves pass s's data like the pass, without the FFT."""
        self._check_tensor(x, "input")
        self._check_tensor(scratch, "scratch", self.out_shape)
        return mdfft_pattern_probe(self.handle, s, x.data_ptr(), scratch.data_ptr(), reps, self._stream(stream))

    def movement_probe(self, s, x, scratch, slots=2, per_sm=3, reps=10, stream=None):
        """ms per launch of the same data movement through a ring of `slots` slots, `per_sm` CTAs per SM."""
        self._check_tensor(x, "input")
        self._check_tensor(scratch, "scratch", self.out_shape)
        return mdfft_movement_probe(self.handle, s, slots, per_sm, x.data_ptr(), scratch.data_ptr(), reps,
                                    self._stream(stream))

    def tuning(self):
        """The launch choices of every pass (store them, e.g. as JSON, after autotune)."""
        return mdfft_plan_tuning(self.handle, self.M)

    def set_tuning(self, tuning):
        """Reapply stored launch choices (same dims, P, order, dtype, batch and flags)."""
        mdfft_plan_set_tuning(self.handle, tuning)

    def check(self):
        """Raises MdfftError (E_TIMEOUT) if a device-side bounded wait gave up."""
        mdfft_plan_check(self.handle)

    def workspace_bytes(self):
        return mdfft_workspace_size(self.handle)

    def launches(self):
        return mdfft_launches_per_exec(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            mdfft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching server on torch CUDA tensors (complex64)."""

    def __init__(self, budget_bytes, max_inflight=256, P=64, stream=None):
        import torch
        s = torch.cuda.current_stream() if stream is None else stream
        self.stream = s
        self.handle = mdfft_server_create(budget_bytes, max_inflight, P, s.cuda_stream)

    def submit(self, x, out, dir=-1, normalize=False):
        import torch
        for t in (x, out):
            if not (t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
                raise ValueError("server requests take contiguous CUDA complex64 tensors")
        if tuple(x.shape) != tuple(out.shape):
            raise ValueError("input and output shapes differ")
        return mdfft_server_submit(self.handle, tuple(x.shape), x.data_ptr(), out.data_ptr(), dir, int(bool(normalize)))

    def step(self):
        return mdfft_server_step(self.handle)

    def run(self, max_steps=4):
        return mdfft_server_run(self.handle, max_steps)

    def poll(self, rid):
        return mdfft_server_poll(self.handle, rid)

    def release(self, rid):
        mdfft_server_release(self.handle, rid)

    def cancel(self, rid):
        mdfft_server_cancel(self.handle, rid)

    def drain(self):
        mdfft_server_drain(self.handle)

    def reset_clock(self):
        mdfft_server_reset_clock(self.handle)

    def set_grid(self, ctas):
        mdfft_server_set_grid(self.handle, ctas)

    def set_chunk(self, chunk):
        mdfft_server_set_chunk(self.handle, chunk)

    def set_depth(self, depth):
        mdfft_server_set_depth(self.handle, depth)

    def set_direct(self, max_requests):
        mdfft_server_set_direct(self.handle, max_requests)

    def set_line_kernel(self, enable):
        mdfft_server_set_line_kernel(self.handle, int(enable))

    def stats(self):
        return mdfft_server_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            mdfft_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class DistPlan:
    """Device g's part of a transform whose P virtual processes sit on G
    devices (torch CUDA tensors).  Every step runs the library's line DFTs,
    pack and unpack on this device; the values cross devices only through
    `exchange(send, send_counts, recv_counts) -> recv`, the caller's
    all-to-all-v (see torch_exchange)."""

    def __init__(self, shape, P, G, g, order=None, dtype="c64"):
        self.plan = Plan(shape, P, order, dtype)
        self.M, self.G, self.g = self.plan.M, int(G), int(g)

    def local_range(self, step):
        return mdfft_dist_local_range(self.plan.handle, step, self.G, self.g)

    def counts(self, step):
        """G x G points sent from device a (row) to device b (column) at step."""
        return mdfft_exchange_counts(self.plan.handle, step, self.G)

    def run(self, x_local, exchange, dir=-1, normalize=False, stream=None):
        """x_local: this device's range of the natural input (layout 0);
        returns its range of the natural-order result."""
        import torch
        st = self.plan._stream(stream)
        h = self.plan.handle
        cur = x_local
        for s in range(self.M):
            work = torch.empty_like(cur)
            mdfft_dist_lines(h, s, self.G, self.g, cur.data_ptr(), work.data_ptr(), dir, int(bool(normalize)), st)
            c = self.counts(s)
            send_counts = c[self.g]
            recv_counts = [c[a][self.g] for a in range(self.G)]
            send = torch.empty(sum(send_counts), dtype=cur.dtype, device=cur.device)
            mdfft_dist_pack(h, s, self.G, self.g, work.data_ptr(), send.data_ptr(), st)
            recv = exchange(send, send_counts, recv_counts)
            x0, x1 = self.local_range(s + 1)
            nxt = torch.empty(x1 - x0, dtype=cur.dtype, device=cur.device)
            mdfft_dist_unpack(h, s, self.G, self.g, recv.data_ptr(), nxt.data_ptr(), st)
            cur = nxt
        return cur

    def close(self):
        self.plan.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def torch_exchange(group=None, via_host=False):
    """An exchange for DistPlan.run over torch.distributed: one
    all_to_all_single with the step's split sizes (NCCL: grouped send/recv of
    device buffers into a local receive buffer; via_host=True carries the
    buffers through host memory, e.g. for the gloo backend)."""
    import torch
    import torch.distributed as dist

    def exchange(send, send_counts, recv_counts):
        src = send.cpu() if via_host else send
        # complex values travel as (re, im) pairs of reals: two per point
        src = torch.view_as_real(src).reshape(-1)
        recv = torch.empty(2 * sum(recv_counts), dtype=src.dtype, device=src.device)
        dist.all_to_all_single(recv, src, output_split_sizes=[2 * c for c in recv_counts],
                               input_split_sizes=[2 * c for c in send_counts], group=group)
        recv = torch.view_as_complex(recv.view(-1, 2))
        return recv.to(send.device) if via_host else recv

    return exchange
