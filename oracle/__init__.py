"""Plain FP64 CPU oracle for the row-wise adaptive decomposition M-D FFT.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares no code with
the CUDA library and never imports it.

This module is argument marshalling around ``oracle.c`` (built into
``liboracle.so`` beside it).  What each function computes, and which passage of
the paper (Duy and Ozaki, arXiv:1302.6189) it follows, is stated in
``oracle.c``:

* ``fftn`` / ``fft_axis`` / ``fft1d`` -- Sec. 2, the M-D DFT as M single-axis
  steps of the unnormalised 1-D DFT (forward sign -1).
* ``dft_naive`` / ``dft_point`` -- Sec. 2, the nested M-D sum evaluated point
  by point (all points / one point).
* ``regime`` / ``fmd`` / ``coords`` / ``linear`` / ``chunk`` -- Sec. 3.1-3.2,
  the row-wise map, f_MD and the start/end coordinates.
* ``owner_array`` / ``comm_volume`` / ``split_line`` -- Sec. 3.1 and 3.3, the
  communication amount as the number of points whose owner changes, by brute
  force over owner arrays.
* ``count_orders`` / ``enumerate_orders`` / ``order_search`` -- Sec. 3.2, the
  C_MD count and Table 1, exhaustive search over every transpose order.
* ``fft_fig4`` -- the parallel algorithm of Fig. 4 with explicit per-rank
  chunk buffers.
* ``amount_slab`` / ``amount_pencil`` / ``amount_volumetric`` -- Sec. 4, the
  comparison methods' closed forms.

Parity status: pinned (see the tests); no function is unpinned.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

AXES = "abcdefghijklmnop"


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no GPU)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        i64, i32, c_int, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_double
        sig = {
            "orc_fft1d": (c_int, [P(dbl), i64, c_int]),
            "orc_fft_axis": (c_int, [P(dbl), c_int, P(i64), c_int, c_int, c_int]),
            "orc_fftnd": (c_int, [P(dbl), c_int, P(i64), c_int, c_int]),
            "orc_dft_naive": (c_int, [P(dbl), P(dbl), c_int, P(i64), c_int]),
            "orc_dft_point": (c_int, [P(dbl), c_int, P(i64), P(i64), c_int, P(dbl)]),
            "orc_regime": (c_int, [c_int, P(i64), i64]),
            "orc_fmd": (i64, [c_int, P(i64), i64, i64]),
            "orc_coords": (None, [c_int, P(i64), i64, P(i64)]),
            "orc_linear": (i64, [c_int, P(i64), P(i64)]),
            "orc_chunk": (c_int, [c_int, P(i64), i64, i64, P(i64), P(i64), P(i64), P(i64)]),
            "orc_owner_array": (c_int, [c_int, P(i64), i64, P(c_int), P(i32)]),
            "orc_split_line": (i64, [c_int, P(i64), i64, P(c_int)]),
            "orc_comm_volume": (c_int, [c_int, P(i64), i64, P(c_int), P(i64), P(i64), P(i64)]),
            "orc_count_orders": (i64, [c_int]),
            "orc_enumerate_orders": (i64, [c_int, P(c_int), i64]),
            "orc_order_search": (c_int, [c_int, P(i64), i64, P(i64), P(i64), P(i64), P(i64),
                                         P(c_int), P(c_int), P(c_int), i64, P(i64)]),
            "orc_fft_fig4": (c_int, [P(dbl), P(dbl), c_int, P(i64), i64, P(c_int), c_int,
                                     P(i64), P(i64)]),
            "orc_amount_slab": (dbl, [dbl, dbl]),
            "orc_amount_pencil": (dbl, [dbl, dbl]),
            "orc_amount_volumetric": (dbl, [c_int, dbl, dbl]),
            "orc_block_volume": (c_int, [c_int, P(i64), i64, c_int, P(c_int), P(i64), P(i64), P(i64)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# ----------------------------------------------------------------------------- helpers

def _dims(N):
    arr = (ctypes.c_int64 * len(N))(*[int(n) for n in N])
    return arr, len(N)


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def parse_layout(layout, M=None):
    """'cab' or [2, 0, 1] -> [2, 0, 1] (axis ids, slowest to fastest)."""
    if isinstance(layout, str):
        return [AXES.index(ch) for ch in layout]
    return [int(v) for v in layout]


def parse_order(order):
    """'abc->cab->cba' or a list of layouts -> list of lists of axis ids."""
    if isinstance(order, str):
        parts = [p.strip() for p in order.replace("→", "->").split("->")]
        return [parse_layout(p) for p in parts]
    return [parse_layout(L) for L in order]


def format_order(order):
    return "->".join("".join(AXES[a] for a in L) for L in parse_order(order))


def _order_arr(order):
    flat = [a for L in parse_order(order) for a in L]
    return (ctypes.c_int * len(flat))(*flat)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


# ----------------------------------------------------------------------------- FFTs

def _as_c128(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def fft1d(x, sign=-1):
    y = _as_c128(x).copy()
    _check(_load().orc_fft1d(_ptr(y.view(np.float64), ctypes.c_double), y.size, sign), "fft1d")
    return y


def fft_axis(x, axis, sign=-1, nthreads=1):
    y = _as_c128(x).copy()
    dims, M = _dims(y.shape)
    rc = _load().orc_fft_axis(_ptr(y.view(np.float64), ctypes.c_double), M, dims, axis, sign, nthreads)
    _check(rc, "fft_axis")
    return y


def fftn(x, sign=-1, nthreads=1):
    """Unnormalised M-D DFT of a natural-order array (forward: sign=-1)."""
    y = _as_c128(x).copy()
    dims, M = _dims(y.shape)
    rc = _load().orc_fftnd(_ptr(y.view(np.float64), ctypes.c_double), M, dims, sign, nthreads)
    _check(rc, "fftnd")
    return y


def fftn_inplace(y, sign=-1, nthreads=1):
    """As fftn, overwriting the contiguous complex128 array y (no copy)."""
    assert y.dtype == np.complex128 and y.flags.c_contiguous
    dims, M = _dims(y.shape)
    rc = _load().orc_fftnd(_ptr(y.view(np.float64), ctypes.c_double), M, dims, sign, nthreads)
    _check(rc, "fftnd")
    return y


def dft_naive(x, sign=-1):
    x = _as_c128(x)
    y = np.empty_like(x)
    dims, M = _dims(x.shape)
    rc = _load().orc_dft_naive(_ptr(x.view(np.float64), ctypes.c_double),
                               _ptr(y.view(np.float64), ctypes.c_double), M, dims, sign)
    _check(rc, "dft_naive")
    return y


def dft_point(x, k, sign=-1):
    """One output value Xbar(k) of the M-D DFT of the natural-order array x."""
    x = _as_c128(x)
    dims, M = _dims(x.shape)
    kk = (ctypes.c_int64 * M)(*[int(v) for v in k])
    out = (ctypes.c_double * 2)()
    rc = _load().orc_dft_point(_ptr(x.view(np.float64), ctypes.c_double), M, dims, kk, sign, out)
    _check(rc, "dft_point")
    return complex(out[0], out[1])


def fft_fig4(x, P, order, sign=-1):
    """Fig. 4 route: returns (result, moved[M], split[M])."""
    x = _as_c128(x)
    M = x.ndim
    y = np.empty_like(x)
    dims, _ = _dims(x.shape)
    moved = np.zeros(M, np.int64)
    split = np.zeros(M, np.int64)
    rc = _load().orc_fft_fig4(_ptr(x.view(np.float64), ctypes.c_double),
                              _ptr(y.view(np.float64), ctypes.c_double), M, dims, int(P),
                              _order_arr(order), sign, _ptr(moved, ctypes.c_int64),
                              _ptr(split, ctypes.c_int64))
    _check(rc, "fft_fig4")
    return y, moved, split


# ----------------------------------------------------------------------------- index maps

def regime(N, P):
    dims, M = _dims(N)
    return _load().orc_regime(M, dims, int(P))


def fmd(N, P, myid):
    dims, M = _dims(N)
    return _load().orc_fmd(M, dims, int(P), int(myid))


def coords(N, x):
    dims, M = _dims(N)
    out = (ctypes.c_int64 * M)()
    _load().orc_coords(M, dims, int(x), out)
    return list(out)


def linear(N, c):
    dims, M = _dims(N)
    cc = (ctypes.c_int64 * M)(*[int(v) for v in c])
    return _load().orc_linear(M, dims, cc)


def chunk(N, P, myid):
    """(x_s, x_e, start coords, end coords) of rank myid."""
    dims, M = _dims(N)
    xs, xe = ctypes.c_int64(), ctypes.c_int64()
    cs, ce = (ctypes.c_int64 * M)(), (ctypes.c_int64 * M)()
    rc = _load().orc_chunk(M, dims, int(P), int(myid), ctypes.byref(xs), ctypes.byref(xe), cs, ce)
    _check(rc, "chunk")
    return xs.value, xe.value, list(cs), list(ce)


def owner_array(N, P, layout):
    """Owner rank of every point (natural order) under the chunks of `layout`."""
    L = parse_layout(layout)
    dims, M = _dims(N)
    own = np.empty(tuple(int(n) for n in N), np.int32)
    rc = _load().orc_owner_array(M, dims, int(P), (ctypes.c_int * M)(*L), _ptr(own, ctypes.c_int32))
    _check(rc, "owner_array")
    return own


def split_line(N, P, layout):
    L = parse_layout(layout)
    dims, M = _dims(N)
    return _load().orc_split_line(M, dims, int(P), (ctypes.c_int * M)(*L))


def comm_volume(N, P, order):
    """Amounts of one order, in points: per transition, final, split lines."""
    dims, M = _dims(N)
    per = np.zeros(max(M - 1, 1), np.int64)
    fin = ctypes.c_int64()
    spl = np.zeros(M, np.int64)
    rc = _load().orc_comm_volume(M, dims, int(P), _order_arr(order), _ptr(per, ctypes.c_int64),
                                 ctypes.byref(fin), _ptr(spl, ctypes.c_int64))
    _check(rc, "comm_volume")
    per = per[: M - 1]
    return {"per_transition": per.tolist(), "total": int(per.sum()),
            "final_to_natural": fin.value, "split_line": spl.tolist(),
            "paper_total": int(per.sum() + spl.sum())}


# ----------------------------------------------------------------------------- orders

def count_orders(M):
    return _load().orc_count_orders(int(M))


def enumerate_orders(M, cap=None):
    n = count_orders(M)
    cap = n if cap is None else min(cap, n)
    out = np.zeros((cap, M, M), np.int32)
    _load().orc_enumerate_orders(int(M), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cap)
    return out


def order_search(N, P, best_cap=256):
    dims, M = _dims(N)
    best, worst, nb, nw, nl = (ctypes.c_int64() for _ in range(5))
    bo = np.zeros((M, M), np.int32)
    wo = np.zeros((M, M), np.int32)
    bl = np.zeros((best_cap, M, M), np.int32)
    rc = _load().orc_order_search(M, dims, int(P), ctypes.byref(best), ctypes.byref(worst),
                                  ctypes.byref(nb), ctypes.byref(nw),
                                  bo.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  wo.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  bl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), best_cap,
                                  ctypes.byref(nl))
    _check(rc, "order_search")
    return {"best": best.value, "worst": worst.value, "n_best": nb.value, "n_worst": nw.value,
            "best_order": bo.tolist(), "worst_order": wo.tolist(),
            "best_orders": [format_order(o) for o in bl[: nl.value].tolist()]}


# ----------------------------------------------------------------------------- Sec. 4

def amount_slab(N, P):
    return _load().orc_amount_slab(float(N), float(P))


def amount_pencil(N, P):
    return _load().orc_amount_pencil(float(N), float(P))


def amount_volumetric(M, N, P):
    return _load().orc_amount_volumetric(int(M), float(N), float(P))


BLOCK_KINDS = {"slab": 1, "pencil": 2, "volumetric": 3}


def block_volume(N, P, kind, fft_axes):
    """Amounts of a comparison method of Sec. 4 (kind 'slab', 'pencil' or
    'volumetric') whose steps transform fft_axes in turn, counted point by
    point; q[s][axis] = processes along that axis in step s."""
    dims, M = _dims(N)
    per = np.zeros(max(M - 1, 1), np.int64)
    spl = np.zeros(M, np.int64)
    q = np.zeros((M, M), np.int64)
    ax = (ctypes.c_int * M)(*[int(a) for a in fft_axes])
    rc = _load().orc_block_volume(M, dims, int(P), BLOCK_KINDS[kind], ax, _ptr(per, ctypes.c_int64),
                                  _ptr(spl, ctypes.c_int64), _ptr(q, ctypes.c_int64))
    if rc == -2:
        raise ValueError(f"{kind}: more blocks than points along a cut axis (P = {P})")
    _check(rc, "block_volume")
    per = per[: M - 1]
    return {"per_transition": per.tolist(), "total": int(per.sum()), "split_line": spl.tolist(),
            "paper_total": int(per.sum() + spl.sum()), "q": q.tolist()}
