#!/usr/bin/env python3
"""Writes smem_layout.h: shared-memory padding of the complex64 pass kernels.

For every complex64 line length N (up to 256) and CTA variant (default, 256 or
512 threads; 192 or 384 for 24 and 48; the alternative radix plan of the
tuned lengths) this replays the kernel's shared-memory accesses -- staged tile
loads, every Stockham stage's reads and writes, the transposed-tile writes of
the last stage and the store role's reads -- warp instruction by warp
instruction, counts the wavefronts each needs (8-byte accesses are served
half a warp at a time: per half, the most distinct 4-byte words one bank
holds), and keeps the layout with the fewest:
    pad(i) = i + i / g           (g in {8, 16, 32})
    line stride  = N + N / g + pe
    tile row     = LINES + te
It mirrors the launch rules of fft_pass.cuh (radix plans, threads per line,
lines per tile); run it again after changing them:
    python gen_smem_layout.py > smem_layout.h
"""
import math
import sys

LENGTHS = [1, 2, 3, 4, 5, 6, 8, 10, 12, 15, 16, 20, 24, 30, 32, 40, 48, 60, 64, 80, 96, 120, 128, 160, 192,
           240, 256]
TUNED = [32, 48, 64, 96, 128, 160, 192, 256, 512]
POW2_DEFAULT = [24, 48, 240, 480, 960]  # pow2_threads_default() of fft_pass.cuh
SERVE = [16, 24, 32, 48, 64, 96, 128, 160, 192, 256]


def radix_plan(n, rp=0):
    e = 0
    while n % 2 == 0:
        n //= 2
        e += 1
    pw = {0: [], 1: [2], 2: [4], 3: [8], 4: [16], 5: [8, 4], 6: [8, 8], 7: [16, 8], 8: [16, 16], 9: [16, 16, 2],
          10: [16, 8, 8]}
    if rp:  # radix_plan_alt()
        pw = {0: [], 1: [2], 2: [4], 3: [8], 4: [4, 4], 5: [16, 2], 6: [16, 4], 7: [8, 4, 4], 8: [8, 8, 4],
              9: [8, 8, 8], 10: [16, 16, 4]}
    r = list(pw[e])
    while n % 5 == 0:
        r.append(5)
        n //= 5
    while n % 3 == 0:
        r.append(3)
        n //= 3
    return r


def launch(n, thr, elem=8, rp=0):
    r = radix_plan(n, rp)
    tl0 = n // max(r) if r else n
    min_lines = 128 // elem
    p = 1
    while p < tl0:
        p *= 2
    if thr:
        tl = min(p, thr // min_lines)
        return r, tl, thr // tl
    tl = p if n in POW2_DEFAULT else tl0
    l = min_lines
    while l > 1 and tl * l > 1024:
        l //= 2
    while l < 256 and 2 * l * n <= 4096 and 2 * tl * l <= 256:  # complex64 tiles grow to 256 threads
        l *= 2
    while (tl * l) % 32 and 2 * tl * l <= 1024:
        l *= 2
    return r, tl, l


def wavefronts(addrs):
    # 8-byte accesses are served half a warp at a time: per half, the most
    # distinct 4-byte words any bank holds
    total = 0
    for half in (addrs[:16], addrs[16:]):
        banks = {}
        for a in half:
            if a is None:
                continue
            for w in (2 * a, 2 * a + 1):
                banks.setdefault(w % 32, set()).add(w)
        total += max((len(v) for v in banks.values()), default=0)
    return total


def cost(n, thr, g, pe, te, rp=0):
    r, tl, lines = launch(n, thr, rp=rp)
    threads = tl * lines
    padn, trow = n + n // g + pe, lines + te

    def pad(i):
        return i + i // g

    total = 0
    def warp_access(fn):
        nonlocal total
        for w0 in range(0, threads, 32):
            a = [fn(tid) for tid in range(w0, w0 + 32)]  # lane order kept: halves are lanes 0-15, 16-31
            if any(x is not None for x in a):
                total += wavefronts(a)

    direct = tl * 8 >= 32
    if not direct:  # staged load of the tile
        for q in range(-(-lines * n // threads)):
            warp_access(lambda tid: None if tid + q * threads >= lines * n else
                        ((tid + q * threads) // n) * padn + pad((tid + q * threads) % n))
    ns = 1
    for si, rr in enumerate(r):
        nb, last = n // rr, si == len(r) - 1
        per = -(-nb // tl)
        for i in range(per):
            for k in range(rr):
                if not (si == 0 and direct):
                    warp_access(lambda tid: None if (tid % tl) + i * tl >= nb else
                                (tid // tl) * padn + pad((tid % tl) + i * tl + k * nb))

                def wr(tid):
                    j = (tid % tl) + i * tl
                    if j >= nb:
                        return None
                    base = (j // ns) * ns * rr + j % ns
                    return (base + k * ns) * trow + tid // tl if last else (tid // tl) * padn + pad(base + k * ns)
                warp_access(wr)
        ns *= rr
    for q in range(-(-n // tl)):  # store role
        warp_access(lambda tid: None if tid // lines + q * tl >= n else (tid // lines + q * tl) * trow + tid % lines)
    return total


def best(n, thr, rp=0):
    default = cost(n, thr, 16, 1, 1, rp)
    cands = []
    for g in (8, 16, 32):
        for pe in range(0, 9):
            for te in (0, 1, 2, 4, 8, 16):
                cands.append((cost(n, thr, g, pe, te, rp), n + n // g + pe + launch(n, thr, rp=rp)[2] + te, g, pe, te))
    c = min(cands)
    return (c[2], c[3], c[4]) if c[0] < default else (16, 1, 1)


THREE_LINES = [24, 48]  # fixed 192 / 384-thread variants (48 / 96 lines)


def main():
    rows = []
    for thr in (0, 256, 512, 192, 384):
        for n in LENGTHS + [512]:
            if thr == 0 and n > 256:
                continue
            if thr in (256, 512) and n not in set(TUNED) | set(SERVE):
                continue
            if thr == 512 and n not in TUNED:
                continue
            if thr in (192, 384) and n not in THREE_LINES:
                continue
            if n < 2 or not radix_plan(n):
                continue
            g, pe, te = best(n, thr)
            if (g, pe, te) != (16, 1, 1):
                rows.append((n, thr, 0, g, pe, te))
    for n in TUNED:  # the alternative radix plans (default CTA shape)
        g, pe, te = best(n, 0, 1)
        if (g, pe, te) != (16, 1, 1):
            rows.append((n, 0, 1, g, pe, te))
    out = sys.stdout
    out.write("// smem_layout.h -- generated by gen_smem_layout.py; do not edit.\n")
    out.write("// Shared-memory padding of the complex64 pass kernels with the fewest bank\n")
    out.write("// conflicts (pad(i) = i + i/g, line stride N + N/g + pe, tile row LINES + te).\n")
    out.write("#pragma once\n\nnamespace mdfft {\n\nstruct SmemLayout {\n    int g, pe, te;\n};\n\n")
    out.write("__host__ __device__ constexpr SmemLayout smem_layout_c64(int n, int thr, int rp = 0) {\n")
    for n, thr, rp, g, pe, te in rows:
        out.write(f"    if (n == {n} && thr == {thr} && rp == {rp}) return SmemLayout{{{g}, {pe}, {te}}};\n")
    out.write("    return SmemLayout{16, 1, 1};\n}\n\n}  // namespace mdfft\n")


if __name__ == "__main__":
    main()
