// tc_group.cuh -- persistent tensor-core pass kernel whose 128-thread groups
// work independently (complex64 data, MDFFT_C64_TC_FP16 / _BF16 plans).
//
// The same pass as fft_pass_tc_kernel (the 1-D DFTs of one step of Fig. 4,
// radix-16 stages as tcgen05 GEMMs with split hi/lo operands and FP32
// accumulators in TMEM, and the transpose after them), organised so that no
// thread waits for another group: a CTA of 256 threads holds two groups of
// 128 (one tcgen05 M = 128 row block each), and each group walks its own
// tiles of 128 / (N / 16) lines with
//  * its own landing buffer, refilled by one bulk copy per line of its next
//    tile, on its own mbarrier;
//  * its own stage buffer, line-major, over which it writes its operand rows;
//  * its own MMA mbarrier and 32 TMEM columns; its first thread issues the
//    group's MMAs, and every warp waits (bounded) on the mbarrier itself;
//  * named barriers of 128 threads (bar.sync 1 + group) only, and its own
//    store of the tile's lines, read line-major from the stage buffer.
// The CTA shares the DFT-16 operand, the twiddles and one TMEM allocation,
// and synchronises as a whole only at set-up and at the end.  While one
// group waits for its MMAs, the other computes operand rows or stores.
//
// Failure handling: a warp whose bounded wait gives up marks itself bad; the
// next group barrier ORs the marks (bar.red.or), so every decision to skip
// work is the same for the whole group and no named barrier is left
// unmatched.  A bad group issues no more MMAs, waits (bounded) for its copies
// in flight and leaves its tile loop; the plan's error flag is set.
//
// Requirements (checked on the host): input and output 16-byte aligned; N a
// power of two from 128 to 1024 (a group holds whole lines).
#pragma once

#include "fft_pipe.cuh"

namespace mdfft {

__device__ __forceinline__ void group_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// bar.sync of the group's 128 threads that also returns the OR of v over them
__device__ __forceinline__ bool group_bar_or(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id)
        : "memory");
    return r != 0;
}

// LAND: each group has a landing buffer refilled by bulk copies (else the
// first stage loads its butterflies straight from HBM: less shared memory,
// more CTAs per SM).
template <int N, int TC, bool LAND_BUF = true> struct TcgCfg {
    static constexpr RadixPlan plan = radix_plan_tc(N);
    static constexpr int NB = N / 16;  // radix-16 butterflies (threads) per line
    static_assert(N % 16 == 0 && NB <= 128 && 128 % NB == 0, "a group of 128 threads holds whole lines");
    static constexpr int LPG = 128 / NB;  // lines per group tile
    static constexpr int G = 2;           // groups per CTA
    static constexpr int THREADS = 128 * G;
    // line stride of the stage buffer: pad16 positions plus padding that puts
    // the store role's reads (LPG lines x 16 / LPG consecutive k per half-warp)
    // on distinct banks (stride = 16 / LPG modulo 16 complex64 words)
    static constexpr int PADN0 = N + N / 16;
    static constexpr int STEP = LPG >= 16 ? 1 : 16 / LPG;
    static constexpr int PADN = PADN0 + ((STEP - PADN0 % 16) % 16 + 16) % 16;
    static constexpr int STAGE = LPG * PADN;  // complex64 per group stage buffer
    static_assert((size_t)STAGE * 8 >= 2 * kTcGroupBytes, "operand rows (hi, lo) fit the group's stage buffer");
    static constexpr int LAND = LAND_BUF ? LPG * N : 0;  // complex64 per group landing buffer
    static constexpr int TWE = tw_entries(plan) > 0 ? tw_entries(plan) : 1;
    static constexpr int TWN = (TWE + 1) / 2 * 2;  // keeps what follows 16-byte aligned
    // head (2 G mbarriers, TMEM slot, group failure flags) | DFT-16 operand |
    // twiddles | per group: landing buffer, stage buffer, line offsets
    static constexpr size_t HEAD = 128;
    static constexpr size_t B_OFF = HEAD;
    static constexpr size_t TW_OFF = B_OFF + 4096;
    static constexpr size_t GRP_OFF = TW_OFF + (size_t)TWN * 8;
    static constexpr size_t GRP_BYTES = ((size_t)LAND * 8 + (size_t)STAGE * 8 + (size_t)LPG * 8 + 15) / 16 * 16;
    static constexpr size_t SMEM = GRP_OFF + G * GRP_BYTES;
    static_assert(SMEM <= 232448, "the CTA's shared memory");
    static_assert(STAGE % 2 == 0 && LAND % 2 == 0, "16-byte aligned group buffers");
    // CTAs per SM the register allocation must allow (3 with landing buffers,
    // whose shared memory allows no more; 4 without)
    static constexpr int MIN_BLOCKS = LAND_BUF ? 3 : 4;
};

// The radix-16 tensor-core stage of one group (see tc_radix16_stage for the
// arithmetic).  Reads the thread's butterfly (from the landing buffer in the
// first stage), writes the group's operand rows over its stage buffer, issues
// the group's MMAs from the group's first thread, waits, and writes the 16
// results line-major into the stage buffer.  Returns the group-uniform bad
// flag (OR over the group at its barriers).
// In the first stage, src is the thread's line (landing buffer or HBM) and
// refill() runs once the whole group has read the landing buffer (after the
// row barrier) -- unless the group is bad.
template <int TC, int N, int NS, bool FIRST, class Hook>
__device__ __forceinline__ bool tcg_radix16(float2 *stage, const float2 *src, const float2 *tw, const uint32_t *bop,
                                            uint32_t tmem, uint64_t *mbar, uint32_t &mpar, int gi, int gt, int line,
                                            int j, bool ok, bool conj, bool bad, const Hook &refill) {
    using K = TcgCfg<N, TC>;
    using T = TcTypes<TC>;
    constexpr int NB = K::NB;
    const int k = j % NS;
    float2 v[16];
    int e = 0;
    if constexpr (FIRST) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = ok ? src[j + r * NB] : make_float2(0.f, 0.f);
        if (conj)
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r].y = -v[r].y;
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            float2 x = stage[line * K::PADN + pad16(j + r * NB)];
            if (r > 0) x = cmul(x, tw[r * NS + k]);
            v[r] = x;
        }
        // every read of the stage buffer before the rows overwrite it
        bad = group_bar_or(1 + gi, bad);
    }
    if constexpr (T::kScale) {
        float m = 0.f;
#pragma unroll
        for (int r = 0; r < 16; ++r) m = fmaxf(m, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
        e = (int)((__float_as_uint(m) >> 23) & 0xff) - 126;
        e = max(-100, min(e, 120));
        const float sc = pow2f(15 - e);
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r].x *= sc, v[r].y *= sc;
    }
    unsigned char *A = reinterpret_cast<unsigned char *>(stage);
    {
        unsigned char *row = A + (gt >> 3) * kTcSbo + (gt & 7) * 16;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int q = (c & 1) * 8 + 2 * w;
                T::split(c < 2 ? v[q].x : v[q].y, c < 2 ? v[q + 1].x : v[q + 1].y, h[w], l[w]);
            }
            *reinterpret_cast<uint4 *>(row + c * kTcLbo) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(row + kTcGroupBytes + c * kTcLbo) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
    fence_proxy_async_shared();  // the rows visible to the tensor cores
    tc_fence_before();           // this thread's earlier TMEM reads before the MMAs
    bad = group_bar_or(1 + gi, bad);
    if (bad) return true;  // group-uniform
    if (gt == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_addr(A), b0 = smem_addr(bop), d = tmem + 32u * (uint32_t)gi;
        constexpr uint32_t idesc = tc_idesc<TC>();
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const uint32_t ao = a0 + ks * 2 * kTcLbo, bo = b0 + ks * 2 * kTcLbo;
            tc_mma(d, tc_desc(ao), tc_desc(bo), idesc, ks);             // hi . hi
            tc_mma(d, tc_desc(ao), tc_desc(bo + 2048), idesc, 1);       // hi . lo
            tc_mma(d, tc_desc(ao + kTcGroupBytes), tc_desc(bo), idesc, 1);  // lo . hi
        }
        tc_commit(mbar);
    }
    if constexpr (FIRST) refill();  // after the MMA issue: the tensor cores start first
    // every warp waits itself; a warp that gives up waits once more (the
    // MMAs must be done before the rows or the columns are reused) and is bad
    bool mine = __all_sync(0xffffffffu, mbar_wait_bounded(mbar, mpar, kTcWaitNs));
    if (!mine) mbar_wait_bounded(mbar, mpar, kTcWaitNs);
    mpar ^= 1;
    if (mine) {  // warp-uniform
        uint32_t d[32];
        tc_fence_after();
        tmem_ld32(tmem + ((uint32_t)(((gt >> 5) & 3) * 32) << 16) + 32u * (uint32_t)gi, d);
        const int base = (j / NS) * NS * 16 + k;
        const float unsc = T::kScale ? pow2f(e - 15) : 1.f;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float2 out = make_float2(__uint_as_float(d[q]), __uint_as_float(d[16 + q]));
            if constexpr (T::kScale) out.x *= unsc, out.y *= unsc;
            stage[line * K::PADN + pad16(base + q * NS)] = out;
        }
    }
    tc_fence_before();
    return !mine;  // made group-uniform at the next group barrier
}

// A radix-R SIMT stage (R = 2, 4, 8) after NS points are combined, line-major
// in place in the group's stage buffer: butterfly jj (< N / R) reads
// x[jj + r N/R], is twiddled by w_{NS R}^{(jj mod NS) r} and writes
// y[(jj / NS) NS R + jj mod NS + r NS].  The line's NB threads share its
// butterflies; all reads come before any write.
template <int N, int R, int NS, int NB, int PADN>
__device__ __forceinline__ void tcg_simt(float2 *stage, const float2 *tw, int line, int j, bool line_in_warp, int gi) {
    constexpr int NBR = N / R, PER = NBR / NB;
    static_assert(NBR % NB == 0, "butterflies per thread");
    float2 v[PER][R];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int jj = j + i * NB;
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = stage[line * PADN + pad16(jj + r * NBR)];
    }
    if (line_in_warp) __syncwarp();
    else group_bar(1 + gi);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int jj = j + i * NB, k = jj % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], tw[r * NS + k]);
        dft<R>(v[i]);
        const int base = (jj / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) stage[line * PADN + pad16(base + r * NS)] = v[i][r];
    }
}

// Stages SI.. of the plan for one group; returns the group's bad flag (made
// uniform at the next group barrier).
template <int TC, int N, int SI, int NS> struct TcgStages {
    using K = TcgCfg<N, TC>;
    static constexpr int R = K::plan.R[SI];
    static constexpr bool LAST = SI == K::plan.S - 1;
    static_assert(SI > 0 || R == 16, "the first stage is a radix-16 tensor-core stage");
    template <class Hook>
    __device__ __forceinline__ static bool run(float2 *stage, const float2 *land, const float2 *tw, const uint32_t *bop,
                                               uint32_t tmem, uint64_t *mbar, uint32_t &mpar, int gi, int gt, int line,
                                               int j, bool ok, bool conj, bool bad, const Hook &refill) {
        constexpr bool IN_WARP = K::NB <= 32;
        if constexpr (R == 16) {
            bad = tcg_radix16<TC, N, NS, SI == 0>(stage, land, tw + tw_offset(K::plan, SI), bop, tmem, mbar, mpar, gi,
                                                  gt, line, j, ok, conj, bad, refill);
        } else {
            tcg_simt<N, R, NS, K::NB, K::PADN>(stage, tw + tw_offset(K::plan, SI), line, j, IN_WARP, gi);
        }
        if constexpr (!LAST) {
            // the next stage reads what the line's threads wrote
            if (IN_WARP) __syncwarp();
            else group_bar(1 + gi);
            return TcgStages<TC, N, SI + 1, NS * R>::run(stage, land, tw, bop, tmem, mbar, mpar, gi, gt, line, j, ok,
                                                         conj, bad, refill);
        }
        return bad;
    }
};

// Store role of one group: its tile's lines, read line-major from the stage
// buffer, go to the output layout (transposed: each thread owns a line and
// writes k = k0, k0 + NB, ...; or whole lines when the output keeps f
// fastest), with the count mode of store_tile.
template <int N, int TC>
__device__ __forceinline__ void tcg_store(const PassArgs &a, const float2 *stage, const int64_t *lbase,
                                          const TileCoord &c, int gt) {
    using K = TcgCfg<N, TC>;
    float2 *out = reinterpret_cast<float2 *>(a.out);
    const bool plain = !(a.conj & 2) && !a.scaled;
    const float sc = plain ? 1.f : (float)a.scale, sy = (a.conj & 2) ? -sc : sc;
    unsigned long long moved = 0, split = 0;
    if (a.line_store) {
        for (int e = gt; e < K::LPG * N; e += 128) {
            const int l = e / N, k = e % N;
            int bg, bh;
            tile_line(a, l, bg, bh);
            if (l < a.Bg * a.Bh && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh) {
                const int64_t o = c.out_base + bh * a.out_sh + bg * a.out_sg + k;
                const float2 v = stage[l * K::PADN + pad16(k)];
                out[o] = plain ? v : make_float2(v.x * sc, v.y * sy);
                if (a.moved) {
                    moved += owner_of(a.own_in, lbase[l] + k) != owner_of(a.own_out, o);
                    if (k == 0)
                        split += (unsigned long long)N *
                                 ((owner_of(a.own_in, lbase[l] + N - 1) - owner_of(a.own_in, lbase[l])) /
                                  a.own_in.line_div);
                }
            }
        }
    } else {
        const int sl = gt % K::LPG, k0 = gt / K::LPG;
        int bg, bh;
        tile_line(a, sl, bg, bh);
        if (sl < a.Bg * a.Bh && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh) {
            const int64_t obase = c.out_base + bh * a.out_sh + bg * a.out_sg;
            float2 *op = out + obase + (int64_t)k0 * a.out_sf;
            const int64_t ostep = (int64_t)K::NB * a.out_sf;
            const float2 *row = stage + sl * K::PADN;
#pragma unroll 4
            for (int k = k0; k < N; k += K::NB, op += ostep) {
                const float2 v = row[pad16(k)];
                *op = plain ? v : make_float2(v.x * sc, v.y * sy);
            }
            if (a.moved) {
                const int64_t ib = lbase[sl];
                for (int k = k0; k < N; k += K::NB)
                    moved += owner_of(a.own_in, ib + k) != owner_of(a.own_out, obase + k * a.out_sf);
                if (k0 == 0)
                    split = (unsigned long long)N *
                            ((owner_of(a.own_in, ib + N - 1) - owner_of(a.own_in, ib)) / a.own_in.line_div);
            }
        }
    }
    if (a.moved) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            moved += __shfl_down_sync(0xffffffffu, moved, o);
            split += __shfl_down_sync(0xffffffffu, split, o);
        }
        if ((gt & 31) == 0) {
            if (moved) atomicAdd(a.moved, moved);
            if (split) atomicAdd(a.split, split);
        }
    }
}

template <int N, int TC, bool LAND_BUF = true>
__global__ void __launch_bounds__(TcgCfg<N, TC, LAND_BUF>::THREADS, TcgCfg<N, TC, LAND_BUF>::MIN_BLOCKS)
    fft_pass_tcg_kernel(const PassArgs a) {
    using K = TcgCfg<N, TC, LAND_BUF>;
    using Tt = TcTypes<TC>;
    extern __shared__ __align__(128) unsigned char tcg_smem[];
    uint64_t *lbar = reinterpret_cast<uint64_t *>(tcg_smem);  // [G] landing buffers
    uint64_t *mbar = lbar + K::G;                              // [G] MMA completion
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + K::G);
    int *gfail = reinterpret_cast<int *>(tmem_slot + 1);  // [G]
    uint32_t *bop = reinterpret_cast<uint32_t *>(tcg_smem + K::B_OFF);
    float2 *tw = reinterpret_cast<float2 *>(tcg_smem + K::TW_OFF);
    const int tid = threadIdx.x, gi = tid >> 7, gt = tid & 127, lane = tid & 31;
    unsigned char *grp = tcg_smem + K::GRP_OFF + (size_t)gi * K::GRP_BYTES;
    float2 *land = reinterpret_cast<float2 *>(grp);
    float2 *stage = land + K::LAND;
    int64_t *lbase = reinterpret_cast<int64_t *>(stage + K::STAGE);
    const float2 *gtw = reinterpret_cast<const float2 *>(a.tw);

    // set-up of the CTA: twiddles, the DFT-16 operand (hi, lo), barriers, TMEM
    for (int q = tid; q < tw_entries(K::plan); q += K::THREADS) tw[q] = gtw[q];
    for (int w = tid; w < 1024; w += K::THREADS) {
        const int hl = w >> 9, n = (w >> 4) & 31, kk = (w & 15) * 2;
        uint32_t hi, lo;
        Tt::split(dft16_block(kk, n), dft16_block(kk + 1, n), hi, lo);
        const uint32_t off = hl * 2048 + (n >> 3) * kTcSbo + (kk >> 3) * kTcLbo + (n & 7) * 16 + (kk & 7) * 2;
        bop[off >> 2] = hl ? lo : hi;
    }
    if (tid == 0) {
        for (int g = 0; g < K::G; ++g) {
            mbar_init(&lbar[g], 1);
            mbar_init(&mbar[g], 1);
            gfail[g] = 0;
        }
        fence_mbarrier_init();
    }
    if (tid < 32) {
        __syncwarp();
        tmem_alloc(tmem_slot, 32 * K::G);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t stride = (int64_t)gridDim.x * K::G;
    int64_t t = (int64_t)blockIdx.x * K::G + gi;
    const bool leader = gt < 32;  // the group's first warp issues its bulk copies
    bool pending = false;         // a landing copy of this group is in flight
    if constexpr (LAND_BUF) {
        if (leader && t < a.ntiles) pipe_issue<N, K::LPG>(a, t, land, &lbar[gi], lane);
        pending = t < a.ntiles;
    }
    uint32_t lpar = 0, mpar = 0;
    bool bad = false;
    const int line = gt / K::NB, j = gt % K::NB;
    for (; t < a.ntiles; t += stride, lpar ^= 1) {
        const TileCoord c = tile_coords(a, t);
        if (gt < K::LPG) {
            int bg, bh;
            tile_line(a, gt, bg, bh);
            lbase[gt] = c.in_base + bg * a.in_sg + bh * a.in_sh;
        }
        if constexpr (LAND_BUF) {
            bool landed = __all_sync(0xffffffffu, mbar_wait_bounded(&lbar[gi], lpar, kTcWaitNs));
            if (!landed) mbar_wait_bounded(&lbar[gi], lpar, kTcWaitNs);  // a second chance before the buffer is reused
            pending = false;
            bad = bad || !landed;
        }
        int fbg, fbh;
        tile_line(a, line, fbg, fbh);
        const bool fok = line < a.Bg * a.Bh && c.g0 + fbg < a.Ng && c.h0 + fbh < a.Nh;
        const float2 *src = LAND_BUF ? land + line * N
                                     : reinterpret_cast<const float2 *>(a.in) + c.in_base + fbg * a.in_sg + fbh * a.in_sh;
        // the first stage reads the landing buffer, writes the rows and reaches
        // the group barrier: then the buffer is refilled with the next tile
        auto refill = [&]() {
            if constexpr (LAND_BUF) {
                if (leader && t + stride < a.ntiles) pipe_issue<N, K::LPG>(a, t + stride, land, &lbar[gi], lane);
                pending = t + stride < a.ntiles;
            }
        };
        bad = TcgStages<TC, N, 0, 1>::run(stage, src, tw, bop, tmem, &mbar[gi], mpar, gi, gt, line, j, fok,
                                          (a.conj & 1) != 0, bad, refill);
        // the results of every line of the group before its store; bad made uniform
        bad = group_bar_or(1 + gi, bad);
        if (bad) break;  // group-uniform
        tcg_store<N, TC>(a, stage, lbase, c, gt);
        group_bar(1 + gi);  // the stage buffer and lbase are rewritten by the next tile
    }
    if (bad) {
        if (pending) mbar_wait_bounded(&lbar[gi], lpar, kTcWaitNs);  // let the copy in flight land
        if (gt == 0) gfail[gi] = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, 32 * K::G);
    }
    if (tid == 0 && a.err)
        for (int g = 0; g < K::G; ++g)
            if (gfail[g]) atomicExch(a.err, 1);
}

}  // namespace mdfft
