// fft_line.cuh -- complex64 pass kernel for short lines with one thread per
// line: the thread holds its line in registers and runs every radix stage of
// the default kernel's plan there, so no shared memory and no barrier lies
// between the stages, and it stores its outputs straight from registers.
//
// The same pass as fft_pass_kernel (the Fig. 4 step and the transpose after
// it): the same radix plan, twiddles and butterflies in the same order, so
// the results are bit-identical.  What changes is the work per point.  With
// several threads per line (the default shape of lengths up to 64) every
// thread repeats its stage's addressing, predicates and loop control for a
// few points, a radix that does not divide the line's butterflies among the
// threads leaves lanes idle, and the stages exchange values through shared
// memory behind barriers; here each instruction of a warp does the work of
// 32 lines.
//
// A warp owns 32 consecutive lines of the tile.  It copies them (16-byte
// units, consecutive lanes on consecutive units of a line) into its own
// staging rows in shared memory; after __syncwarp each lane reads its row
// (16-byte reads: the row stride, 2 mod 4 elements, puts 8 consecutive rows
// on distinct bank groups), transforms it and writes element k of its line
// for k = 0 .. N-1: at fixed k the lanes write consecutive points of the
// tile's g axis, the output layout's fastest (runs of Bg elements, as the
// default store writes).  No CTA barrier at all: the twiddles come from the
// read-only cache (the same table the default kernel stages).
#pragma once

#include "fft_pass.cuh"

namespace mdfft {

// the radix stages of PassCfg<float, N, 0, 0, RP>'s plan on a line held in
// registers: stage SI after NS points already combined, butterfly j as in
// Stages::simt
template <int N, int SI, int NS, int RP = 0> struct RegStages {
    static constexpr RadixPlan P = PassCfg<float, N, 0, 0, RP>::plan;
    static constexpr int R = P.R[SI], NB = N / R, TWOFF = tw_offset(P, SI);
    __device__ __forceinline__ static void run(float2 (&x)[N], const float2 *tw) {
        float2 y[N];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = x[j + r * NB];
            const int k = j % NS;
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + TWOFF + r * NS + k));
            }
            dft<R>(v);
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) y[base + r * NS] = v[r];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = y[i];
        if constexpr (SI + 1 < P.S) RegStages<N, SI + 1, NS * R, RP>::run(x, tw);
    }
};

// RP: the radix plan (as in PassCfg); WARPS: warps per CTA (32 lines each)
template <int N, int RP = 0, int WARPS = 4> struct LineCfg {
    static_assert(N % 2 == 0 && N >= 2, "lines are copied in 16-byte units (two complex64)");
    static constexpr RadixPlan plan = PassCfg<float, N, 0, 0, RP>::plan;
    static constexpr int LINES = 32 * WARPS, THREADS = LINES;
    static constexpr int CH = N / 2;                     // 16-byte units per line
    static constexpr int RS = N % 4 == 2 ? N : N + 2;    // staging row stride (complex64), 2 mod 4
    static constexpr size_t SMEM = (size_t)LINES * RS * sizeof(float2) + (size_t)LINES * sizeof(int64_t);
};

// One warp's 32 lines of tile c: tile lines w0 .. w0 + 31, lane = line - w0.
// line_issue copies them into the warp's 32 staging rows (RS elements each;
// lbase: 32 entries) as one cp.async commit group; line_finish, once that
// group has landed and the warp has met at __syncwarp, transforms and stores
// them.  line_issue begins with __syncwarp, so a warp may refill rows it has
// read before.
template <int N, int RP = 0>
__device__ __forceinline__ void line_issue(const PassArgs &a, const TileCoord &c, int w0, float2 *stage,
                                           int64_t *lbase, int lane) {
    using LC = LineCfg<N, RP, 1>;
    using C = float2;
    const C *in = reinterpret_cast<const C *>(a.in);
    const int line = w0 + lane;
    int bg, bh;
    tile_line(a, line, bg, bh);
    const bool ok = line < a.Bg * a.Bh && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh;
    const int64_t ib = c.in_base + (int64_t)bg * a.in_sg + (int64_t)bh * a.in_sh;
    __syncwarp();  // earlier reads of these rows and offsets are done
    lbase[lane] = ok ? ib : -1;
    __syncwarp();
    // unit e = lane + 32 i is unit u of line l
#pragma unroll
    for (int i = 0; i < LC::CH; ++i) {
        const int e = lane + 32 * i, l = e / LC::CH, u = e - l * LC::CH;
        const int64_t b = lbase[l];
        if (b >= 0) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(stage + l * LC::RS + 2 * u);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(in + b + 2 * u) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N, int RP = 0>
__device__ __forceinline__ void line_finish(const PassArgs &a, const TileCoord &c, int w0, const float2 *stage,
                                            int lane) {
    using LC = LineCfg<N, RP, 1>;
    using C = float2;
    C *out = reinterpret_cast<C *>(a.out);
    const C *gtw = reinterpret_cast<const C *>(a.tw);
    const int line = w0 + lane;
    int bg, bh;
    tile_line(a, line, bg, bh);
    const bool ok = line < a.Bg * a.Bh && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh;
    const int64_t ib = c.in_base + (int64_t)bg * a.in_sg + (int64_t)bh * a.in_sh;
    C x[N];
    const C *row = stage + lane * LC::RS;
#pragma unroll
    for (int u = 0; u < LC::CH; ++u) {
        const float4 q = *reinterpret_cast<const float4 *>(row + 2 * u);
        x[2 * u] = C{q.x, q.y};
        x[2 * u + 1] = C{q.z, q.w};
    }
    if (a.conj & 1)
#pragma unroll
        for (int k = 0; k < N; ++k) x[k].y = -x[k].y;
    if constexpr (LC::plan.S > 0) RegStages<N, 0, 1, RP>::run(x, gtw);

    const int64_t ob = c.out_base + (int64_t)bh * a.out_sh + (int64_t)bg * a.out_sg;
    if (ok) {
        C *op = out + ob;
        if (!(a.conj & 2) && !a.scaled) {
#pragma unroll
            for (int k = 0; k < N; ++k) op[k * a.out_sf] = x[k];
        } else {
            const float sc = (float)a.scale, sy = (a.conj & 2) ? -sc : sc;
#pragma unroll
            for (int k = 0; k < N; ++k) op[k * a.out_sf] = C{x[k].x * sc, x[k].y * sy};
        }
    }
    if (a.moved) {  // count mode: owner of every point before and after, the split-line amount once per line
        unsigned long long moved = 0, split = 0;
        if (ok) {
            for (int k = 0; k < N; ++k)
                moved += owner_of(a.own_in, ib + k) != owner_of(a.own_out, ob + k * a.out_sf);
            split = (unsigned long long)N *
                    ((owner_of(a.own_in, ib + N - 1) - owner_of(a.own_in, ib)) / a.own_in.line_div);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            moved += __shfl_down_sync(0xffffffffu, moved, o);
            split += __shfl_down_sync(0xffffffffu, split, o);
        }
        if (lane == 0) {
            if (moved) atomicAdd(a.moved, moved);
            if (split) atomicAdd(a.split, split);
        }
    }
}

// The whole tile for one warp: copy, wait, transform and store.
template <int N, int RP = 0>
__device__ __forceinline__ void line_warp(const PassArgs &a, const TileCoord &c, int w0, float2 *stage,
                                          int64_t *lbase, int lane) {
    line_issue<N, RP>(a, c, w0, stage, lbase, lane);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    line_finish<N, RP>(a, c, w0, stage, lane);
}

// One tile of LINES = 32 WARPS lines per CTA; warp w takes tile lines 32 w ..
template <int N, int RP = 0, int WARPS = 4>
__global__ void __launch_bounds__(LineCfg<N, RP, WARPS>::THREADS) fft_pass_line_kernel(const PassArgs a) {
    using LC = LineCfg<N, RP, WARPS>;
    extern __shared__ __align__(16) unsigned char line_smem[];
    float2 *stage = reinterpret_cast<float2 *>(line_smem);                     // [LINES][RS]
    int64_t *lbase = reinterpret_cast<int64_t *>(stage + LC::LINES * LC::RS);  // input offset of each line, -1: none
    const int tid = threadIdx.x, lane = tid & 31, w0 = tid - lane;
    const TileCoord c = tile_coords(a, blockIdx.x);
    line_warp<N, RP>(a, c, w0, stage + w0 * LC::RS, lbase + w0, lane);
}

// Two threads per line, for two-stage plans whose radices are even (32 = 8 x 4,
// 64 = 8 x 8, and the alternative plans 16 x 2, 16 x 4): half the registers
// of one thread per line, so more warps per SM for the longer short lines.
// Lane pair (2 l, 2 l + 1) owns line l of the warp's 16; lane parity t holds
// the points of index parity t.  The first stage's butterflies j = 2 q + t
// read only those points (their inputs j + r R1 have the parity of j, R1
// even); the second stage's butterfly j1 = 2 p + t needs column j1 of every
// first-stage row, half of them held by the partner lane, which sends them
// in one exchange of N / 4 values (warp shuffle, lane ^ 1).  Same
// butterflies, twiddles and order as Stages::simt: bit-identical results.
template <int N, int RP = 0> struct Line2Cfg {
    static constexpr RadixPlan plan = PassCfg<float, N, 0, 0, RP>::plan;
    static constexpr int R0 = plan.R[0], R1 = plan.R[1], H = N / 2;
    static_assert(plan.S == 2 && R0 % 2 == 0 && R1 % 2 == 0 && N % 4 == 0, "two stages, even radices");
    static constexpr int WARPS = 4, LPW = 16, LINES = LPW * WARPS, THREADS = 32 * WARPS;
    static constexpr int CH = N / 2;                   // 16-byte units per line
    static constexpr int RS = N % 4 == 2 ? N : N + 2;  // row stride 2 mod 4: lanes (l, t) on distinct banks
    static constexpr int TWOFF1 = tw_offset(plan, 1);
    static constexpr size_t SMEM = (size_t)LINES * RS * sizeof(float2) + (size_t)LINES * sizeof(int64_t);
};

template <int N, int RP = 0>
__device__ __forceinline__ void line2_warp(const PassArgs &a, const TileCoord &c, int w0, float2 *stage,
                                           int64_t *lbase, int lane) {
    using L2 = Line2Cfg<N, RP>;
    using C = float2;
    constexpr int R0 = L2::R0, R1 = L2::R1;
    const C *in = reinterpret_cast<const C *>(a.in);
    C *out = reinterpret_cast<C *>(a.out);
    const C *gtw = reinterpret_cast<const C *>(a.tw);
    const int l = lane >> 1, t = lane & 1, line = w0 + l;
    int bg, bh;
    tile_line(a, line, bg, bh);
    const bool ok = line < a.Bg * a.Bh && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh;
    const int64_t ib = c.in_base + (int64_t)bg * a.in_sg + (int64_t)bh * a.in_sh;
    __syncwarp();  // earlier reads of these rows and offsets are done (a warp may run tile after tile)
    if (t == 0) lbase[l] = ok ? ib : -1;
    __syncwarp();
    // the warp's 16 lines into its rows: unit e = lane + 32 i is unit u of line ll
#pragma unroll
    for (int i = 0; i < L2::CH / 2; ++i) {
        const int e = lane + 32 * i, ll = e / L2::CH, u = e - ll * L2::CH;
        const int64_t b = lbase[ll];
        if (b >= 0) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(stage + ll * L2::RS + 2 * u);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(in + b + 2 * u) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();

    C x[L2::H];  // points 2 m + t of the line
    const C *row = stage + l * L2::RS + t;
#pragma unroll
    for (int m = 0; m < L2::H; ++m) x[m] = row[2 * m];
    if (a.conj & 1)
#pragma unroll
        for (int m = 0; m < L2::H; ++m) x[m].y = -x[m].y;
    // first stage (no twiddles): butterfly j = 2 q + t reads points j + r R1 = x[q + r R1 / 2]
    C y[R1 / 2][R0];
#pragma unroll
    for (int q = 0; q < R1 / 2; ++q) {
        C v[R0];
#pragma unroll
        for (int r = 0; r < R0; ++r) v[r] = x[q + r * (R1 / 2)];
        dft<R0>(v);
#pragma unroll
        for (int r = 0; r < R0; ++r) y[q][r] = v[r];
    }
    // exchange: send column 2 p + 1 - t of every own row, receive column 2 p + t of the partner's
    C z[R1 / 2][R0 / 2];
#pragma unroll
    for (int q = 0; q < R1 / 2; ++q)
#pragma unroll
        for (int p = 0; p < R0 / 2; ++p) {
            const C snd = t ? y[q][2 * p] : y[q][2 * p + 1];
            z[q][p].x = __shfl_xor_sync(0xffffffffu, snd.x, 1);
            z[q][p].y = __shfl_xor_sync(0xffffffffu, snd.y, 1);
        }
    // second stage: butterfly j1 = 2 p + t reads column j1 of rows r (row r of parity t is own)
    const int64_t ob = c.out_base + (int64_t)bh * a.out_sh + (int64_t)bg * a.out_sg;
    C *op = out + ob;
    const bool plain = !(a.conj & 2) && !a.scaled;
    const float sc = (float)a.scale, sy = (a.conj & 2) ? -sc : sc;
#pragma unroll
    for (int p = 0; p < R0 / 2; ++p) {
        const int j1 = 2 * p + t;
        C v[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const C own = (r & 1) ? y[r / 2][2 * p + 1] : y[r / 2][2 * p];
            v[r] = ((r & 1) == t) ? own : z[r / 2][p];
        }
#pragma unroll
        for (int r = 1; r < R1; ++r) v[r] = cmul(v[r], __ldg(gtw + L2::TWOFF1 + r * R0 + j1));
        dft<R1>(v);
        if (ok) {
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int64_t k = j1 + r * R0;
                op[k * a.out_sf] = plain ? v[r] : C{v[r].x * sc, v[r].y * sy};
            }
        }
    }
    if (a.moved) {  // count mode: every point of the line once (each lane its parity), the split amount once
        unsigned long long moved = 0, split = 0;
        if (ok) {
            for (int k = t; k < N; k += 2)
                moved += owner_of(a.own_in, ib + k) != owner_of(a.own_out, ob + k * a.out_sf);
            if (t == 0)
                split = (unsigned long long)N *
                        ((owner_of(a.own_in, ib + N - 1) - owner_of(a.own_in, ib)) / a.own_in.line_div);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            moved += __shfl_down_sync(0xffffffffu, moved, o);
            split += __shfl_down_sync(0xffffffffu, split, o);
        }
        if (lane == 0) {
            if (moved) atomicAdd(a.moved, moved);
            if (split) atomicAdd(a.split, split);
        }
    }
}

// One tile of 64 lines per CTA; warp w takes tile lines 16 w ..
template <int N, int RP = 0>
__global__ void __launch_bounds__(Line2Cfg<N, RP>::THREADS) fft_pass_line2_kernel(const PassArgs a) {
    using L2 = Line2Cfg<N, RP>;
    extern __shared__ __align__(16) unsigned char line2_smem[];
    float2 *stage = reinterpret_cast<float2 *>(line2_smem);                     // [LINES][RS]
    int64_t *lbase = reinterpret_cast<int64_t *>(stage + L2::LINES * L2::RS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, w0 = warp * L2::LPW;
    const TileCoord c = tile_coords(a, blockIdx.x);
    line2_warp<N, RP>(a, c, w0, stage + w0 * L2::RS, lbase + w0, lane);
}

}  // namespace mdfft
