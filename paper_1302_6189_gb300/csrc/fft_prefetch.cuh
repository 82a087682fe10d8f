// fft_prefetch.cuh -- persistent complex64 pass kernel that loads the next
// tile's first-stage inputs into registers while the current tile is
// transformed and stored (short lines, where a tile's work between its HBM
// loads and its barriers is small).
//
// The same pass as fft_pass_kernel (Fig. 4 step + the transpose after it),
// same tiles, stages and store; each CTA walks tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (the host launches one resident wave).  At the
// top of tile t every thread issues the loads of its first-stage butterflies
// of tile t + gridDim.x; they are consumed one tile later, so their latency
// overlaps tile t.  The twiddles are staged once per CTA.  MINB: CTAs per SM
// the register allocation must allow (2: no spills, 4: a few spilled bytes).
#pragma once

#include "fft_pass.cuh"

namespace mdfft {

template <int N, int RP = 0> struct PfCfg {
    using Cfg = PassCfg<float, N, 0, 0, RP>;
    static_assert(Cfg::DIRECT, "the first stage must read HBM directly");
    static constexpr int R0 = Cfg::plan.R[0];
    static constexpr int NB0 = N / R0;
    static constexpr int PER0 = (NB0 + Cfg::TL - 1) / Cfg::TL;
    static constexpr bool SINGLE = Cfg::plan.S == 1;
    // two sets of tile coordinates and line offsets (tile parity)
    static constexpr size_t SMEM = Cfg::SMEM + (size_t)(Cfg::LINES + 4) * sizeof(int64_t);
};

// Input offset of this thread's line in tile t, and whether the line exists.
template <int N, int RP>
__device__ __forceinline__ bool pf_line(const PassArgs &a, int64_t t, int line, int64_t *base) {
    const TileCoord c = tile_coords(a, t);
    int bg, bh;
    tile_line(a, line, bg, bh);
    *base = c.in_base + bg * a.in_sg + bh * a.in_sh;
    return line < a.Bg * a.Bh && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh;
}

template <int N, int RP>
__device__ __forceinline__ void pf_load(const float2 *in, int64_t base, bool ok, int tl, bool conj,
                                        float2 (&v)[PfCfg<N, RP>::PER0][PfCfg<N, RP>::R0]) {
    using P = PfCfg<N, RP>;
    using Cfg = typename P::Cfg;
#pragma unroll
    for (int i = 0; i < P::PER0; ++i) {
        const int j = tl + i * Cfg::TL;
#pragma unroll
        for (int r = 0; r < P::R0; ++r) {
            float2 x = make_float2(0.f, 0.f);
            if ((P::NB0 % Cfg::TL == 0 || j < P::NB0) && ok) x = __ldg(in + base + j + r * P::NB0);
            if (conj) x.y = -x.y;
            v[i][r] = x;
        }
    }
}

template <int N, int RP = 0, int MINB = 2>
__global__ void __launch_bounds__(PassCfg<float, N, 0, 0, RP>::THREADS, MINB) fft_pass_pf_kernel(const PassArgs a) {
    using P = PfCfg<N, RP>;
    using Cfg = typename P::Cfg;
    using C = float2;
    extern __shared__ __align__(16) unsigned char pf_smem[];
    C *buf = reinterpret_cast<C *>(pf_smem);  // stage buffer / transposed tile
    C *tw = buf + Cfg::DATA;
    int64_t *sets = reinterpret_cast<int64_t *>(tw + Cfg::TWN + Cfg::BFRAG);  // 2 x (line offsets, tile coordinates)
    const int tid = threadIdx.x;
    const int line = tid / Cfg::TL, tl = tid % Cfg::TL;
    const C *in = reinterpret_cast<const C *>(a.in);
    const C *gtw = reinterpret_cast<const C *>(a.tw);
    const bool conj = (a.conj & 1) != 0;
    for (int q = tid; q < tw_entries(Cfg::plan); q += Cfg::THREADS) tw[q] = gtw[q];

    __syncthreads();  // the twiddles before any stage reads them
    const int64_t G = gridDim.x;
    int64_t t = blockIdx.x;
    C cur[P::PER0][P::R0], nxt[P::PER0][P::R0];
    int64_t base = 0;
    bool ok = false;
    if (t < a.ntiles) {
        ok = pf_line<N, RP>(a, t, line, &base);
        pf_load<N, RP>(in, base, ok, tl, conj, cur);
    }
    for (int par = 0; t < a.ntiles; t += G, par ^= 1) {
        const bool fok = ok;
        // the next tile's inputs: in flight while this tile is computed and stored
        if (t + G < a.ntiles) {
            ok = pf_line<N, RP>(a, t + G, line, &base);
            pf_load<N, RP>(in, base, ok, tl, conj, nxt);
        }
        int64_t *lbase = sets + par * (Cfg::LINES + 4);
        TileCoord *shc = reinterpret_cast<TileCoord *>(lbase + Cfg::LINES);
        if (tid < 32) {
            const TileCoord w0 = tile_coords(a, t);
            if (tid == 0) *shc = w0;
            for (int l = tid; l < Cfg::LINES; l += 32) {
                int bg, bh;
                tile_line(a, l, bg, bh);
                lbase[l] = w0.in_base + bg * a.in_sg + bh * a.in_sh;
            }
        }
        // the first stage (no twiddles) from the registers (the previous
        // tile's store finished reading the buffer at the end of its iteration)
        constexpr int R = P::R0, NB = P::NB0;
#pragma unroll
        for (int i = 0; i < P::PER0; ++i) {
            const int j = tl + i * Cfg::TL;
            if ((NB % Cfg::TL == 0 || j < NB) && fok) {
                dft<R>(cur[i]);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if constexpr (P::SINGLE) buf[(j * R + r) * Cfg::TROW + line] = cur[i][r];
                    else buf[line * Cfg::PADN + padg<Cfg::PADG>(j * R + r)] = cur[i][r];
                }
            }
        }
        if constexpr (P::SINGLE) {
            __syncthreads();
        } else {
            constexpr bool WARP_LOCAL = 32 % Cfg::TL == 0;
            if constexpr (WARP_LOCAL && Cfg::plan.S > 1) __syncwarp();
            else __syncthreads();
            Stages<float, N, 1, R, 0, 0, -1, RP>::run(buf, buf, tw, nullptr, line, tl, fok, false, true);
        }
        store_tile<float, N, 0, 0, RP>(a, buf, lbase, *shc, tid);
        __syncthreads();  // the buffer is rewritten by the next tile's first stage
#pragma unroll
        for (int i = 0; i < P::PER0; ++i)
#pragma unroll
            for (int r = 0; r < R; ++r) cur[i][r] = nxt[i][r];
    }
}

}  // namespace mdfft

namespace mdfft {

// 256-point lines (radix 16 x 16, 16 threads per line) with the exchange
// between the two stages done in registers: after the first stage, thread j
// of a line holds y[16 j + q], q = 0..15, and the second stage's butterfly j
// needs y[16 r + j], r = 0..15 -- a 16 x 16 transpose across the line's 16
// lanes, done in four XOR steps of warp shuffles (step m swaps, between lanes
// j and j ^ m, the elements whose index differs from the lane in bit m).  No
// shared memory between the stages; the second stage writes the transposed
// tile and the store is unchanged.  An autotuning variant.
__global__ void __launch_bounds__(PassCfg<float, 256>::THREADS, 4) fft_pass_shfl256_kernel(const PassArgs a) {
    using Cfg = PassCfg<float, 256>;
    using C = float2;
    static_assert(Cfg::TL == 16 && Cfg::plan.S == 2 && Cfg::plan.R[0] == 16 && Cfg::plan.R[1] == 16, "256 = 16 x 16");
    extern __shared__ __align__(16) unsigned char sh_smem[];
    C *buf = reinterpret_cast<C *>(sh_smem);  // transposed tile [k][TROW]
    C *tw = buf + Cfg::DATA;
    int64_t *lbase = reinterpret_cast<int64_t *>(tw + Cfg::TWN + Cfg::BFRAG);
    TileCoord *shc = reinterpret_cast<TileCoord *>(lbase + Cfg::LINES);
    const int tid = threadIdx.x;
    const C *in = reinterpret_cast<const C *>(a.in);
    const C *gtw = reinterpret_cast<const C *>(a.tw);
    if (tid < 32) {
        const TileCoord w0 = tile_coords(a, blockIdx.x);
        if (tid == 0) *shc = w0;
        for (int l = tid; l < Cfg::LINES; l += 32) {
            int bg, bh;
            tile_line(a, l, bg, bh);
            lbase[l] = w0.in_base + bg * a.in_sg + bh * a.in_sh;
        }
    }
    for (int q = tid; q < tw_entries(Cfg::plan); q += Cfg::THREADS) tw[q] = gtw[q];
    __syncthreads();
    const TileCoord c = *shc;
    const int line = tid / 16, j = tid % 16;
    int fbg, fbh;
    tile_line(a, line, fbg, fbh);
    const bool ok = line < a.Bg * a.Bh && c.g0 + fbg < a.Ng && c.h0 + fbh < a.Nh;
    C v[16];
    const C *src = in + lbase[line];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        C x = ok ? __ldg(src + j + 16 * r) : C{0, 0};
        if (a.conj & 1) x.y = -x.y;
        v[r] = x;
    }
    dft<16>(v);  // v[q] = y[16 j + q]
    // transpose across the line's 16 lanes: afterwards v[r] = y[16 r + j]
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) {
        const bool hi = (j & m) != 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i & m) continue;
            const C send = hi ? v[i] : v[i | m];
            C got;
            got.x = __shfl_xor_sync(0xffffffffu, send.x, m);
            got.y = __shfl_xor_sync(0xffffffffu, send.y, m);
            if (hi) v[i] = got;
            else v[i | m] = got;
        }
    }
    // second stage: twiddles w_256^{j r}, DFT-16, results to the transposed tile
    constexpr int TWOFF = tw_offset(Cfg::plan, 1);
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw[TWOFF + r * 16 + j]);
    dft<16>(v);
    if (ok)
#pragma unroll
        for (int q = 0; q < 16; ++q) buf[(j + 16 * q) * Cfg::TROW + line] = v[q];
    __syncthreads();
    store_tile<float, 256, 0, 0>(a, buf, lbase, c, tid);
}

}  // namespace mdfft
