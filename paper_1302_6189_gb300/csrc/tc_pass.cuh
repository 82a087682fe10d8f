// tc_pass.cuh -- persistent pass kernel with tensor-core radix-16 stages
// (complex64 data, MDFFT_C64_TC_FP16 / MDFFT_C64_TC_BF16 plans).
//
// The same pass as fft_pass_kernel (the 1-D DFTs of one step of Fig. 4 and
// the transpose after it), but each CTA walks tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (the host launches at most one resident wave):
//  * the per-CTA set-up of the tensor-core stages -- the DFT-16 operand, the
//    mbarriers and the TMEM accumulator columns -- is paid once per CTA;
//  * the next tile's lines are copied into a landing buffer in shared memory
//    (one cp.async.bulk per line, warp 0, completing on an mbarrier with the
//    tile's byte count) while the current tile is transformed and stored, so
//    the HBM latency is not on each tile's path.
// Per tile: warp 0 turns the tile index into coordinates and waits (bounded)
// for the landing buffer; the radix-16 stages run as tcgen05 GEMMs
// (tc_stage.cuh; the first reads the landing buffer, which is refilled right
// after it), any remaining radix 2/4/8/3/5 stages on the SIMT path, and the
// transposed tile is stored as in fft_pass_kernel.  A wait that gives up sets
// the plan's error flag (MDFFT_E_TIMEOUT from mdfft_plan_check).
//
// Requirements (checked on the host): input and output 16-byte aligned.
#pragma once

#include "fft_pipe.cuh"

namespace mdfft {

__host__ __device__ constexpr int tc_stage_count(const RadixPlan &p) {
    int c = 0;
    for (int i = 0; i < p.S; ++i) c += p.R[i] == 16;
    return c;
}

template <int N, int TC, int THR = 0> struct TcPassCfg {
    using Cfg = PassCfg<float, N, TC, THR>;
    static constexpr int LAND = Cfg::LINES * N;  // complex64 per landing buffer
    static constexpr size_t HEAD = 128;          // the landing buffer's mbarrier, padded
    // + a second set of line offsets and tile coordinates (the next tile's are
    // written while the current tile is still being stored)
    static constexpr int COORDS = Cfg::LINES + 4;  // int64 per set
    static constexpr size_t SMEM = HEAD + (size_t)LAND * sizeof(float2) + Cfg::SMEM + COORDS * sizeof(int64_t);
    // CTAs per SM the register allocation must allow: about 768 threads (24
    // warps); without a bound the compiler picked a register cap that spilled
    // hundreds of bytes per thread for some lengths
    static constexpr int MIN_BLOCKS = 768 / Cfg::THREADS > 1 ? 768 / Cfg::THREADS : 1;
    // shared memory per SM (228 KiB, 1 KiB of it reserved per CTA) and per CTA (227 KiB)
    static constexpr int MAX_RESIDENT = (int)(233472 / (SMEM + 1024));
    static_assert(SMEM <= 232448, "tile does not fit one CTA's shared memory");
    // the TMEM columns of all CTAs of one launch that can share an SM fit its
    // 512 columns, so within one launch tcgen05.alloc never waits.  Tensor-core
    // kernels of different launches running at once (two plans on two
    // streams) can share an SM; a CTA's tcgen05.alloc then waits until the
    // other kernel's CTAs on that SM free their columns at their end (a
    // stall, not a deadlock: no CTA waits on another kernel)
    static_assert(TcGeom<Cfg::THREADS>::COLS * MAX_RESIDENT <= 512, "TMEM columns of the resident CTAs");
};

template <int N, int TC, int THR = 0>
__global__ void __launch_bounds__(PassCfg<float, N, TC, THR>::THREADS, TcPassCfg<N, TC, THR>::MIN_BLOCKS)
    fft_pass_tc_kernel(const PassArgs a) {
    using Cfg = PassCfg<float, N, TC, THR>;
    using P = TcPassCfg<N, TC, THR>;
    using C = float2;
    using St = Stages<float, N, 0, 1, TC, THR>;
    static_assert(N % 2 == 0, "bulk copies need lines of whole 16-byte units");
    constexpr uint32_t kParStep = tc_stage_count(Cfg::plan) & 1;  // MMA mbarrier phases per tile, mod 2
    extern __shared__ __align__(128) unsigned char tc_smem[];
    uint64_t *lbar = reinterpret_cast<uint64_t *>(tc_smem);
    C *land = reinterpret_cast<C *>(tc_smem + P::HEAD);
    C *buf = land + P::LAND;  // stage buffer / tensor-core operand rows / transposed tile
    C *tw = buf + Cfg::DATA;
    TcShared *ts = reinterpret_cast<TcShared *>(tw + Cfg::TWN);
    int64_t *coords = reinterpret_cast<int64_t *>(tw + Cfg::TWN + Cfg::BFRAG);  // 2 sets: line offsets, tile
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t G = gridDim.x;
    const C *gtw = reinterpret_cast<const C *>(a.tw);

    for (int q = tid; q < tw_entries(Cfg::plan); q += Cfg::THREADS) tw[q] = gtw[q];
    tc_begin<TC, Cfg::THREADS>(ts, tid);
    if (tid == 0) {
        mbar_init(lbar, 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    tc_fence_after();
    if (tid < 32 && (int64_t)blockIdx.x < a.ntiles) pipe_issue<N, Cfg::LINES>(a, blockIdx.x, land, lbar, lane);

    const int line = tid / Cfg::TL, tl = tid % Cfg::TL;  // line < LINES: THREADS = TL x LINES
    int fbg, fbh;
    tile_line(a, line, fbg, fbh);
    uint32_t par = 0, lpar = 0;
    for (int64_t t = blockIdx.x; t < a.ntiles; t += G, lpar ^= 1) {
        int64_t *lbase = coords + lpar * P::COORDS;  // input offset of each tile line
        TileCoord *shc = reinterpret_cast<TileCoord *>(lbase + Cfg::LINES);
        if (tid < 32) {
            const TileCoord w0 = tile_coords(a, t);
            if (tid == 0) *shc = w0;
            for (int l = tid; l < Cfg::LINES; l += 32) {
                int bg, bh;
                tile_line(a, l, bg, bh);
                lbase[l] = w0.in_base + bg * a.in_sg + bh * a.in_sh;
            }
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(lbar, lpar, kTcWaitNs))) {
                mbar_wait_bounded(lbar, lpar, kTcWaitNs);  // a second bounded chance for the copy to land
                if (tid == 0) ts->failed = 1;
            }
        }
        __syncthreads();
        if (ts->failed) break;  // uniform: set before the barrier
        tc_fence_after();
        const TileCoord c = *shc;
        const bool fok = line < a.Bg * a.Bh && c.g0 + fbg < a.Ng && c.h0 + fbh < a.Nh;
        auto refill = [&]() {  // the first stage has read the landing buffer
            if (tid < 32 && t + G < a.ntiles) pipe_issue<N, Cfg::LINES>(a, t + G, land, lbar, lane);
        };
        St::run(buf, buf, tw, land + (size_t)line * N, line, tl, fok, (a.conj & 1) != 0, true, refill, par);
        if (ts->failed) {  // uniform: set before a barrier; let the refill land (bounded) before leaving
            if (tid < 32 && t + G < a.ntiles) mbar_wait_bounded(lbar, lpar ^ 1, kTcWaitNs);
            break;
        }
        store_tile<float, N, TC, THR>(a, buf, lbase, c, tid);
        par ^= kParStep;
        // no barrier: the next tile's coordinates go to the other set, and its
        // first stage writes the tile region only after the next loop-top barrier
    }
    tc_end<Cfg::THREADS>(ts, tid, a.err);
}

}  // namespace mdfft
