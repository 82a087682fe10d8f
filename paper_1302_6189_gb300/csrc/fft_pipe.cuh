// fft_pipe.cuh -- persistent pass kernel with a bulk-copy (TMA) load pipeline.
//
// Same pass as fft_pass_kernel (Fig. 4 step + the transpose after it), but
// each CTA walks tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... and keeps
// the input of the next tiles in flight while it computes and stores the
// current one.  One or two landing buffers in shared memory take a tile's
// lines unpadded; warp 0 fills them with one cp.async.bulk (1-D TMA) copy per
// line, completing on the buffer's mbarrier with the tile's byte count.  A
// tile is consumed by the first Stockham stage straight from its landing
// buffer, which is refilled right after that stage with the tile NBUF steps
// ahead, while the rest of the FFT and the store of the current tile run.
//
// Waits on an mbarrier are bounded (2 s of %globaltimer); a CTA whose wait
// gives up sets *err, waits (bounded) for its other copies, and exits with
// the whole CTA; the host reports MDFFT_E_TIMEOUT.
//
// Requirements (checked on the host): complex64, even N (lines are whole
// 16-byte units), input 16-byte aligned.
#pragma once

#include "fft_pass.cuh"
#include "ptx_sync.cuh"

namespace mdfft {

template <int N, int NBUF> struct PipeCfg {
    using Cfg = PassCfg<float, N, 0, 0>;
    static_assert(N % 2 == 0, "bulk copies need lines of whole 16-byte units");
    static_assert(NBUF == 1 || NBUF == 2, "one or two landing buffers");
    static constexpr int LAND = Cfg::LINES * N;  // complex64 per landing buffer
    static constexpr size_t HEAD = 128;          // the mbarriers, padded
    static constexpr size_t SMEM = HEAD + NBUF * (size_t)LAND * sizeof(float2) + Cfg::SMEM;
    static constexpr uint64_t kWaitLimitNs = 2000000000ull;
};

// Warp 0: arm barrier b with the byte count of tile t and copy its valid
// lines (a tile of LINES lines of N complex64).
template <int N, int LINES = PassCfg<float, N, 0, 0>::LINES>
__device__ __forceinline__ void pipe_issue(const PassArgs &a, int64_t t, float2 *land, uint64_t *bar, int lane) {
    const TileCoord c = tile_coords(a, t);
    const int64_t vg = a.Ng - c.g0 < a.Bg ? a.Ng - c.g0 : a.Bg;
    const int64_t vh = a.Nh - c.h0 < a.Bh ? a.Nh - c.h0 : a.Bh;
    if (lane == 0) {
        fence_proxy_async_shared();  // earlier generic reads of this buffer before the async writes
        mbar_arrive_expect_tx(bar, (uint32_t)(vg * vh * N * sizeof(float2)));
    }
    __syncwarp();
    const float2 *in = reinterpret_cast<const float2 *>(a.in);
    for (int l = lane; l < LINES; l += 32) {
        int bg, bh;
        tile_line(a, l, bg, bh);
        if (l < a.Bg * a.Bh && bg < vg && bh < vh)
            bulk_copy_g2s(land + (size_t)l * N, in + c.in_base + bg * a.in_sg + bh * a.in_sh,
                          (uint32_t)(N * sizeof(float2)), bar);
    }
}

// NBUF landing buffers: tile k of this CTA lands in buffer k % NBUF; right
// after the first stage has read it, that buffer is refilled with tile
// k + NBUF, so the copy overlaps the rest of tile k (and, with two buffers,
// all of tile k + 1).
template <int N, int NBUF>
__global__ void __launch_bounds__(PassCfg<float, N, 0, 0>::THREADS) fft_pass_pipe_kernel(const PassArgs a) {
    using Cfg = PassCfg<float, N, 0, 0>;
    using P = PipeCfg<N, NBUF>;
    using C = float2;
    extern __shared__ __align__(128) unsigned char pipe_smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(pipe_smem);
    C *land = reinterpret_cast<C *>(pipe_smem + P::HEAD);
    unsigned char *work = pipe_smem + P::HEAD + NBUF * (size_t)P::LAND * sizeof(C);
    C *buf = reinterpret_cast<C *>(work);
    C *tw = buf + Cfg::DATA;
    int64_t *lbase = reinterpret_cast<int64_t *>(tw + Cfg::TWN + Cfg::BFRAG);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t G = gridDim.x, ntiles = a.ntiles;

    const C *gtw = reinterpret_cast<const C *>(a.tw);
    for (int q = tid; q < tw_entries(Cfg::plan); q += Cfg::THREADS) tw[q] = gtw[q];
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&bar[b], 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    if (warp == 0)
        for (int b = 0; b < NBUF; ++b)
            if ((int64_t)blockIdx.x + b * G < ntiles)
                pipe_issue<N>(a, blockIdx.x + b * G, land + (size_t)b * P::LAND, &bar[b], lane);

    const int line = tid / Cfg::TL, tl = tid % Cfg::TL;
    int fbg, fbh;
    tile_line(a, line, fbg, fbh);
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += G, ++k) {
        const int b = (int)(k % NBUF);
        const uint32_t parity = (uint32_t)((k / NBUF) & 1);
        const TileCoord c = tile_coords(a, t);
        if (tid < Cfg::LINES) {
            int bg, bh;
            tile_line(a, tid, bg, bh);
            lbase[tid] = c.in_base + bg * a.in_sg + bh * a.in_sh;
        }
        const bool ok = mbar_wait_bounded(&bar[b], parity, P::kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.err) atomicExch(a.err, 1);
            // the other buffers may still be filling: give their copies a bounded chance to land
            for (int o = 1; o < NBUF; ++o)
                if (t + o * G < ntiles)
                    mbar_wait_bounded(&bar[(k + o) % NBUF], (uint32_t)(((k + o) / NBUF) & 1), P::kWaitLimitNs);
            return;
        }
        const bool fok = line < a.Bg * a.Bh && c.g0 + fbg < a.Ng && c.h0 + fbh < a.Nh;
        C *mine = land + (size_t)b * P::LAND;
        auto refill = [&]() {  // buffer b has been read by the first stage
            if (warp == 0 && t + NBUF * G < ntiles) pipe_issue<N>(a, t + NBUF * G, mine, &bar[b], lane);
        };
        Stages<float, N, 0, 1, 0, 0, 2>::run(buf, buf, tw, mine + (size_t)line * N, line, tl, fok, (a.conj & 1) != 0, true,
                                             refill);
        store_tile<float, N, 0, 0>(a, buf, lbase, c, tid);
        __syncthreads();  // the tile region and lbase are rewritten by the next tile
    }
}

}  // namespace mdfft
