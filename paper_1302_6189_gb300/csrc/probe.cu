// probe.cu -- data movement of a pass without the FFT (mdfft_pattern_probe
// with the default kernel's structure, mdfft_movement_probe with the ring
// kernel's), and the device's FP64 multiply-add rate (mdfft_fp64_rate_probe).
//
// The same tile as the pass kernel with the butterflies left out: each line
// is read into registers exactly as the first stage reads it (every thread
// its elements of the line, all loads issued before any store), put into
// the transposed tile, and written by the same store role.  It moves exactly
// the bytes of a pass in the same pattern, so its speed is the bound that
// pattern puts on the pass.
#include "fft_ring.cuh"
#include "plan_internal.h"

namespace mdfft {

template <int N>
__global__ void __launch_bounds__(PassCfg<float, N, 0, 0>::THREADS) move_pass_kernel(const PassArgs a) {
    using Cfg = PassCfg<float, N, 0, 0>;
    using C = float2;
    constexpr int PER = (N + Cfg::TL - 1) / Cfg::TL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    int64_t *lbase = reinterpret_cast<int64_t *>(buf + Cfg::DATA + Cfg::TWN + Cfg::BFRAG);
    const int tid = threadIdx.x;
    const C *in = reinterpret_cast<const C *>(a.in);
    const TileCoord c = tile_coords(a, blockIdx.x);
    if (tid < Cfg::LINES) {
        int bg, bh;
        tile_line(a, tid, bg, bh);
        lbase[tid] = c.in_base + bg * a.in_sg + bh * a.in_sh;
    }
    __syncthreads();
    const int line = tid / Cfg::TL, tl = tid % Cfg::TL;
    int fbg, fbh;
    tile_line(a, line, fbg, fbh);
    if (line < a.Bg * a.Bh && c.g0 + fbg < a.Ng && c.h0 + fbh < a.Nh) {
        const C *src = in + lbase[line];
        C v[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int k = tl + i * Cfg::TL;
            v[i] = (N % Cfg::TL == 0 || k < N) ? __ldg(src + k) : C{0, 0};
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int k = tl + i * Cfg::TL;
            if (N % Cfg::TL == 0 || k < N) buf[k * Cfg::TROW + line] = v[i];
        }
    }
    __syncthreads();
    store_tile<float, N, 0, 0>(a, buf, lbase, c, tid);
}

template <int N> static PassKernel make_move() {
    using Cfg = PassCfg<float, N, 0, 0>;
    return PassKernel{(const void *)&move_pass_kernel<N>, Cfg::THREADS, Cfg::LINES, Cfg::TL, Cfg::SMEM, Cfg::plan};
}

bool find_move_kernel_c64(int64_t n, PassKernel *k) {
    switch (n) {
#define MDFFT_CASE(N)        \
    case N:                  \
        *k = make_move<N>(); \
        return true;
        MDFFT_TUNED_LENGTHS(MDFFT_CASE) MDFFT_CASE(24)
#undef MDFFT_CASE
        default:
            return false;
    }
}

// The ring kernel's data movement without the butterflies: a persistent CTA
// streams its tiles through S slots filled by 16-byte cp.async copies (the
// same slots, commit groups and barriers as fft_pass_ring_kernel); each
// thread copies its line from the slot into the transposed tile, and the
// store role writes it to the next layout.  Its bandwidth is the bound the
// pass's access pattern puts on a kernel that keeps S - 1 tiles' loads in
// flight per CTA.
template <int N, int S>
__global__ void __launch_bounds__(PassCfg<float, N>::THREADS) move_ring_kernel(const PassArgs a) {
    using Cfg = PassCfg<float, N>;
    using RC = RingCfg<N, S, 0>;
    using C = float2;
    constexpr int PER = (N + Cfg::TL - 1) / Cfg::TL;
    extern __shared__ __align__(16) unsigned char mr_smem[];
    C *slots = reinterpret_cast<C *>(mr_smem);
    C *tile = slots + S * RC::SLOT + Cfg::DATA;
    int64_t *meta = reinterpret_cast<int64_t *>(tile + RC::TILE + Cfg::TWN);
    const int tid = threadIdx.x;
    const int line = tid / Cfg::TL, tl = tid % Cfg::TL;
    int bg, bh;
    tile_line(a, line, bg, bh);
    const bool lok = line < a.Bg * a.Bh;
    const int64_t loff = (int64_t)bg * a.in_sg + (int64_t)bh * a.in_sh;
    const C *in = reinterpret_cast<const C *>(a.in);
    const int64_t G = gridDim.x;
    auto issue = [&](int64_t t, int slot, int e) {
        if (t < a.ntiles) {
            const TileCoord c = tile_coords(a, t);
            if (tid == 0) *reinterpret_cast<TileCoord *>(meta + e * RC::META) = c;
            if (lok && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh) {
                const C *src = in + c.in_base + loff;
                C *dst = slots + slot * RC::SLOT + line * RC::RS;
#pragma unroll
                for (int i = 0; i < RC::CPT; ++i) {
                    const int u = tl + i * Cfg::TL;
                    if (RC::CH % Cfg::TL == 0 || u < RC::CH) ring_copy16(dst + 2 * u, src + 2 * u);
                }
            }
        }
        ring_commit();
    };
#pragma unroll
    for (int s = 0; s < S - 1; ++s) issue(blockIdx.x + s * G, s, s);
    int slot = 0, e = 0;
    for (int64_t t = blockIdx.x; t < a.ntiles; t += G) {
        issue(t + (S - 1) * G, slot == 0 ? S - 1 : slot - 1, (e + S - 1) % (S + 1));
        ring_wait<S - 1>();
        __syncthreads();
        const TileCoord c = *reinterpret_cast<const TileCoord *>(meta + e * RC::META);
        if (lok && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh) {
            const C *src = slots + slot * RC::SLOT + line * RC::RS;
            C v[PER];
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int k = tl + j * Cfg::TL;
                v[j] = (N % Cfg::TL == 0 || k < N) ? src[k] : C{0, 0};
            }
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int k = tl + j * Cfg::TL;
                if (N % Cfg::TL == 0 || k < N) tile[k * Cfg::TROW + line] = v[j];
            }
        }
        __syncthreads();
        store_tile<float, N, 0, 0>(a, tile, nullptr, c, tid);
        slot = slot + 1 == S ? 0 : slot + 1;
        e = e == S ? 0 : e + 1;
    }
    ring_wait<0>();
}

template <int N, int S> static PassKernel make_move_ring() {
    using Cfg = PassCfg<float, N>;
    PassKernel k{(const void *)&move_ring_kernel<N, S>, Cfg::THREADS, Cfg::LINES, Cfg::TL, RingCfg<N, S, 0>::SMEM,
                 Cfg::plan};
    k.persistent = S;
    k.bulk = 1;
    return k;
}

bool find_move_ring_kernel_c64(int64_t n, int slots, PassKernel *k) {
    if (slots != 2 && slots != 3) return false;
    switch (n) {
#define MDFFT_CASE(N)                                                         \
    case N:                                                                   \
        *k = slots == 2 ? make_move_ring<N, 2>() : make_move_ring<N, 3>();    \
        return true;
        MDFFT_RING_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft

namespace {

// 8 independent multiply-add chains per thread: enough independent work per
// warp to keep the FP64 pipe busy whatever its latency.
__global__ void __launch_bounds__(256) dfma_rate_kernel(double *out, int64_t iters) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double m = 0.999999999, c = 1e-9 * (double)(threadIdx.x & 7);
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 1.0 + 1e-3 * (double)i + 1e-12 * (double)gid;
    for (int64_t it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = fma(v[i], m, c);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += v[i];
    out[gid] = s;
}

}  // namespace

extern "C" mdfft_status mdfft_fp64_rate_probe(double *out, int ctas, int64_t iters, mdfft_stream_t stream,
                                              double *tflops) {
    if (!out || !tflops) return mdfft::detail::fail(MDFFT_E_ARG, "null argument");
    if (ctas < 1 || ctas > (1 << 20) || iters < 1 || iters > (1 << 24))
        return mdfft::detail::fail(MDFFT_E_ARG, "ctas must be in [1, 2^20] and iters in [1, 2^24]");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return mdfft::detail::fail(MDFFT_E_CUDA, "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return mdfft::detail::fail(MDFFT_E_CUDA, "cudaEventCreate");
    }
    dfma_rate_kernel<<<ctas, 256, 0, st>>>(out, iters < 64 ? iters : 64);  // warm-up
    cudaEventRecord(e0, st);
    dfma_rate_kernel<<<ctas, 256, 0, st>>>(out, iters);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return mdfft::detail::cuda_fail(e, "FP64 rate probe");
    *tflops = 2.0 * 8.0 * 256.0 * (double)ctas * (double)iters / ((double)ms * 1e-3) / 1e12;
    return MDFFT_OK;
}
