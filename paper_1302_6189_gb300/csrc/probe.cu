// probe.cu -- data movement of a pass without the FFT (mdfft_pattern_probe),
// and the device's FP64 multiply-add rate (mdfft_fp64_rate_probe).
//
// The same tile as the pass kernel with the butterflies left out: each line
// is read into registers exactly as the first stage reads it (every thread
// its elements of the line, all loads issued before any store), put into
// the transposed tile, and written by the same store role.  It moves exactly
// the bytes of a pass in the same pattern, so its speed is the bound that
// pattern puts on the pass.
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
