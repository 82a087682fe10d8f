// probe.cu -- data movement of a pass without the FFT (mdfft_pattern_probe).
//
// The same tile as the pass kernel with the butterflies left out: each line
// is read into registers exactly as the first stage reads it (every thread
// its elements of the line, all loads issued before any store), put into
// the transposed tile, and written by the same store role.  It moves exactly
// the bytes of a pass in the same pattern, so its speed is the bound that
// pattern puts on the pass.
#include "passes.h"

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
        const int bg = tid % a.Bg, bh = tid / a.Bg;
        lbase[tid] = c.in_base + bg * a.in_sg + bh * a.in_sh;
    }
    __syncthreads();
    const int line = tid / Cfg::TL, tl = tid % Cfg::TL;
    const int fbg = line % a.Bg, fbh = line / a.Bg;
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
        MDFFT_TUNED_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
