// pass_c64_tuned.cu -- complex64 pass kernels with a fixed CTA size (256 or 512
// threads) for the common line lengths, and 192 or 384 threads (48 or 96
// lines of 4 threads) for 24 and 48: the autotuner's alternatives to the
// default launch shape of pass_c64.cu.  (48 and 96 lines tile axes whose
// extent is a multiple of 3, e.g. 24 x 2 lines, without idle lines.)
#include "fft_prefetch.cuh"
#include "passes.h"

namespace mdfft {

template <int N, int THR> static PassKernel make_c64_thr() {
    using Cfg = PassCfg<float, N, 0, THR>;
    return PassKernel{(const void *)&fft_pass_kernel<float, N, 0, THR>, Cfg::THREADS, Cfg::LINES, Cfg::TL, Cfg::SMEM,
                      Cfg::plan};
}

bool find_pass_kernel_c64_thr(int64_t n, int thr, PassKernel *k) {
    if (thr == 192 || thr == 384) {
        switch (n) {
#define MDFFT_CASE(N)                                                      \
    case N:                                                                \
        *k = thr == 192 ? make_c64_thr<N, 192>() : make_c64_thr<N, 384>(); \
        return true;
            MDFFT_CASE(24) MDFFT_CASE(48)
#undef MDFFT_CASE
            default:
                return false;
        }
    }
    if (thr != 256 && thr != 512) return false;
    switch (n) {
#define MDFFT_CASE(N)                                                           \
    case N:                                                                     \
        *k = thr == 256 ? make_c64_thr<N, 256>() : make_c64_thr<N, 512>();      \
        return true;
        MDFFT_TUNED_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

// Persistent kernel with the next tile's first-stage loads in registers
// (fft_prefetch.cuh), for short lines; rp selects the radix plan.
template <int N, int RP, int MINB> static PassKernel make_pf() {
    using Cfg = PassCfg<float, N, 0, 0, RP>;
    PassKernel k{(const void *)&fft_pass_pf_kernel<N, RP, MINB>, Cfg::THREADS, Cfg::LINES, Cfg::TL,
                 PfCfg<N, RP>::SMEM, Cfg::plan};
    k.persistent = 1;
    return k;
}

bool find_pass_kernel_c64_pf(int64_t n, int rp, int minb, PassKernel *k) {
    if (minb != 2 && minb != 4) return false;
    if (rp == 1) {
        if (n != 64) return false;
        *k = minb == 2 ? make_pf<64, 1, 2>() : make_pf<64, 1, 4>();
        return true;
    }
    switch (n) {
#define MDFFT_CASE(N)                                               \
    case N:                                                         \
        *k = minb == 2 ? make_pf<N, 0, 2>() : make_pf<N, 0, 4>();   \
        return true;
        MDFFT_CASE(24) MDFFT_CASE(32) MDFFT_CASE(48) MDFFT_CASE(64)
#undef MDFFT_CASE
        default:
            return false;
    }
}

bool find_pass_kernel_c64_shfl(int64_t n, PassKernel *k) {
    if (n != 256) return false;
    using Cfg = PassCfg<float, 256>;
    *k = PassKernel{(const void *)&fft_pass_shfl256_kernel, Cfg::THREADS, Cfg::LINES, Cfg::TL, Cfg::SMEM, Cfg::plan};
    return true;
}

// The default launch shape with a register cap for 6 CTAs per SM (short
// lines; a few registers spill), an autotuning variant.
bool find_pass_kernel_c64_occ(int64_t n, PassKernel *k) {
    switch (n) {
#define MDFFT_CASE(N)                                                                                       \
    case N:                                                                                                 \
        *k = PassKernel{(const void *)&fft_pass_occ_kernel<N, 6>, PassCfg<float, N>::THREADS,               \
                        PassCfg<float, N>::LINES, PassCfg<float, N>::TL, PassCfg<float, N>::SMEM, PassCfg<float, N>::plan}; \
        return true;
        MDFFT_CASE(24) MDFFT_CASE(32) MDFFT_CASE(48) MDFFT_CASE(64)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
