// pass_tc.cu -- instantiations of the persistent pass kernel with tensor-core radix-16
// stages (complex64 data; split hi/lo FP16 or BF16 operands, FP32 accumulation).
#include "passes.h"
#include "tc_group.cuh"
#include "tc_pass.cuh"

namespace mdfft {

template <int N, int TC, int THR = 0> static PassKernel make_tc() {
    using Cfg = PassCfg<float, N, TC, THR>;
    PassKernel k{(const void *)&fft_pass_tc_kernel<N, TC, THR>, Cfg::THREADS, Cfg::LINES, Cfg::TL,
                 TcPassCfg<N, TC, THR>::SMEM, Cfg::plan};
    k.persistent = 1;
    k.bulk = 1;
    return k;
}

bool find_pass_kernel_tc(int64_t n, int tc, PassKernel *k) {
    if (tc != kTcFp16 && tc != kTcBf16) return false;
    switch (n) {
#define MDFFT_CASE(N)                                                     \
    case N:                                                               \
        *k = tc == kTcFp16 ? make_tc<N, kTcFp16>() : make_tc<N, kTcBf16>(); \
        return true;
        MDFFT_TC_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

// the tensor-core kernel with independent 128-thread groups (tc_group.cuh): the
// host sees tiles of one group (128 / (N / 16) lines) and one persistent wave
template <int N, int TC, bool LAND> static PassKernel make_tcg() {
    using K = TcgCfg<N, TC, LAND>;
    PassKernel k{(const void *)&fft_pass_tcg_kernel<N, TC, LAND>, K::THREADS, K::LPG, K::NB, K::SMEM, K::plan};
    k.persistent = 1;
    k.bulk = LAND ? 1 : 0;  // bulk copies need 16-byte aligned lines
    return k;
}

bool find_pass_kernel_tcg(int64_t n, int tc, bool land, PassKernel *k) {
    if (tc != kTcFp16 && tc != kTcBf16) return false;
    switch (n) {
#define MDFFT_CASE(N)                                                                                    \
    case N:                                                                                              \
        *k = tc == kTcFp16 ? (land ? make_tcg<N, kTcFp16, true>() : make_tcg<N, kTcFp16, false>())       \
                           : (land ? make_tcg<N, kTcBf16, true>() : make_tcg<N, kTcBf16, false>());      \
        return true;
        MDFFT_CASE(256) MDFFT_CASE(512)
#undef MDFFT_CASE
        default:
            return false;
    }
}

// 128-thread tensor-core CTAs (half the lines per tile, twice the CTAs per SM),
// an autotuning variant for the lengths of the precision and 256^3 configurations
bool find_pass_kernel_tc_thr(int64_t n, int tc, int thr, PassKernel *k) {
    if ((tc != kTcFp16 && tc != kTcBf16) || thr != 128) return false;
    switch (n) {
#define MDFFT_CASE(N)                                                                      \
    case N:                                                                                \
        *k = tc == kTcFp16 ? make_tc<N, kTcFp16, 128>() : make_tc<N, kTcBf16, 128>(); \
        return true;
        MDFFT_CASE(128) MDFFT_CASE(256) MDFFT_CASE(512)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
