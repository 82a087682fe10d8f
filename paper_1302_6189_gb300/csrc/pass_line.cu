// pass_line.cu -- instantiations of the one-thread-per-line complex64 pass
// kernel (fft_line.cuh): an autotuning variant for short even lengths.
#include "fft_line.cuh"
#include "passes.h"

namespace mdfft {

template <int N, int RP, int WARPS> static PassKernel make_line() {
    using LC = LineCfg<N, RP, WARPS>;
    PassKernel k{(const void *)&fft_pass_line_kernel<N, RP, WARPS>, LC::THREADS, LC::LINES, 1, LC::SMEM, LC::plan};
    k.bulk = 1;  // 16-byte copies from line starts: input and output 16-byte aligned
    return k;
}

// rp 0: the default radix plan, 4 or 2 warps per CTA (2: the register-heavy
// lengths 48 to 64, more CTAs per SM); rp 1: the alternative plan of 32 and
// 64 (4 warps)
bool find_pass_kernel_line(int64_t n, int rp, int warps, PassKernel *k) {
    if (rp == 1) {
        if (warps != 4) return false;
        if (n == 32) *k = make_line<32, 1, 4>();
        else if (n == 64) *k = make_line<64, 1, 4>();
        else return false;
        return true;
    }
    if (rp != 0) return false;
    if (warps == 2) {
        switch (n) {
            case 48: *k = make_line<48, 0, 2>(); return true;
            case 60: *k = make_line<60, 0, 2>(); return true;
            case 64: *k = make_line<64, 0, 2>(); return true;
            default: return false;
        }
    }
    if (warps != 4) return false;
    switch (n) {
#define MDFFT_CASE(N)                 \
    case N:                           \
        *k = make_line<N, 0, 4>();    \
        return true;
        MDFFT_LINE_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

// Two threads per line (fft_pass_line2_kernel): 32 and 64, default or alternative radix plan.
template <int N, int RP> static PassKernel make_line2() {
    using L2 = Line2Cfg<N, RP>;
    PassKernel k{(const void *)&fft_pass_line2_kernel<N, RP>, L2::THREADS, L2::LINES, 2, L2::SMEM, L2::plan};
    k.bulk = 1;  // 16-byte copies from line starts: input and output 16-byte aligned
    return k;
}

bool find_pass_kernel_line2(int64_t n, int rp, PassKernel *k) {
    if (rp != 0 && rp != 1) return false;
    if (n == 32) *k = rp ? make_line2<32, 1>() : make_line2<32, 0>();
    else if (n == 64) *k = rp ? make_line2<64, 1>() : make_line2<64, 0>();
    else return false;
    return true;
}

}  // namespace mdfft
