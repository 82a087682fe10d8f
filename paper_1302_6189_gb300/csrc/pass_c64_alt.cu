// pass_c64_alt.cu -- complex64 pass kernels with the alternative radix plan
// (radix_plan_alt in fft_pass.cuh: e.g. 256 = 8x8x4 instead of 16x16, 512 =
// 8x8x8 instead of 16x16x2) and the default CTA shape rule, for the common
// line lengths: the autotuner's radix-split alternatives.  A pass run with
// one needs the twiddle table of that plan (the plan regenerates it).
#include "passes.h"

namespace mdfft {

template <int N> static PassKernel make_c64_alt() {
    using Cfg = PassCfg<float, N, 0, 0, 1>;
    return PassKernel{(const void *)&fft_pass_kernel<float, N, 0, 0, 1>, Cfg::THREADS, Cfg::LINES, Cfg::TL, Cfg::SMEM,
                      Cfg::plan};
}

bool find_pass_kernel_c64_alt(int64_t n, PassKernel *k) {
    switch (n) {
#define MDFFT_CASE(N)            \
    case N:                      \
        *k = make_c64_alt<N>();  \
        return true;
        MDFFT_TUNED_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
