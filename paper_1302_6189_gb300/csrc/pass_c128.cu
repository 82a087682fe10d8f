// pass_c128.cu -- instantiations of the fused pass kernel for complex128 (FP64 arithmetic).
#include "passes.h"

namespace mdfft {

template <int N> static PassKernel make_c128() {
    using Cfg = PassCfg<double, N>;
    return PassKernel{(const void *)&fft_pass_kernel<double, N>, Cfg::THREADS, Cfg::LINES, Cfg::TL, Cfg::SMEM, Cfg::plan};
}

bool find_pass_kernel_c128(int64_t n, PassKernel *k) {
    switch (n) {
#define MDFFT_CASE(N) \
    case N:           \
        *k = make_c128<N>(); \
        return true;
        MDFFT_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
