// pass_c64.cu -- instantiations of the fused pass kernel for complex64 (FP32 arithmetic).
#include "passes.h"

namespace mdfft {

template <int N> static PassKernel make_c64() {
    using Cfg = PassCfg<float, N>;
    return PassKernel{(const void *)&fft_pass_kernel<float, N>, Cfg::THREADS, Cfg::LINES, Cfg::TL, Cfg::SMEM, Cfg::plan};
}

bool find_pass_kernel_c64(int64_t n, PassKernel *k) {
    switch (n) {
#define MDFFT_CASE(N) \
    case N:           \
        *k = make_c64<N>(); \
        return true;
        MDFFT_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
