// pass_line.cu -- instantiations of the one-thread-per-line complex64 pass
// kernel (fft_line.cuh): an autotuning variant for short even lengths.
#include "fft_line.cuh"
#include "passes.h"

namespace mdfft {

template <int N> static PassKernel make_line() {
    using LC = LineCfg<N>;
    PassKernel k{(const void *)&fft_pass_line_kernel<N>, LC::THREADS, LC::LINES, 1, LC::SMEM, LC::plan};
    k.bulk = 1;  // 16-byte copies from line starts: input and output 16-byte aligned
    return k;
}

bool find_pass_kernel_line(int64_t n, PassKernel *k) {
    switch (n) {
#define MDFFT_CASE(N)         \
    case N:                   \
        *k = make_line<N>();  \
        return true;
        MDFFT_LINE_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
