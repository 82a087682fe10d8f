// pass_pipe.cu -- instantiations of the persistent, bulk-copy pipelined pass kernel (complex64).
#include "fft_pipe.cuh"
#include "passes.h"

namespace mdfft {

template <int N, int NBUF> static PassKernel make_pipe() {
    using Cfg = PassCfg<float, N, 0, 0>;
    PassKernel k{(const void *)&fft_pass_pipe_kernel<N, NBUF>, Cfg::THREADS, Cfg::LINES, Cfg::TL,
                 PipeCfg<N, NBUF>::SMEM, Cfg::plan};
    k.persistent = NBUF;
    return k;
}

bool find_pass_kernel_pipe(int64_t n, int nbuf, PassKernel *k) {
    if (nbuf != 1 && nbuf != 2) return false;
    switch (n) {
#define MDFFT_CASE(N)                                                \
    case N:                                                          \
        *k = nbuf == 1 ? make_pipe<N, 1>() : make_pipe<N, 2>(); \
        return true;
        MDFFT_PIPE_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
