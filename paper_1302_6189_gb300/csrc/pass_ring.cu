// pass_ring.cu -- instantiations of the persistent complex64 pass kernel that
// streams tiles through a ring of shared-memory slots (fft_ring.cuh): the
// autotuner's variants for short lines, S slots and a cap of resident CTAs
// per SM.
#include "fft_ring.cuh"
#include "passes.h"

namespace mdfft {

template <int N, int S, int RP> static PassKernel make_ring(int per_sm) {
    using Cfg = PassCfg<float, N, 0, 0, RP>;
    PassKernel k{(const void *)&fft_pass_ring_kernel<N, S, RP>, Cfg::THREADS, Cfg::LINES, Cfg::TL,
                 RingCfg<N, S, RP>::SMEM, Cfg::plan};
    k.persistent = S;
    k.bulk = 1;  // 16-byte copies from line starts: input and output 16-byte aligned
    k.per_sm = per_sm;
    return k;
}

bool find_pass_kernel_ring(int64_t n, int slots, int per_sm, int rp, PassKernel *k) {
    if ((slots != 2 && slots != 3) || per_sm < 1 || per_sm > 8) return false;
    if (rp == 1) {
        if (n != 64) return false;
        *k = slots == 2 ? make_ring<64, 2, 1>(per_sm) : make_ring<64, 3, 1>(per_sm);
        return true;
    }
    if (rp != 0) return false;
    switch (n) {
#define MDFFT_CASE(N)                                                               \
    case N:                                                                         \
        *k = slots == 2 ? make_ring<N, 2, 0>(per_sm) : make_ring<N, 3, 0>(per_sm); \
        return true;
        MDFFT_RING_LENGTHS(MDFFT_CASE)
#undef MDFFT_CASE
        default:
            return false;
    }
}

}  // namespace mdfft
