// pass_pipe.cu -- instantiations of the persistent, bulk-copy pipelined pass kernel (complex64).
#include "fft_pipe.cuh"
#include "passes.h"
#include "plan_internal.h"

#include <chrono>

namespace mdfft {

template <int N, int NBUF> static PassKernel make_pipe() {
    using Cfg = PassCfg<float, N, 0, 0>;
    PassKernel k{(const void *)&fft_pass_pipe_kernel<N, NBUF>, Cfg::THREADS, Cfg::LINES, Cfg::TL,
                 PipeCfg<N, NBUF>::SMEM, Cfg::plan};
    k.persistent = NBUF;
    k.bulk = 1;
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

namespace {

// The bounded mbarrier wait of the pipelined kernel on its own: one thread
// arms a barrier for 16 bytes that no copy will bring (arrive = 0), or arrives
// plainly (arrive = 1, the phase completes), and waits at most limit_ns.
// *status: 1 the phase completed, 2 the wait gave up.
__global__ void wait_selftest_kernel(int arrive, uint64_t limit_ns, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mdfft::mbar_init(&bar, 1);
    mdfft::fence_mbarrier_init();
    if (arrive)
        mdfft::mbar_arrive(&bar);
    else
        mdfft::mbar_arrive_expect_tx(&bar, 16);
    *status = mdfft::mbar_wait_bounded(&bar, 0, limit_ns) ? 1 : 2;
}

}  // namespace

extern "C" mdfft_status mdfft_selftest_wait(int arrive, int64_t limit_us, int64_t *waited_us) {
    using mdfft::detail::cuda_fail;
    using mdfft::detail::fail;
    if (limit_us < 1 || limit_us > 10000000) return fail(MDFFT_E_ARG, "limit_us must be in [1, 10^7]");
    int *status = nullptr;
    cudaError_t e = cudaMalloc(&status, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    cudaMemset(status, 0, sizeof(int));
    const auto t0 = std::chrono::steady_clock::now();
    wait_selftest_kernel<<<1, 32>>>(arrive != 0, (uint64_t)limit_us * 1000ull, status);
    int host = 0;
    e = cudaMemcpy(&host, status, sizeof(int), cudaMemcpyDeviceToHost);  // waits for the kernel
    const auto t1 = std::chrono::steady_clock::now();
    cudaFree(status);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    if (waited_us) *waited_us = std::chrono::duration_cast<std::chrono::microseconds>(t1 - t0).count();
    if (host == 2) return fail(MDFFT_E_TIMEOUT, "the bounded device wait gave up (as the self-test intends)");
    if (host != 1) return fail(MDFFT_E_CUDA, "wait self-test did not report");
    return MDFFT_OK;
}
