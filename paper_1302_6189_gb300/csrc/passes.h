// passes.h -- registry of the compiled pass kernels (one per line length and precision).
#pragma once

#include <cstddef>
#include <cstdint>

#include "fft_pass.cuh"

// Line lengths built into the library: 1 and products of 2, 3 and 5 up to
// 1024 whose radix plan is in fft_pass.cuh.
#define MDFFT_LENGTHS(X)                                                                                   \
    X(1) X(2) X(3) X(4) X(5) X(6) X(8) X(10) X(12) X(15) X(16) X(20) X(24) X(30) X(32) X(40) X(48) X(60) X(64) \
        X(80) X(96) X(120) X(128) X(160) X(192) X(240) X(256) X(320) X(384) X(480) X(512) X(640) X(768)    \
            X(960) X(1024)

// Line lengths with a tensor-core variant (a multiple of 16 in the list above).
#define MDFFT_TC_LENGTHS(X)                                                                                    \
    X(16) X(32) X(48) X(64) X(80) X(96) X(128) X(160) X(192) X(240) X(256) X(320) X(384) X(480) X(512) X(640) \
        X(768) X(960) X(1024)

// Even line lengths with a persistent bulk-copy pipelined variant (two landing
// buffers of a tile fit in shared memory).
#define MDFFT_PIPE_LENGTHS(X) X(16) X(32) X(48) X(64) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512)

// Line lengths with a persistent ring-of-slots variant (fft_ring.cuh).
#define MDFFT_RING_LENGTHS(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(256)

// Even line lengths with a one-thread-per-line variant (fft_line.cuh).
#define MDFFT_LINE_LENGTHS(X) X(8) X(12) X(16) X(20) X(24) X(30) X(32) X(40) X(48) X(60) X(64)

// Line lengths with fixed-CTA-size variants for the autotuner.
#define MDFFT_TUNED_LENGTHS(X) X(32) X(48) X(64) X(96) X(128) X(160) X(192) X(256) X(512)

namespace mdfft {

struct PassKernel {
    const void *fn;  // __global__ fft_pass_kernel<Real, N>
    int threads, lines, tl;
    size_t smem;
    RadixPlan plan;      // radix plan of the kernel; its twiddle table follows tw_offset()
    int persistent = 0;  // > 0: walks tiles with a grid stride (launch at most one wave)
    int bulk = 0;        // 1: loads lines with bulk copies (input and output 16-byte aligned)
    int per_sm = 0;      // persistent kernels: at most this many resident CTAs per SM (0: as many as fit)
};

bool find_pass_kernel_c64(int64_t n, PassKernel *k);
bool find_pass_kernel_c128(int64_t n, PassKernel *k);
bool find_pass_kernel_tc(int64_t n, int tc, PassKernel *k);  // tc: kTcFp16 or kTcBf16
bool find_pass_kernel_tc_thr(int64_t n, int tc, int thr, PassKernel *k);  // thr: 128-thread CTAs
bool find_pass_kernel_tcg(int64_t n, int tc, bool land, PassKernel *k);  // independent 128-thread groups (256, 512)
bool find_pass_kernel_c64_thr(int64_t n, int thr, PassKernel *k);  // thr: 256 or 512 threads; 192 or 384 for 24, 48
bool find_pass_kernel_pipe(int64_t n, int nbuf, PassKernel *k);    // persistent, bulk-copy pipelined
bool find_pass_kernel_c64_alt(int64_t n, PassKernel *k);           // alternative radix plan (radix_plan_alt)
bool find_pass_kernel_c64_occ(int64_t n, PassKernel *k);           // register cap for 6 CTAs per SM (24..64)
bool find_pass_kernel_c64_pf(int64_t n, int rp, int minb, PassKernel *k);  // persistent, next tile's loads in registers
bool find_pass_kernel_c64_shfl(int64_t n, PassKernel *k);          // 256: warp-shuffle exchange between the stages
bool find_pass_kernel_ring(int64_t n, int slots, int per_sm, int rp, PassKernel *k);  // persistent, ring of slots
bool find_pass_kernel_line(int64_t n, int rp, int warps, PassKernel *k);  // one thread per line, stages in registers
bool find_pass_kernel_line2(int64_t n, int rp, PassKernel *k);  // two threads per line (32, 64), one exchange
bool find_move_kernel_c64(int64_t n, PassKernel *k);               // data movement of a pass, no FFT
bool find_move_ring_kernel_c64(int64_t n, int slots, PassKernel *k);  // the same through a ring of slots

}  // namespace mdfft
