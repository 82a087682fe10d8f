// tc_stage.cuh -- radix-16 Stockham stage as a tcgen05 tensor-core GEMM
// (complex64 data).
//
// A radix-16 stage applies the 16-point DFT (Sec. 2, the 1-D DFT equation)
// to every butterfly of the tile.  Written in real arithmetic, one butterfly
// is a row [Re v_0..Re v_15, Im v_0..Im v_15] (K = 32) and the stage is
//     D[rows x 32] = A[rows x 32] . B^T,   B[n][k] = block form of the DFT-16,
// B = [[C, -S], [S, C]] with C = cos(2 pi r q/16), S = sin(2 pi r q/16),
// giving rows [Re V_0..Re V_15, Im V_0..Im V_15] (forward sign).
//
// Operands are split x = hi + lo in FP16 or BF16 and the three products
// hi.hi + hi.lo + lo.hi are accumulated in FP32 (lo.lo lies below the FP32
// rounding of the sum).  FP16 rows are scaled by an exact power of two so
// that their largest component lies in [2^14, 2^15) before the split; the
// scale is undone on the FP32 results.
//
// Every thread of the CTA owns one butterfly row (the tile has exactly as many
// radix-16 butterflies as the CTA has threads).  Per stage:
//  1. each thread reads its 16 inputs (from the tile's landing buffer in the
//     first stage, else from the stage buffer), twiddles, scales and splits
//     them, and writes its A row (hi and lo) into shared memory in the
//     no-swizzle K-major layout of the tensor cores (8-row x 16-byte core
//     matrices): over the stage buffer in the first stage (its old contents
//     are no longer needed), into the landing buffer (consumed by then) in
//     the later ones;
//  2. one thread issues, per 128-row group, 2 k-steps x 3 products of
//     tcgen05.mma (M = 128, N = 32, K = 16) into a 32-column TMEM
//     accumulator and commits them to an mbarrier;
//  3. warp 0 waits (bounded) on the mbarrier and releases the CTA through a
//     barrier; every warp then reads its 32 TMEM lanes
//     (row = thread) with tcgen05.ld and writes the 16 complex results to the
//     next stage buffer or, in the last stage, to the transposed tile.
// The DFT-16 matrix B (hi and lo) is built once per CTA.  A wait that gives up
// after 2 s marks the CTA failed: it skips its remaining tensor-core work and
// sets the plan's error flag (MDFFT_E_TIMEOUT from mdfft_plan_check).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ptx_sync.cuh"

namespace mdfft {

enum { kTcNone = 0, kTcFp16 = 1, kTcBf16 = 2 };

// Radix plan for the tensor-core variant: as many radix-16 stages as the
// power of two allows, the rest (2, 4, 8, 5, 3) on the SIMT path.
__host__ __device__ constexpr RadixPlan radix_plan_tc(int n) {
    RadixPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, 1};
    int e = 0;
    while (n % 2 == 0) n /= 2, ++e;
    if (e < 4 || e > 10) {
        p.S = -1;
        return p;
    }
    while (e >= 4) p.R[p.S++] = 16, e -= 4;
    if (e) p.R[p.S++] = 1 << e;
    while (n % 5 == 0) p.R[p.S++] = 5, n /= 5;
    while (n % 3 == 0) p.R[p.S++] = 3, n /= 3;
    for (int i = 0; i < p.S; ++i) p.maxR = p.R[i] > p.maxR ? p.R[i] : p.maxR;
    if (n != 1) p.S = -1;
    return p;
}

// cos and sin of 2 pi m / 16 for any integer m
__device__ __forceinline__ float dft16_cos(int m) {
    m &= 15;
    return m < 8 ? (float)cos16(m) : -(float)cos16(m - 8);
}
__device__ __forceinline__ float dft16_sin(int m) {
    m &= 15;
    return m < 8 ? (float)sin16(m) : -(float)sin16(m - 8);
}

// entry (k, n) of the real 32 x 32 block form of the forward DFT-16 matrix
__device__ __forceinline__ float dft16_block(int k, int n) {
    const int r = k & 15, q = n & 15, m = r * q;
    const bool im_in = k >= 16, im_out = n >= 16;
    if (!im_in && !im_out) return dft16_cos(m);
    if (im_in && !im_out) return dft16_sin(m);
    if (!im_in && im_out) return -dft16_sin(m);
    return dft16_cos(m);
}

// split(x0, x1): the pair rounded to two 16-bit values (hi, x0 in the low
// half) and the rounded remainders (lo), each packed in one 32-bit word.
template <int TC> struct TcTypes;
template <> struct TcTypes<kTcFp16> {
    __device__ __forceinline__ static void split(float x0, float x1, uint32_t &hi, uint32_t &lo) {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 f = __half22float2(h);
        const __half2 l = __floats2half2_rn(x0 - f.x, x1 - f.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
    static constexpr bool kScale = true;
    static constexpr uint32_t kFormat = 0;  // instruction-descriptor operand format: F16
};
template <> struct TcTypes<kTcBf16> {
    __device__ __forceinline__ static void split(float x0, float x1, uint32_t &hi, uint32_t &lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 f = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - f.x, x1 - f.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
    static constexpr bool kScale = false;
    static constexpr uint32_t kFormat = 1;  // BF16
};

// Power of two 2^e as a float (|e| <= 126).
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }

// ------------------------------------------------------------------ tcgen05 in inline PTX

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits
// 4-5), A and B format (7-9, 10-12), both K-major (bits 15, 16 clear),
// N >> 3 (bits 17-22) and M >> 4 (bits 24-28).
template <int TC> __host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | (TcTypes<TC>::kFormat << 7) | (TcTypes<TC>::kFormat << 10) | ((32u >> 3) << 17) |
           ((128u >> 4) << 24);
}

// Operand layout in shared memory (no swizzle, K-major): element (row, k) of
// a 16-bit matrix at byte (row / 8) * kTcSbo + (k / 8) * kTcLbo + (row % 8) * 16
// + (k % 8) * 2, i.e. 8-row x 16-byte core matrices, 4 per 8 rows (K = 32).
constexpr uint32_t kTcLbo = 128;  // between core matrices adjacent along K
constexpr uint32_t kTcSbo = 512;  // between core matrices adjacent along the rows
constexpr uint32_t kTcGroupBytes = 128 / 8 * kTcSbo;  // one 128-row group: 8 KiB

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor
// version 1 (bit 46), no swizzle (bits 61-63 clear).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kTcLbo >> 4) << 16) | ((uint64_t)(kTcSbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrives once on bar when every tcgen05.mma this thread issued has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// warp-collective: allocate ncols TMEM columns, base address written to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// warp-collective: 32 consecutive FP32 columns of the warp's 32 TMEM lanes
// (lane i of the warp receives TMEM lane base + i)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&d)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15]),
          "=r"(d[16]), "=r"(d[17]), "=r"(d[18]), "=r"(d[19]), "=r"(d[20]), "=r"(d[21]), "=r"(d[22]), "=r"(d[23]),
          "=r"(d[24]), "=r"(d[25]), "=r"(d[26]), "=r"(d[27]), "=r"(d[28]), "=r"(d[29]), "=r"(d[30]), "=r"(d[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------------ per-CTA state

// The DFT-16 block matrix B (hi, then lo: 32 rows x 32 K each, operand
// layout above), the MMA mbarrier, the TMEM base and the failure flag.
struct alignas(16) TcShared {
    uint32_t b[1024];
    uint64_t bar;
    uint32_t tmem;
    int failed;
};
static_assert(sizeof(TcShared) == kTcSharedBytes, "tensor-core shared state");

constexpr uint64_t kTcWaitNs = 2000000000ull;

// 128-row groups of a CTA and its TMEM columns (32 per group, a power of two)
template <int THREADS> struct TcGeom {
    static constexpr int G = (THREADS + 127) / 128;
    static constexpr uint32_t COLS = G <= 1 ? 32 : G <= 2 ? 64 : G <= 4 ? 128 : 256;
    static_assert(G <= 8, "tensor-core CTA too large");
};

// All threads, before the CTA's first barrier: build B, initialise the
// mbarrier (thread 0) and allocate the accumulator columns (warp 0).  After
// that barrier every thread runs tc_fence_after() before using ts->tmem.
template <int TC, int THREADS> __device__ __forceinline__ void tc_begin(TcShared *ts, int tid) {
    using T = TcTypes<TC>;
    for (int w = tid; w < 1024; w += THREADS) {
        const int hl = w >> 9, n = (w >> 4) & 31, k = (w & 15) * 2;
        uint32_t hi, lo;
        T::split(dft16_block(k, n), dft16_block(k + 1, n), hi, lo);
        const uint32_t off = hl * 2048 + (n >> 3) * kTcSbo + (k >> 3) * kTcLbo + (n & 7) * 16 + (k & 7) * 2;
        ts->b[off >> 2] = hl ? lo : hi;
    }
    if (tid == 0) {
        mbar_init(&ts->bar, 1);
        fence_mbarrier_init();
        ts->failed = 0;
    }
    if (tid < 32) {
        __syncwarp();
        tmem_alloc(&ts->tmem, TcGeom<THREADS>::COLS);
    }
    tc_fence_before();
}

// All threads, at the end of the tile (every TMEM read finished before the
// last tensor-core stage's closing barrier): free the columns, report failure.
template <int THREADS> __device__ __forceinline__ void tc_end(TcShared *ts, int tid, int *err) {
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(ts->tmem, TcGeom<THREADS>::COLS);
    }
    if (tid == 0 && ts->failed && err) atomicExch(err, 1);
}

// One radix-16 stage on tensor cores.  Same index maps as the SIMT stage:
//   butterfly j of a line reads x[j + r NB], is twiddled by w_{16 NS}^{(j mod NS) r}
//   and writes y[(j / NS) 16 NS + j mod NS + q NS].
// parity: which phase of the mbarrier this stage's commit completes.
// The first stage (NS = 1) reads its butterfly from gsrc, the thread's line
// in the tile's landing buffer, ok false for lines outside the array (zeros),
// conj conjugates the loaded values; later stages read the stage buffer.
//
// A_LAND: the operand rows go to the landing buffer (LINES x N complex64 right
// before the stage buffer in fft_pass_tc_kernel; free once the first stage
// has read it) instead of over the stage buffer, so no barrier is needed
// between reading the stage buffer and writing them.  END_CTA: close with a
// CTA barrier (else a warp barrier: the next stage reads only lines that this
// warp wrote).  HOOK: when to call hook() (warp 0 refills the landing buffer):
// 1 right after the operand rows are written (the first stage's source is
// consumed), 2 right after the MMAs completed (operand rows in the landing
// buffer consumed), 0 never.
template <int TC, int N, int LINES, int THREADS, int PADN, int TROW, int NS, bool LAST, bool A_LAND, bool END_CTA,
          int HOOK, class Hook>
__device__ __forceinline__ void tc_radix16_stage(float2 *buf, float2 *tile, const float2 *tw, TcShared *ts,
                                                 bool active, const float2 *gsrc, bool ok, bool conj, uint32_t parity,
                                                 const Hook &hook) {
    constexpr bool FIRST = NS == 1;
    static_assert(!(FIRST && A_LAND), "the first stage reads the landing buffer");
    static_assert(!A_LAND || (size_t)LINES * N * sizeof(float2) >= (size_t)(THREADS + 127) / 128 * 2 * kTcGroupBytes,
                  "operand rows must fit the landing buffer");
    using T = TcTypes<TC>;
    using Geom = TcGeom<THREADS>;
    constexpr int NB = N / 16;
    static_assert(LINES * NB == THREADS, "one radix-16 butterfly per thread");
    constexpr uint32_t kLoOff = Geom::G * kTcGroupBytes;  // lo rows follow the hi rows
    if (ts->failed) return;  // uniform: only written before a barrier
    const int tid = threadIdx.x;
    const int line = tid / NB, j = tid % NB, k = j % NS;

    float2 v[16];
    int e = 0;
    if (active) {
        if constexpr (FIRST) {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = ok ? gsrc[j + r * NB] : make_float2(0.f, 0.f);
            if (conj)
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r].y = -v[r].y;
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                float2 x = buf[line * PADN + pad16(j + r * NB)];
                if (r > 0) x = cmul(x, tw[r * NS + k]);
                v[r] = x;
            }
        }
        if constexpr (T::kScale) {
            float m = 0.f;
#pragma unroll
            for (int r = 0; r < 16; ++r) m = fmaxf(m, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
            // m < 2^e from the exponent bits (m normal); the clamp keeps 2^(15-e) normal
            e = (int)((__float_as_uint(m) >> 23) & 0xff) - 126;
            e = max(-100, min(e, 120));
            const float sc = pow2f(15 - e);  // exact: largest component in [2^14, 2^15)
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r].x *= sc, v[r].y *= sc;
        }
    }
    // every read of the stage buffer before the operand rows overwrite it
    if constexpr (!FIRST && !A_LAND) __syncthreads();

    unsigned char *A = reinterpret_cast<unsigned char *>(buf) - (A_LAND ? (size_t)LINES * N * sizeof(float2) : 0);
    if (active) {
        unsigned char *row = A + (tid >> 3) * kTcSbo + (tid & 7) * 16;
#pragma unroll
        for (int c = 0; c < 4; ++c) {  // K = 8c..8c+7: real parts of v[0..15] (c = 0, 1), then imaginary
            uint32_t h[4], l[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int q = (c & 1) * 8 + 2 * w;
                T::split(c < 2 ? v[q].x : v[q].y, c < 2 ? v[q + 1].x : v[q + 1].y, h[w], l[w]);
            }
            *reinterpret_cast<uint4 *>(row + c * kTcLbo) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(row + kLoOff + c * kTcLbo) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
    fence_proxy_async_shared();  // the operand rows (and B) visible to the tensor cores
    tc_fence_before();           // earlier TMEM reads of this thread before the MMAs below
    __syncthreads();
    if constexpr (HOOK == 1) hook();

    if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_addr(A), b0 = smem_addr(ts->b);
        constexpr uint32_t idesc = tc_idesc<TC>();
#pragma unroll
        for (int g = 0; g < Geom::G; ++g) {
            const uint32_t d = ts->tmem + 32u * g;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {  // K = 16 per instruction: 2 core matrices along K
                const uint32_t ao = a0 + g * kTcGroupBytes + ks * 2 * kTcLbo, bo = b0 + ks * 2 * kTcLbo;
                tc_mma(d, tc_desc(ao), tc_desc(bo), idesc, ks);                 // hi . hi
                tc_mma(d, tc_desc(ao), tc_desc(bo + 2048), idesc, 1);           // hi . lo
                tc_mma(d, tc_desc(ao + kLoOff), tc_desc(bo), idesc, 1);         // lo . hi
            }
        }
        tc_commit(&ts->bar);
    }

    // warp 0 alone waits for the MMAs (the other warps sleep in the barrier
    // instead of polling the mbarrier and taking issue slots)
    if (tid < 32) {
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&ts->bar, parity, kTcWaitNs))) {
            // a second bounded chance for the MMAs to finish before the operands
            // and the columns are reused or freed; the CTA's output is invalid
            mbar_wait_bounded(&ts->bar, parity, kTcWaitNs);
            if (tid == 0) ts->failed = 1;
        }
        tc_fence_before();
    }
    __syncthreads();
    if constexpr (HOOK == 2) hook();
    if (ts->failed) return;  // uniform: written before the barrier
    if (active) {  // warp-uniform
        uint32_t d[32];
        tc_fence_after();
        // warp w reads TMEM lanes 32 (w % 4) .. +31 of group tid / 128: row = tid
        tmem_ld32(ts->tmem + ((uint32_t)(((tid >> 5) & 3) * 32) << 16) + 32u * (uint32_t)(tid >> 7), d);
        const int base = (j / NS) * NS * 16 + k;
        const float unsc = T::kScale ? pow2f(e - 15) : 1.f;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float2 out = make_float2(__uint_as_float(d[q]), __uint_as_float(d[16 + q]));
            if constexpr (T::kScale) out.x *= unsc, out.y *= unsc;
            if constexpr (LAST) tile[(base + q * NS) * TROW + line] = out;
            else buf[line * PADN + pad16(base + q * NS)] = out;
        }
    }
    tc_fence_before();
    if constexpr (END_CTA) __syncthreads();
    else __syncwarp();
}

}  // namespace mdfft
