// tc_stage.cuh -- radix-16 Stockham stage as a tensor-core GEMM (complex64 data).
//
// A radix-16 stage applies the 16-point DFT (Sec. 2, the 1-D DFT equation)
// to every butterfly of the tile.  Written in real arithmetic, one butterfly
// is a row [Re v_0..Re v_15, Im v_0..Im v_15] (K = 32) times the 32 x 32 block
// matrix  B = [[C, -S], [S, C]],  C[r][q] = cos(2 pi r q/16),
// S[r][q] = sin(2 pi r q/16), giving [Re V_0..Re V_15, Im V_0..Im V_15]
// (forward sign).  A warp handles 16 butterflies at a time with
// mma.sync.m16n8k16 (2 k-steps x 4 n-tiles).  Operands are split x = hi + lo
// in FP16 or BF16 and three products hi*hi + hi*lo + lo*hi are accumulated in
// FP32 (lo*lo is below the FP32 rounding of the sum).  FP16 rows are scaled by
// an exact power of two so that their largest component lies in [2^14, 2^15)
// before the split; the scale is undone on the FP32 results.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

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

template <int TC> struct TcTypes;
template <> struct TcTypes<kTcFp16> {
    __device__ __forceinline__ static uint32_t pack(float lo_k, float hi_k) {  // lower column in the low half
        __half2 h = __halves2half2(__float2half_rn(lo_k), __float2half_rn(hi_k));
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __device__ __forceinline__ static float round(float x) { return __half2float(__float2half_rn(x)); }
    __device__ __forceinline__ static void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    static constexpr bool kScale = true;
};
template <> struct TcTypes<kTcBf16> {
    __device__ __forceinline__ static uint32_t pack(float lo_k, float hi_k) {
        __nv_bfloat162 h = __halves2bfloat162(__float2bfloat16_rn(lo_k), __float2bfloat16_rn(hi_k));
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __device__ __forceinline__ static float round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
    __device__ __forceinline__ static void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    static constexpr bool kScale = false;
};

// One radix-16 stage on tensor cores.  Reads the stage buffer (padded, one
// line per LINES), writes the next stage buffer or, for the last stage, the
// transposed tile.  Same index maps as the SIMT stage:
//   butterfly j of a line reads x[j + r NB], is twiddled by w_{16 NS}^{(j mod NS) r}
//   and writes y[(j / NS) 16 NS + j mod NS + q NS].
// Power of two 2^e as a float (|e| <= 126).
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }

// The B fragments of the DFT-16 block matrix, split hi/lo, for every lane:
// word ((ks*4 + nt)*2 + i)*2 + hl of lane L holds, for k-step ks, n-tile nt,
// register i (k = 2tq + 8i, +1 of column n = nt*8 + g), the hi (hl = 0) or lo
// (hl = 1) pair.  1024 words, written once per CTA.
constexpr int kTcBfragWords = 2 * 4 * 2 * 2 * 32;
template <int TC, int THREADS> __device__ __forceinline__ void tc_build_bfrag(uint32_t *bf, int tid) {
    using T = TcTypes<TC>;
    for (int w = tid; w < kTcBfragWords; w += THREADS) {
        const int lane = w & 31, idx = w >> 5;
        const int hl = idx & 1, i = (idx >> 1) & 1, nt = (idx >> 2) & 3, ks = idx >> 4;
        const int g = lane >> 2, tq = lane & 3;
        const int k0 = ks * 16 + 2 * tq + 8 * i, n = nt * 8 + g;
        const float x0 = dft16_block(k0, n), x1 = dft16_block(k0 + 1, n);
        const float h0 = T::round(x0), h1 = T::round(x1);
        bf[w] = hl ? T::pack(x0 - h0, x1 - h1) : T::pack(h0, h1);
    }
}

template <int TC, int N, int LINES, int THREADS, int PADN, int TROW, int NS, bool LAST>
__device__ __forceinline__ void tc_radix16_stage(float2 *buf, float2 *tile, const float2 *tw, const uint32_t *bf,
                                                 bool active) {
    using T = TcTypes<TC>;
    constexpr int NB = N / 16;
    constexpr int ROWS = LINES * NB;
    static_assert(ROWS % 16 == 0, "butterflies per tile must fill whole mma tiles");
    constexpr int GROUPS = ROWS / 16;
    constexpr int NWARPS = THREADS / 32;
    constexpr int GPW = (GROUPS + NWARPS - 1) / NWARPS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;

    // B fragments (built once per CTA by tc_build_bfrag): word [((ks*4 + nt)*2 + i)*2 + hl][lane]
    float acc[GPW][4][4];
    int expo[GPW][2];
#pragma unroll
    for (int gi = 0; gi < GPW; ++gi) {
        const int grp = warp + gi * NWARPS;
        if (!active || grp >= GROUPS) break;  // uniform within the warp (THREADS is a multiple of 32)
        float2 v[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = grp * 16 + g + 8 * h;
            const int line = row / NB, j = row % NB, k = j % NS;
            const int rr[4] = {2 * tq, 2 * tq + 1, 2 * tq + 8, 2 * tq + 9};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float2 x = buf[line * PADN + pad16(j + rr[i] * NB)];
                if constexpr (NS > 1) x = cmul(x, tw[rr[i] * NS + k]);
                v[h][i] = x;
            }
            int e = 0;
            if constexpr (T::kScale) {
                float m = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) m = fmaxf(m, fmaxf(fabsf(v[h][i].x), fabsf(v[h][i].y)));
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
                // m < 2^e with e from the exponent bits (m normal); clamp keeps 2^(15-e) normal
                e = (int)((__float_as_uint(m) >> 23) & 0xff) - 126;
                e = max(-100, min(e, 120));
                const float sc = pow2f(15 - e);  // exact scaling: max component in [2^14, 2^15)
#pragma unroll
                for (int i = 0; i < 4; ++i) v[h][i].x *= sc, v[h][i].y *= sc;
            }
            expo[gi][h] = e;
        }
        // A fragments: k-step 0 = real parts, k-step 1 = imaginary parts;
        // a0/a1: rows g / g+8 at k = 2tq, 2tq+1; a2/a3: at k = 2tq+8, 2tq+9
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int reg = 0; reg < 4; ++reg) {
                const int h = reg & 1, i0 = (reg >> 1) * 2;
                const float x0 = ks ? v[h][i0].y : v[h][i0].x;
                const float x1 = ks ? v[h][i0 + 1].y : v[h][i0 + 1].x;
                const float h0 = T::round(x0), h1 = T::round(x1);
                ah[ks][reg] = T::pack(h0, h1);
                al[ks][reg] = T::pack(x0 - h0, x1 - h1);
            }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint32_t *b = bf + ((ks * 4 + nt) * 2) * 2 * 32 + lane;
                const uint32_t bh0 = b[0], bl0 = b[32], bh1 = b[64], bl1 = b[96];
                T::mma(c, ah[ks], bh0, bh1);
                T::mma(c, ah[ks], bl0, bl1);
                T::mma(c, al[ks], bh0, bh1);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[gi][nt][i] = c[i];
        }
    }
    __syncthreads();  // every read of buf before any write
#pragma unroll
    for (int gi = 0; gi < GPW; ++gi) {
        const int grp = warp + gi * NWARPS;
        if (!active || grp >= GROUPS) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = grp * 16 + g + 8 * h;
            const int line = row / NB, j = row % NB, k = j % NS;
            const int base = (j / NS) * NS * 16 + k;
            const float unsc = T::kScale ? pow2f(expo[gi][h] - 15) : 1.f;
#pragma unroll
            for (int half = 0; half < 2; ++half)      // q = 2tq + e (n-tiles 0/2) or 8 + 2tq + e (1/3)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int q = 8 * half + 2 * tq + e;
                    float re = acc[gi][half][2 * h + e], im = acc[gi][half + 2][2 * h + e];
                    if (T::kScale) re *= unsc, im *= unsc;
                    const float2 out = make_float2(re, im);
                    if constexpr (LAST) tile[(base + q * NS) * TROW + line] = out;
                    else buf[line * PADN + pad16(base + q * NS)] = out;
                }
        }
    }
    __syncthreads();
}

}  // namespace mdfft
