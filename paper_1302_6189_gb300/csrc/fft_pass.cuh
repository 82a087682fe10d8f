// fft_pass.cuh -- one fused pass of the M-D FFT for sm_103a.
//
// A pass is one step of the parallel algorithm of Fig. 4 (Duy and Ozaki,
// arXiv:1302.6189) together with the transpose that follows it: the 1-D
// DFTs (Sec. 2) along f, the fastest axis of the input layout, and the
// redistribution of the result into the output layout, whose fastest axis g
// is a different axis.  On one GPU the transpose is the store itself.
//
// Tiling.  A CTA owns a tile of lines: Bg lines that are consecutive along g
// times Bh lines consecutive along h (the next axis of the output layout).
//  1. load   each line is contiguous in the input (stride 1 along f), so the
//            first radix stage reads straight from HBM into registers with
//            warp-contiguous accesses (or, for very short lines, the tile is
//            first copied into shared memory);
//  2. FFT    Stockham autosort stages, radices 16/8/4/2/5/3, one butterfly
//            per thread per stage in registers, padded shared memory between
//            stages; twiddles w_N^q come from a table made in FP64;
//  3. store  the last stage writes the tile transposed ([k][line]) into
//            shared memory; every thread then owns one line and writes its
//            k values, so a warp writes runs of Bg consecutive elements of
//            the output layout's fastest axis.
// Inverse transforms conjugate the input of their first pass and the output
// of their last one (conj(DFT(conj x)) is the exp(+2 pi i/N) sum; between
// passes the two conjugations cancel); `scale` multiplies the stored values.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "smem_layout.h"

namespace mdfft {

constexpr int kMaxTileDims = 8;

// Owner of a row-major index x of a layout.  f_MD chunks (Sec. 3.2, blk
// null): with q = x / tail (the index over the `lead` product of the leading
// dims the chunks are cut on), owner = floor(((q + 1) P - 1) / lead).  Block
// decompositions of the comparison methods (Sec. 4, blk non-null): blk holds
// 3 nd entries, per layout position (slowest first) its extent d, the blocks
// q it is cut into and the pid stride ps; a coordinate c lies in block
// floor(((c + 1) q - 1) / d) and owner = sum of block * ps.  line_div turns
// the owner difference of a line's ends into the owners on it minus one.
struct OwnerMap {
    int64_t tail, lead, P;
    const int64_t *blk;
    int nd;
    int64_t line_div;
};

// Division of a 32-bit n by a divisor d fixed for the launch, as a
// multiply-high and a shift (Granlund and Montgomery, division by invariant
// integers using multiplication: with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, floor(n / d) = (mulhi(m, n) + n) >> l,
// the sum taken in 64 bits).  The host fills m and l (fastdiv_make).
struct FastDiv {
    uint32_t d, m, l;
};
__host__ __device__ constexpr FastDiv fastdiv_make(uint32_t d) {
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    return FastDiv{d, (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1), l};
}

struct PassArgs {
    const void *in;
    void *out;
    const void *tw;                 // twiddle table of the radix plan (tw_offset layout), pass precision
    int64_t gblocks, hblocks;       // tiles along g and along h
    int nrest;                      // remaining axes (not f, g, h), one tile unit each
    int64_t rest_count[kMaxTileDims];
    int64_t rest_in[kMaxTileDims];  // input stride of that axis (elements)
    int64_t rest_out[kMaxTileDims]; // output stride
    int Bg, Bh;                     // lines per tile along g and h
    int64_t Ng, Nh;                 // extents of g and h (ragged last tiles are masked)
    int64_t in_sg, in_sh;           // input strides of g and h
    int64_t out_sh, out_sf;         // output strides of h and f
    int64_t out_sg;                 // output stride of g: 1 (g the output's fastest axis), N_f when the
                                    // output keeps f fastest, or any stride (input-chunk tile order)
    int line_store;                 // 1: the output keeps f fastest (lines stored whole, no transpose)
    int conj;                       // inverse: bit 0 conjugates the loaded input, bit 1 the stored output
    double scale;                   // multiplies every stored value
    int scaled;                     // scale != 1 (set with scale, so the kernel tests an integer, not a double)
    int64_t ntiles;                 // tiles of the pass (persistent kernels walk them)
    int tile32;                     // every tile index and tile count fits 32 bits (cheaper divisions)
    FastDiv fd_g, fd_h, fd_rest[kMaxTileDims];  // gblocks, hblocks, rest_count as multiply-shift divisors
    FastDiv fd_bg;                  // Bg as a multiply-shift divisor (tile line -> g, h; used when fd_bg.d == Bg)
    int *err;                       // persistent kernels: set to 1 if a bounded wait gave up (may be null)
    unsigned long long *moved;      // count mode: points whose owner changes (null: off)
    unsigned long long *split;      // count mode: split-line amount of the input layout
    OwnerMap own_in, own_out;
};

// ------------------------------------------------------------------ radix plans

struct RadixPlan {
    int S;       // stages
    int R[12];   // radix of each stage
    int maxR;
};

__host__ __device__ constexpr RadixPlan radix_plan(int n) {
    RadixPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, 1};
    int e = 0;
    while (n % 2 == 0) n /= 2, ++e;
    // powers of two: as few stages as radix 16 allows, balanced
    const int pw[11][3] = {{0, 0, 0},  {2, 0, 0},  {4, 0, 0},  {8, 0, 0},  {16, 0, 0}, {8, 4, 0},
                           {8, 8, 0},  {16, 8, 0}, {16, 16, 0}, {16, 16, 2}, {16, 8, 8}};
    if (e <= 10)
        for (int i = 0; i < 3; ++i)
            if (pw[e][i]) p.R[p.S++] = pw[e][i];
    while (n % 5 == 0) p.R[p.S++] = 5, n /= 5;
    while (n % 3 == 0) p.R[p.S++] = 3, n /= 3;
    for (int i = 0; i < p.S; ++i) p.maxR = p.R[i] > p.maxR ? p.R[i] : p.maxR;
    if (n != 1 || e > 10) p.S = -1;  // unsupported length
    return p;
}

// The autotuner's alternative radix plan of a length: the power-of-two part
// split otherwise (16 = 4x4, 32 = 16x2, 64 = 16x4, 128 = 8x4x4, 256 = 8x8x4,
// 512 = 8x8x8, 1024 = 16x16x4; odd factors as in radix_plan).
__host__ __device__ constexpr RadixPlan radix_plan_alt(int n) {
    RadixPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, 1};
    int e = 0;
    while (n % 2 == 0) n /= 2, ++e;
    const int pw[11][3] = {{0, 0, 0},  {2, 0, 0},  {4, 0, 0},  {8, 0, 0},  {4, 4, 0},  {16, 2, 0},
                           {16, 4, 0}, {8, 4, 4}, {8, 8, 4}, {8, 8, 8}, {16, 16, 4}};
    if (e <= 10)
        for (int i = 0; i < 3; ++i)
            if (pw[e][i]) p.R[p.S++] = pw[e][i];
    while (n % 5 == 0) p.R[p.S++] = 5, n /= 5;
    while (n % 3 == 0) p.R[p.S++] = 3, n /= 3;
    for (int i = 0; i < p.S; ++i) p.maxR = p.R[i] > p.maxR ? p.R[i] : p.maxR;
    if (n != 1 || e > 10) p.S = -1;
    return p;
}

// Twiddle table of a radix plan.  Stage 0 needs none (w^0 = 1); stage s >= 1,
// after NS = R_0 ... R_{s-1} points are combined, uses w_{NS R}^{k r} for
// k < NS, r < R, stored as entry r * NS + k (consecutive k are consecutive
// words, so the lanes of a warp read distinct banks) at tw_offset(plan, s).
__host__ __device__ constexpr int tw_offset(const RadixPlan &p, int s) {
    int off = 0, ns = 1;
    for (int i = 0; i < s && i < p.S; ++i) {
        if (i > 0) off += ns * p.R[i];
        ns *= p.R[i];
    }
    return off;
}
__host__ __device__ constexpr int tw_entries(const RadixPlan &p) { return tw_offset(p, p.S); }

template <typename Real> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__host__ __device__ constexpr RadixPlan radix_plan_tc(int n);
// shared state of the tensor-core stages (the DFT-16 operand, an mbarrier,
// the TMEM base, a flag), TcShared in tc_stage.cuh
constexpr int kTcSharedBytes = 4112;

// Launch configuration of the pass kernel for line length N.  TC != 0 selects
// the tensor-core variant (complex64 only): radix-16 stages run as GEMMs.
// THR != 0 fixes the CTA at THR threads for every length (the persistent
// serving kernel): a power-of-two number of threads per line and THR / that
// many lines per tile (stage loops skip butterflies a thread does not own);
// for a tensor-core kernel THR / (N / 16) lines (one butterfly per thread).
__host__ __device__ constexpr int pow2ceil(int x) {
    int p = 1;
    while (p < x) p *= 2;
    return p;
}

// complex64 lengths whose default CTA shape takes a power-of-two number of
// threads per line (direct loads, warp-local stages) instead of N / (largest
// radix): the ones where that measured faster on a GB300 (one pass over
// 64 x 64 x N: N = 24 1.47x, 48 1.59x, 240 1.31x, 480 1.08x, 960 1.03x; the
// other lengths with an odd factor measured slower with it).
__host__ __device__ constexpr bool pow2_threads_default(int n) {
    return n == 24 || n == 48 || n == 240 || n == 480 || n == 960;
}

// RP = 1 selects the alternative radix plan (radix_plan_alt; SIMT kernels).
template <typename Real, int N, int TC = 0, int THR = 0, int RP = 0> struct PassCfg {
    using C = typename Cx<Real>::T;
    static_assert(TC == 0 || sizeof(Real) == 4, "tensor-core stages are complex64 only");
    static_assert(RP == 0 || TC == 0, "alternative radix plans are SIMT only");
    static constexpr RadixPlan plan = TC ? radix_plan_tc(N) : RP ? radix_plan_alt(N) : radix_plan(N);
    static_assert(plan.S >= 0, "unsupported line length");  // S = 0: N = 1, a pure redistribution
    static constexpr int TL0 = N / plan.maxR;  // one butterfly per thread in the widest stage
    static constexpr int kMinLines = 128 / (int)sizeof(C);
    static constexpr bool POW2 = sizeof(Real) == 4 && TC == 0 && pow2_threads_default(N);
    // (tensor-core CTAs keep one radix-16 butterfly per thread: THR only sets their line count)
    static constexpr int TL = TC     ? TL0
                              : THR  ? (pow2ceil(TL0) < THR / kMinLines ? pow2ceil(TL0) : THR / kMinLines)
                              : POW2 ? pow2ceil(TL0)
                                     : TL0;
    static constexpr int kTileElems = sizeof(Real) == 4 ? 4096 : 2048;
    // lines per tile: a power of two near kTileElems / N, at least enough for
    // 128-byte store runs (16 complex64 / 8 complex128), and a whole number
    // of warps per CTA; complex64 tiles grow only up to 256 threads (more,
    // smaller CTAs per SM measured faster for every length it changes)
    // (tensor-core CTAs stay at <= 512 threads: their stages need ~100 registers)
    static constexpr int kMaxThreads = TC ? 512 : 1024;
    static constexpr int kGrowThreads = (sizeof(Real) == 4 && TC == 0) ? 256 : kMaxThreads;
    static constexpr int lines_for() {
        if (THR) return THR / TL;
        // tensor-core CTAs for 512-point lines: 8 lines (256 threads), so that
        // two CTAs share an SM (16 lines take 512 threads at 128 registers)
        if (TC && TL == 32) return 8;
        int l = kMinLines;
        while (l > 1 && TL * l > kMaxThreads) l /= 2;
        while (l < 256 && 2 * l * N <= kTileElems && 2 * TL * l <= kGrowThreads) l *= 2;
        while ((TL * l) % 32 != 0 && 2 * TL * l <= kMaxThreads) l *= 2;
        return l;
    }
    static constexpr int LINES = lines_for();
    static_assert(TL * LINES <= kMaxThreads && (TL * LINES) % 32 == 0, "CTA shape");
    static constexpr int THREADS = TL * LINES;
    // shared-memory padding (the bank-conflict-free choice of smem_layout.h
    // for complex64; tensor-core and complex128 configurations use the default)
    static constexpr SmemLayout LAY = (sizeof(Real) == 4 && TC == 0) ? smem_layout_c64(N, THR, RP) : SmemLayout{16, 1, 1};
    static constexpr int PADG = LAY.g;                // pad(i) = i + i / PADG
    static constexpr int PADN = N + N / PADG + LAY.pe;  // line stride of the stage buffer
    static constexpr int TROW = LINES + LAY.te;         // row of the transposed tile
    static constexpr int DATA0 = LINES * PADN > N * TROW ? LINES * PADN : N * TROW;
    // tensor-core stages write their operand rows (hi and lo, 128 B per row,
    // whole 128-row groups) over the stage buffer; offsets stay 16-byte aligned
    static constexpr int TC_ROWS = TC ? (TL * LINES + 127) / 128 * 128 : 0;
    static constexpr int DATA = TC ? ((DATA0 > TC_ROWS * 16 ? DATA0 : TC_ROWS * 16) + 1) / 2 * 2 : DATA0;
    static constexpr int TWN0 = tw_entries(plan) > 0 ? tw_entries(plan) : 1;  // twiddle entries
    static constexpr int TWN = TC ? (TWN0 + 1) / 2 * 2 : TWN0;
    static constexpr int BFRAG = TC ? kTcSharedBytes / (int)sizeof(C) : 0;  // tensor-core shared state (C units)
    // + the input offset of every tile line and the tile's coordinates (4 int64)
    static constexpr size_t SMEM = (size_t)(DATA + TWN + BFRAG) * sizeof(C) + (size_t)(LINES + 4) * sizeof(int64_t);
    // first stage loads from HBM directly (always for tensor-core plans, whose
    // first stage is a radix-16 GEMM with one butterfly per thread)
    static constexpr bool DIRECT = TC != 0 || TL * (int)sizeof(C) >= 32;
};

// ------------------------------------------------------------------ complex helpers

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
// Every multiply-add of the butterflies is written out as one fused
// multiply-add (fmadd) or, for a sum of two products, one rounded product
// and one fused multiply-add (fma_prod): left to the compiler, whether and
// which product is fused can differ between kernels that inline the same
// butterflies (register pressure, scheduling), and their results with it.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }  // a b + c
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_prod(float a, float b, float c, float d) {
    return __fmaf_rn(a, b, __fmul_rn(c, d));  // a b + c d
}
__device__ __forceinline__ double fma_prod(double a, double b, double c, double d) {
    return __fma_rn(a, b, __dmul_rn(c, d));
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return {fma_prod(a.x, b.x, -a.y, b.y), fma_prod(a.x, b.y, a.y, b.x)};
}

// w_16^k = cos(2 pi k/16) - i sin(2 pi k/16), k < 8: cosines and sines of
// multiples of pi/8
__host__ __device__ constexpr double cos16(int k) {
    return k == 0 ? 1.0
         : k == 1 ? 0.92387953251128675613
         : k == 2 ? 0.70710678118654752440
         : k == 3 ? 0.38268343236508977173
         : k == 4 ? 0.0
         : k == 5 ? -0.38268343236508977173
         : k == 6 ? -0.70710678118654752440
                  : -0.92387953251128675613;
}
__host__ __device__ constexpr double sin16(int k) { return cos16(k <= 4 ? 4 - k : k - 4); }  // sin(k pi/8) = cos((4-k) pi/8)

// e +- o w_16^K in six multiply-adds for the angles that need a product:
// o w = (o.x c + o.y s, o.y c - o.x s) (c, s = cos, sin of 2 pi K/16) is
// written f (u.x, u.y) with the larger of |c|, |s| factored out as f, so
// that u needs one multiply-add per part with a factor of magnitude <= 1;
// then e + f u and e - f u are one multiply-add per part each.
template <int K, typename C> __device__ __forceinline__ void butterfly16(C &lo, C &hi, const C &e, const C &o) {
    using R = decltype(o.x);
    if constexpr (K == 0) {
        lo = cadd(e, o), hi = csub(e, o);
    } else if constexpr (K == 4) {  // o (-i)
        lo = C{e.x + o.y, e.y - o.x}, hi = C{e.x - o.y, e.y + o.x};
    } else {
        constexpr double c = cos16(K), s = sin16(K);
        constexpr bool by_c = (c < 0 ? -c : c) >= (s < 0 ? -s : s);
        constexpr R f = (R)(by_c ? c : s), t = (R)(by_c ? s / c : c / s);
        const C u = by_c ? C{fmadd(t, o.y, o.x), fmadd(-t, o.x, o.y)} : C{fmadd(t, o.x, o.y), fmadd(t, o.y, -o.x)};
        lo = C{fmadd(f, u.x, e.x), fmadd(f, u.y, e.y)};
        hi = C{fmadd(-f, u.x, e.x), fmadd(-f, u.y, e.y)};
    }
}

template <int R, typename C> struct DftPow2 {
    template <int K> __device__ __forceinline__ static void combine(C (&v)[R], const C (&e)[R / 2],
                                                                    const C (&o)[R / 2]) {
        if constexpr (K < R / 2) {
            butterfly16<K * (16 / R)>(v[K], v[K + R / 2], e[K], o[K]);
            combine<K + 1>(v, e, o);
        }
    }
    __device__ __forceinline__ static void run(C (&v)[R]) {
        if constexpr (R == 2) {
            C a = v[0], b = v[1];
            v[0] = cadd(a, b);
            v[1] = csub(a, b);
        } else {
            C e[R / 2], o[R / 2];
#pragma unroll
            for (int i = 0; i < R / 2; ++i) e[i] = v[2 * i], o[i] = v[2 * i + 1];
            DftPow2<R / 2, C>::run(e);
            DftPow2<R / 2, C>::run(o);
            combine<0>(v, e, o);
        }
    }
};

template <typename C> __device__ __forceinline__ void dft3(C (&v)[3]) {
    using R = decltype(v[0].x);
    const R s = (R)0.86602540378443864676;  // sin(2 pi / 3)
    C t1 = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C m = {fmadd((R)-0.5, t1.x, v[0].x), fmadd((R)-0.5, t1.y, v[0].y)};
    v[0] = cadd(v[0], t1);
    // -i s d and +i s d
    v[1] = {fmadd(s, d.y, m.x), fmadd(-s, d.x, m.y)};
    v[2] = {fmadd(-s, d.y, m.x), fmadd(s, d.x, m.y)};
}

template <typename C> __device__ __forceinline__ void dft5(C (&v)[5]) {
    using R = decltype(v[0].x);
    const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
    const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
    C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    C x0 = v[0];
    C p1 = {fmadd(c2, a2.x, fmadd(c1, a1.x, x0.x)), fmadd(c2, a2.y, fmadd(c1, a1.y, x0.y))};
    C p2 = {fmadd(c1, a2.x, fmadd(c2, a1.x, x0.x)), fmadd(c1, a2.y, fmadd(c2, a1.y, x0.y))};
    C q1 = {fma_prod(s1, b1.x, s2, b2.x), fma_prod(s1, b1.y, s2, b2.y)};    // X1 = p1 - i q1, X4 = p1 + i q1
    C q2 = {fma_prod(s2, b1.x, -s1, b2.x), fma_prod(s2, b1.y, -s1, b2.y)};  // X2 = p2 - i q2, X3 = p2 + i q2
    v[0] = {x0.x + a1.x + a2.x, x0.y + a1.y + a2.y};
    v[1] = {p1.x + q1.y, p1.y - q1.x};
    v[4] = {p1.x - q1.y, p1.y + q1.x};
    v[2] = {p2.x + q2.y, p2.y - q2.x};
    v[3] = {p2.x - q2.y, p2.y + q2.x};
}

template <int R, typename C> __device__ __forceinline__ void dft(C (&v)[R]) {
    if constexpr (R == 3) dft3(v);
    else if constexpr (R == 5) dft5(v);
    else DftPow2<R, C>::run(v);
}

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
// (indices are never negative: unsigned division by the constant G is a shift)
template <int G> __device__ __forceinline__ int padg(int i) { return i + (int)((unsigned)i / (unsigned)G); }

}  // namespace mdfft

#include "tc_stage.cuh"

namespace mdfft {

__device__ __forceinline__ int64_t owner_of(const OwnerMap &m, int64_t x) {
    if (m.blk) {
        int64_t pid = 0;
        for (int i = m.nd - 1; i >= 0; --i) {
            const int64_t d = m.blk[i], q = m.blk[m.nd + i];
            const int64_t c = x % d;
            x /= d;
            if (q > 1) pid += (((c + 1) * q - 1) / d) * m.blk[2 * m.nd + i];
        }
        return pid;
    }
    unsigned __int128 q = (unsigned __int128)(x / m.tail);
    return (int64_t)(((q + 1) * (unsigned __int128)m.P - 1) / (unsigned __int128)m.lead);
}

// ------------------------------------------------------------------ stages

// One Stockham stage with radix R after NS points already combined.
// Butterfly j (< N/R) reads x[j + r N/R], applies w_{NS R}^{(j mod NS) r},
// does DFT_R and writes y[(j / NS) NS R + j mod NS + r NS].
// SRC selects where the first stage reads: -1 the default of the
// configuration (HBM directly when DIRECT, else the staged tile), 2 a landing
// buffer in shared memory holding the tile's lines unpadded (gsrc = the line),
// 3 a slot of a ring of such buffers that is refilled only after the tile's
// closing barrier (line-local stages keep their warp barriers); with 3 the
// last stage writes a transposed-tile buffer of its own (tile != buf) that
// nothing reads while the stages run, so it needs no barrier before its writes.
template <typename Real, int N, int SI, int NS, int TC = 0, int THR = 0, int SRC = -1, int RP = 0> struct Stages {
    using Cfg = PassCfg<Real, N, TC, THR, RP>;
    static constexpr int SRC0 = SRC >= 0 ? SRC : (Cfg::DIRECT ? 1 : 0);
    using C = typename Cfg::C;
    static constexpr int R = Cfg::plan.R[SI];
    static constexpr int NB = N / R;
    static constexpr int PER = (NB + Cfg::TL - 1) / Cfg::TL;
    static constexpr bool FIRST = SI == 0;
    static constexpr bool LAST = SI == Cfg::plan.S - 1;
    static constexpr int TWOFF = tw_offset(Cfg::plan, SI);
    // a line's threads lie in one warp and a stage that is not the last reads
    // and writes only its own line: warp barriers suffice around it (the last
    // stage writes the transposed tile across lines and needs the CTA barrier;
    // so does a landing buffer, refilled for every warp after the first stage)
    static constexpr bool WARP_LOCAL = TC == 0 && 32 % Cfg::TL == 0 && SRC != 2;
    // tensor-core plans (radix-16 stages first; see tc_radix16_stage): later
    // radix-16 stages write their operand rows into the landing buffer; a
    // stage that is not the last closes with a warp barrier when every line
    // lies in one warp; the landing buffer is refilled once its last reader
    // is done (after the first stage's operand rows are written when only
    // the first stage is radix 16, else after the last radix-16 stage's MMAs)
    static constexpr int TC_LAST = [] {
        int l = -1;
        for (int i = 0; i < Cfg::plan.S; ++i)
            if (Cfg::plan.R[i] == 16) l = i;
        return l;
    }();
    static constexpr bool TC_A_LAND = TC != 0 && !FIRST;
    static constexpr bool TC_END_CTA = LAST || !(Cfg::TL <= 32 && 32 % Cfg::TL == 0);
    static constexpr int TC_HOOK = TC_LAST == 0 ? (SI == 0 ? 1 : 0) : (SI == TC_LAST ? 2 : 0);

    struct NoHook {
        __device__ __forceinline__ void operator()() const {}
    };

    // gsrc: this thread's line in HBM (first stage, direct loads) or null.
    // after_first() runs once the first stage is done with its source (all
    // threads, after the stage's closing barrier; in tensor-core plans, once
    // the landing buffer's last reader is done, see TC_HOOK).  tc_par: parity of the
    // tensor-core mbarrier phase at the tile's first radix-16 stage.
    template <class Hook = NoHook>
    __device__ __forceinline__ static void run(C *buf, C *tile, const C *tw, const C *gsrc, int line, int t,
                                               bool ok, bool conj, bool active, const Hook &after_first = Hook(),
                                               uint32_t tc_par = 0) {
        if constexpr (TC != 0 && R == 16) {
            tc_radix16_stage<TC, N, Cfg::LINES, Cfg::THREADS, Cfg::PADN, Cfg::TROW, NS, LAST, TC_A_LAND,
                             TC_END_CTA, TC_HOOK>(buf, tile, tw + TWOFF,
                                                  reinterpret_cast<TcShared *>(const_cast<C *>(tw) + Cfg::TWN), active,
                                                  gsrc, ok, conj, tc_par ^ (uint32_t)(SI & 1), after_first);
        } else {
            simt(buf, tile, tw, gsrc, line, t, ok, conj);
            if constexpr (FIRST) after_first();
        }
        if constexpr (!LAST)
            Stages<Real, N, SI + 1, NS * R, TC, THR, SRC, RP>::run(buf, tile, tw, gsrc, line, t, ok, conj, active,
                                                               after_first, tc_par);
    }

    __device__ __forceinline__ static void simt(C *buf, C *tile, const C *tw, const C *gsrc, int line, int t,
                                                bool ok, bool conj) {
        C v[PER][R];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int j = t + i * Cfg::TL;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if ((NB % Cfg::TL == 0 || j < NB) && ok) {
                    if constexpr (FIRST && SRC0 == 1) {
                        C x = __ldg(gsrc + j + r * NB);
                        if (conj) x.y = -x.y;
                        v[i][r] = x;
                    } else if constexpr (FIRST && (SRC0 == 2 || SRC0 == 3)) {
                        C x = gsrc[j + r * NB];
                        if (conj) x.y = -x.y;
                        v[i][r] = x;
                    } else {
                        v[i][r] = buf[line * Cfg::PADN + padg<Cfg::PADG>(j + r * NB)];
                    }
                } else {
                    v[i][r] = C{0, 0};
                }
            }
        }
        if constexpr (!(FIRST && SRC0 != 0) && !(LAST && SRC == 3)) {  // all reads of buf before any write
            if constexpr (WARP_LOCAL && !LAST) __syncwarp();
            else __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int j = t + i * Cfg::TL;
            if ((NB % Cfg::TL == 0 || j < NB) && ok) {
                const int k = (int)((unsigned)j % (unsigned)NS);  // j >= 0: unsigned arithmetic by constants
                if constexpr (NS > 1) {
#pragma unroll
                    for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], tw[TWOFF + r * NS + k]);
                }
                dft<R>(v[i]);
                const int base = (int)((unsigned)j / (unsigned)NS) * NS * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if constexpr (LAST) {
                        tile[(base + r * NS) * Cfg::TROW + line] = v[i][r];
                    } else {
                        buf[line * Cfg::PADN + padg<Cfg::PADG>(base + r * NS)] = v[i][r];
                    }
                }
            }
        }
        if constexpr (WARP_LOCAL && !LAST) __syncwarp();
        else __syncthreads();
    }
};

// ------------------------------------------------------------------ one tile

// Tile t of a pass: where its lines start in the input and output arrays and
// its first line along g and h.
struct TileCoord {
    int64_t in_base, out_base, g0, h0;
};

// Tile index -> coordinates, g fastest.  With tile32 (the host checked that
// the pass has fewer than 2^32 tiles, so every count and quotient fits) the
// divisions run in 32 bits, several times cheaper than in 64.
__device__ __forceinline__ uint32_t fastdiv(uint32_t n, const FastDiv &f) {
    return (uint32_t)(((uint64_t)__umulhi(n, f.m) + n) >> f.l);
}

// Line l of a tile (g fastest) -> its position (bg, bh) along g and h: by the
// multiply-shift divisor when the host set it for this Bg, else by division.
__device__ __forceinline__ void tile_line(const PassArgs &a, int l, int &bg, int &bh) {
    if (a.fd_bg.d == (uint32_t)a.Bg) {
        bh = (int)fastdiv((uint32_t)l, a.fd_bg);
        bg = l - bh * a.Bg;
    } else {
        bg = l % a.Bg;
        bh = l / a.Bg;
    }
}

__device__ __forceinline__ TileCoord tile_coords32(const PassArgs &a, uint32_t t) {
    TileCoord c;
    uint32_t q = fastdiv(t, a.fd_g);
    const uint32_t gb = t - q * a.fd_g.d;
    t = q;
    q = fastdiv(t, a.fd_h);
    const uint32_t hb = t - q * a.fd_h.d;
    t = q;
    c.g0 = (int64_t)gb * a.Bg, c.h0 = (int64_t)hb * a.Bh;
    c.in_base = c.g0 * a.in_sg + c.h0 * a.in_sh;
    c.out_base = c.g0 * a.out_sg + c.h0 * a.out_sh;
    for (int i = 0; i < a.nrest; ++i) {
        q = fastdiv(t, a.fd_rest[i]);
        const uint32_t r = t - q * a.fd_rest[i].d;
        t = q;
        c.in_base += (int64_t)r * a.rest_in[i];
        c.out_base += (int64_t)r * a.rest_out[i];
    }
    return c;
}

__device__ __forceinline__ TileCoord tile_coords(const PassArgs &a, int64_t t) {
    if (a.tile32) return tile_coords32(a, (uint32_t)t);
    TileCoord c;
    const int64_t gb = t % a.gblocks;
    t /= a.gblocks;
    const int64_t hb = t % a.hblocks;
    t /= a.hblocks;
    c.g0 = gb * a.Bg, c.h0 = hb * a.Bh;
    c.in_base = c.g0 * a.in_sg + c.h0 * a.in_sh;
    c.out_base = c.g0 * a.out_sg + c.h0 * a.out_sh;
    for (int i = 0; i < a.nrest; ++i) {
        const int64_t q = t % a.rest_count[i];
        t /= a.rest_count[i];
        c.in_base += q * a.rest_in[i];
        c.out_base += q * a.rest_out[i];
    }
    return c;
}

// Store role: the transposed tile in shared memory (buf as [k][TROW]) goes
// to the output layout; every thread owns line sl and writes k = k0, k0 + TL,
// ...  so a warp writes runs of Bg consecutive elements.  Count mode adds the
// points whose owner changes and the split-line amount (lbase: input offset
// of every tile line).
template <typename Real, int N, int TC, int THR, int RP = 0>
__device__ __forceinline__ void store_tile(const PassArgs &a, const typename PassCfg<Real, N, TC, THR, RP>::C *buf,
                                           const int64_t *lbase, const TileCoord &c, const int tid) {
    using Cfg = PassCfg<Real, N, TC, THR, RP>;
    using C = typename Cfg::C;
    C *out = reinterpret_cast<C *>(a.out);
    const bool active = tid < Cfg::THREADS;
    const int sl = tid % Cfg::LINES, k0 = tid / Cfg::LINES;
    int sbg, sbh;
    tile_line(a, sl, sbg, sbh);
    const bool sok = active && sl < a.Bg * a.Bh && c.g0 + sbg < a.Ng && c.h0 + sbh < a.Nh;
    unsigned long long moved = 0, split = 0;
    if (a.line_store) {  // the output keeps f fastest: every line is stored whole, k fastest across lanes
        const bool plain = !(a.conj & 2) && !a.scaled;
        const Real sc = plain ? (Real)1 : (Real)a.scale, sy = (a.conj & 2) ? -sc : sc;
        for (int e = tid; e < Cfg::LINES * N && active; e += Cfg::THREADS) {
            const int l = e / N, k = e % N;
            int bg, bh;
            tile_line(a, l, bg, bh);
            if (l < a.Bg * a.Bh && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh) {
                const int64_t o = c.out_base + bh * a.out_sh + bg * a.out_sg + k;
                const C v = buf[k * Cfg::TROW + l];
                out[o] = plain ? v : C{v.x * sc, v.y * sy};
                if (a.moved) {
                    moved += owner_of(a.own_in, lbase[l] + k) != owner_of(a.own_out, o);
                    if (k == 0)
                        split += (unsigned long long)N *
                                ((owner_of(a.own_in, lbase[l] + N - 1) - owner_of(a.own_in, lbase[l])) /
                                 a.own_in.line_div);
                }
            }
        }
    } else if (sok) {
        const int64_t obase = c.out_base + sbh * a.out_sh + sbg * a.out_sg;
        C *op = out + obase + (int64_t)k0 * a.out_sf;
        const int64_t ostep = (int64_t)Cfg::TL * a.out_sf;
        const C *bp = buf + k0 * Cfg::TROW + sl;
        if (!(a.conj & 2) && !a.scaled) {  // all passes but the last of an inverse
            if constexpr (N % Cfg::TL == 0) {  // N / TL elements per thread: a loop of fixed trip count
#pragma unroll
                for (int i = 0; i < N / Cfg::TL; ++i, op += ostep) *op = bp[i * Cfg::TL * Cfg::TROW];
            } else {
#pragma unroll 4
                for (int k = k0; k < N; k += Cfg::TL, op += ostep, bp += Cfg::TL * Cfg::TROW) *op = *bp;
            }
        } else {
            const Real sc = (Real)a.scale, sy = (a.conj & 2) ? -sc : sc;
#pragma unroll 4
            for (int k = k0; k < N; k += Cfg::TL, op += ostep, bp += Cfg::TL * Cfg::TROW) {
                const C v = *bp;
                *op = C{v.x * sc, v.y * sy};
            }
        }
        if (a.moved) {  // count mode: owner of the point before and after the store
            const int64_t ib = lbase[sl];
            for (int k = k0; k < N; k += Cfg::TL)
                moved += owner_of(a.own_in, ib + k) != owner_of(a.own_out, obase + k * a.out_sf);
            if (k0 == 0)
                split = (unsigned long long)N *
                        ((owner_of(a.own_in, ib + N - 1) - owner_of(a.own_in, ib)) / a.own_in.line_div);
        }
    }
    if (a.moved) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            moved += __shfl_down_sync(0xffffffffu, moved, o);
            split += __shfl_down_sync(0xffffffffu, split, o);
        }
        if ((tid & 31) == 0) {
            if (moved) atomicAdd(a.moved, moved);
            if (split) atomicAdd(a.split, split);
        }
    }
}

// The whole pass for one tile of lines.  Threads tid >= THREADS (a CTA shared
// by several line lengths, see the grouped serving kernel) take part in the
// barriers only.  (Tensor-core plans use the persistent kernel of
// tc_pass.cuh instead.)
template <typename Real, int N, int TC, int THR = 0, int RP = 0>
__device__ __forceinline__ void pass_tile(const PassArgs &a, int64_t t, unsigned char *smem_raw, const int tid) {
    using Cfg = PassCfg<Real, N, TC, THR, RP>;
    using C = typename Cfg::C;
    C *buf = reinterpret_cast<C *>(smem_raw);  // stage buffer [LINES][PADN] / transposed tile [N][TROW]
    C *tw = buf + Cfg::DATA;
    int64_t *lbase = reinterpret_cast<int64_t *>(tw + Cfg::TWN + Cfg::BFRAG);  // input offset of each tile line
    TileCoord *shc = reinterpret_cast<TileCoord *>(lbase + Cfg::LINES);
    const bool active = tid < Cfg::THREADS;

    const C *in = reinterpret_cast<const C *>(a.in);
    const C *gtw = reinterpret_cast<const C *>(a.tw);

    // warp 0 alone turns the tile index into coordinates (64-bit divisions)
    // and the lines' input offsets; the other warps read them after the barrier
    if (tid < 32) {
        const TileCoord w0 = tile_coords(a, t);
        if (tid == 0) *shc = w0;
        for (int l = tid; l < Cfg::LINES; l += 32) {
            int bg, bh;
            tile_line(a, l, bg, bh);
            lbase[l] = w0.in_base + bg * a.in_sg + bh * a.in_sh;
        }
    }
    if (active)
        for (int q = tid; q < tw_entries(Cfg::plan); q += Cfg::THREADS) tw[q] = gtw[q];
    __syncthreads();
    const TileCoord c = *shc;

    // FFT role: thread (line, t) with t fastest
    const int line = tid / Cfg::TL, tl = tid % Cfg::TL;
    int fbg, fbh;
    tile_line(a, line, fbg, fbh);
    const bool fok = active && line < a.Bg * a.Bh && c.g0 + fbg < a.Ng && c.h0 + fbh < a.Nh;

    if constexpr (!Cfg::DIRECT) {  // stage the whole tile through shared memory
        if (active) {
            for (int e = tid; e < Cfg::LINES * N; e += Cfg::THREADS) {
                const int l = e / N, i = e % N;
                int bg, bh;
                tile_line(a, l, bg, bh);
                if (l < a.Bg * a.Bh && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh) {
                    C x = in[lbase[l] + i];
                    if (a.conj & 1) x.y = -x.y;
                    buf[l * Cfg::PADN + padg<Cfg::PADG>(i)] = x;
                }
            }
        }
        __syncthreads();
    }
    if constexpr (Cfg::plan.S == 0) {  // length-1 lines: the DFT is the identity
        C v = C{0, 0};
        if (active) v = buf[line * Cfg::PADN];
        __syncthreads();
        if (active) buf[line] = v;  // tile[k = 0][line]
        __syncthreads();
    } else {
        const C *gsrc = in + lbase[line < Cfg::LINES ? line : 0];
        Stages<Real, N, 0, 1, TC, THR, -1, RP>::run(buf, buf, tw, gsrc, line, tl, fok, (a.conj & 1) != 0, active);
    }
    store_tile<Real, N, TC, THR, RP>(a, buf, lbase, c, tid);
}

// ------------------------------------------------------------------ the kernel

template <typename Real, int N, int TC = 0, int THR = 0, int RP = 0>
__global__ void __launch_bounds__(PassCfg<Real, N, TC, THR, RP>::THREADS) fft_pass_kernel(const PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pass_tile<Real, N, TC, THR, RP>(a, blockIdx.x, smem_raw, threadIdx.x);
}

// The same kernel with a register cap for MINB resident CTAs per SM (more
// warps in flight for short lines; some registers spill): an autotuning variant.
template <int N, int MINB>
__global__ void __launch_bounds__(PassCfg<float, N>::THREADS, MINB) fft_pass_occ_kernel(const PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pass_tile<float, N, 0, 0, 0>(a, blockIdx.x, smem_raw, threadIdx.x);
}

}  // namespace mdfft
