// fft_ring.cuh -- persistent complex64 pass kernel that streams its tiles
// through a ring of S shared-memory slots filled by 16-byte asynchronous
// copies (cp.async), so that the loads of the next S - 1 tiles are in flight
// while a tile is transformed and stored.
//
// The same pass as fft_pass_kernel (the Fig. 4 step and the transpose after
// it): same CTA shape, tiles, radix stages and store, so the results are
// bit-identical; only where the first stage reads from differs.  Short lines
// (a few hundred bytes) make a tile's work between its loads and its barriers
// small, and one tile's loads per CTA are then too few bytes in flight to
// keep HBM busy; the ring keeps (S - 1) tiles' loads outstanding per CTA, and
// the host caps the resident CTAs per SM (PassKernel::per_sm).
//
// Each thread owns one line of every tile (line = tid / TL) for the copies
// and the first stage, so its line's input offset is fixed up to the tile's
// base; slot rows are the line padded to ring_row_stride() elements.
// A tile's copies form one commit group: waiting until at most S - 1 groups
// are pending leaves the oldest (this tile's) complete; a CTA barrier (B1)
// then makes every thread's copies visible.  The stages write the transposed
// tile into a buffer of its own, closed by a second CTA barrier (B2), and the
// store reads it; two CTA barriers per tile.  Hazards, for tile i:
//  - the slot of tile i is refilled when tile i + 1 is issued, after B2(i),
//    by which every warp has finished its first stage;
//  - the stage buffer and the transposed tile of tile i + 1 are written after
//    B1(i + 1), which every thread reaches only after its store of tile i;
//  - the tile coordinates and line offsets of tile i (read by the store
//    role) live in a ring of S + 1 entries: the issue of tile i + S at the top
//    of iteration i + 1 may run while other threads still store tile i, and
//    writes entry (i + S) mod (S + 1), which is not tile i's.
// No wait spins: cp.async.wait_group returns when the thread's own copies
// have landed.
#pragma once

#include "fft_pass.cuh"

namespace mdfft {

__device__ __forceinline__ void ring_copy16(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void ring_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING> __device__ __forceinline__ void ring_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Row stride (complex64 elements) of a ring slot: N padded by an even count
// (rows stay whole 16-byte units) chosen so that the first stage's reads --
// thread (line, t) reads element j + r N/R0 of its line, j = t + i TL -- fall
// on distinct 8-byte bank pairs within each half-warp as far as a padding of
// at most 14 allows (cost: the sum over the read instructions of the largest
// number of distinct addresses on one bank pair).
template <int N, int RP> constexpr int ring_row_stride() {
    using Cfg = PassCfg<float, N, 0, 0, RP>;
    constexpr int R0 = Cfg::plan.R[0], NB = N / R0, TL = Cfg::TL;
    constexpr int PER = (NB + TL - 1) / TL;
    int best = N, best_cost = 1 << 30;
    for (int pad = 0; pad <= 14; pad += 2) {
        const int rs = N + pad;
        int cost = 0;
        for (int h = 0; h < 2; ++h)
            for (int i = 0; i < PER; ++i)
                for (int r = 0; r < R0; ++r) {
                    int addr[16] = {}, n = 0;
                    for (int q = 0; q < 16; ++q) {
                        const int tid = 16 * h + q, line = tid / TL, t = tid % TL, j = t + i * TL;
                        if (j < NB && line < Cfg::LINES) addr[n++] = rs * line + j + r * NB;
                    }
                    int worst = 0;
                    for (int b = 0; b < 16; ++b) {
                        int cnt = 0;
                        for (int x = 0; x < n; ++x) {
                            if (addr[x] % 16 != b) continue;
                            bool seen = false;
                            for (int y = 0; y < x; ++y) seen = seen || addr[y] == addr[x];
                            cnt += seen ? 0 : 1;
                        }
                        worst = cnt > worst ? cnt : worst;
                    }
                    cost += worst;
                }
        if (cost < best_cost) best_cost = cost, best = rs;
    }
    return best;
}

template <int N, int S, int RP = 0> struct RingCfg {
    using Cfg = PassCfg<float, N, 0, 0, RP>;
    static_assert(N % 2 == 0, "ring slots are filled in 16-byte units (two complex64)");
    static_assert(S >= 2 && S <= 4, "ring depth");
    static constexpr int RS = ring_row_stride<N, RP>();
    static constexpr int CH = N / 2;                       // 16-byte units per line
    static constexpr int CPT = (CH + Cfg::TL - 1) / Cfg::TL;  // units per thread
    static constexpr int SLOT = Cfg::LINES * RS;           // elements per slot
    static constexpr int TILE = N * Cfg::TROW;             // transposed tile [N][TROW]
    static constexpr int META = 4 + Cfg::LINES;            // int64 per tile: coordinates, line offsets
    // slots, stage buffer, transposed tile, twiddles, then S + 1 entries of
    // tile coordinates (4 int64) and the input offset of every line
    static constexpr size_t SMEM = (size_t)(S * SLOT + Cfg::DATA + TILE + Cfg::TWN) * sizeof(float2) +
                                   (size_t)(S + 1) * META * sizeof(int64_t);
};

template <int N, int S, int RP = 0>
__global__ void __launch_bounds__(PassCfg<float, N, 0, 0, RP>::THREADS) fft_pass_ring_kernel(const PassArgs a) {
    using Cfg = PassCfg<float, N, 0, 0, RP>;
    using RC = RingCfg<N, S, RP>;
    using C = float2;
    extern __shared__ __align__(16) unsigned char ring_smem[];
    C *slots = reinterpret_cast<C *>(ring_smem);
    C *buf = slots + S * RC::SLOT;  // stage buffer [LINES][PADN]
    C *tile = buf + Cfg::DATA;      // transposed tile [N][TROW]
    C *tw = tile + RC::TILE;
    int64_t *meta = reinterpret_cast<int64_t *>(tw + Cfg::TWN);  // S + 1 x (TileCoord, LINES offsets)
    const int tid = threadIdx.x;
    const int line = tid / Cfg::TL, tl = tid % Cfg::TL;
    int bg, bh;
    tile_line(a, line, bg, bh);
    const bool lok = line < a.Bg * a.Bh;
    const int64_t loff = (int64_t)bg * a.in_sg + (int64_t)bh * a.in_sh;
    const C *in = reinterpret_cast<const C *>(a.in);
    const C *gtw = reinterpret_cast<const C *>(a.tw);
    const bool conj = (a.conj & 1) != 0;
    const int64_t G = gridDim.x;

    // tile t's lines into slot `slot`, its coordinates and line offsets into
    // meta entry e (one commit group per call, empty past the last tile);
    // every thread computes the coordinates itself (warp 0 alone, one
    // iteration ahead, measured slower: it lengthens warp 0's part of the tile)
    auto issue = [&](int64_t t, int slot, int e) {
        if (t < a.ntiles) {
            const TileCoord c = tile_coords(a, t);
            int64_t *m = meta + e * RC::META;
            if (tid == 0) *reinterpret_cast<TileCoord *>(m) = c;
            if (tl == 0) m[4 + line] = c.in_base + loff;
            if (lok && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh) {
                const C *src = in + c.in_base + loff;
                C *dst = slots + slot * RC::SLOT + line * RC::RS;
#pragma unroll
                for (int i = 0; i < RC::CPT; ++i) {
                    const int u = tl + i * Cfg::TL;
                    if (RC::CH % Cfg::TL == 0 || u < RC::CH) ring_copy16(dst + 2 * u, src + 2 * u);
                }
            }
        }
        ring_commit();
    };

    for (int q = tid; q < tw_entries(Cfg::plan); q += Cfg::THREADS) tw[q] = gtw[q];
#pragma unroll
    for (int s = 0; s < S - 1; ++s) issue(blockIdx.x + s * G, s, s);
    int slot = 0, e = 0;  // tile i's slot (i mod S) and meta entry (i mod (S + 1))
    for (int64_t t = blockIdx.x; t < a.ntiles; t += G) {
        // tile i + S - 1 into the slot tile i - 1 used, meta entry (i + S - 1) mod (S + 1)
        issue(t + (S - 1) * G, slot == 0 ? S - 1 : slot - 1, (e + S - 1) % (S + 1));
        ring_wait<S - 1>();
        __syncthreads();  // B1: every thread's copies of tile i (on the first tile also the twiddles)
        const int64_t *m = meta + e * RC::META;
        const TileCoord c = *reinterpret_cast<const TileCoord *>(m);
        const bool ok = lok && c.g0 + bg < a.Ng && c.h0 + bh < a.Nh;
        // the last stage ends with B2 (the transposed tile complete)
        Stages<float, N, 0, 1, 0, 0, 3, RP>::run(buf, tile, tw, slots + slot * RC::SLOT + line * RC::RS, line, tl,
                                                 ok, conj, true);
        store_tile<float, N, 0, 0, RP>(a, tile, m + 4, c, tid);
        slot = slot + 1 == S ? 0 : slot + 1;
        e = e == S ? 0 : e + 1;
    }
    ring_wait<0>();  // nothing in flight at exit (the copies past the last tile are empty groups)
}

}  // namespace mdfft
