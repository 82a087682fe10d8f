// mdfft.cu -- C ABI of libmdfft (see include/mdfft.h).
//
// A plan holds the transpose order, one fused pass per step of Fig. 4
// (Duy and Ozaki, arXiv:1302.6189) and the device resources the passes use:
// twiddle tables made in FP64 on the device and one workspace array.  Pass s
// reads layout s, transforms its last axis and stores layout s+1 (natural
// order after the last step).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "plan_internal.h"

using mdfft::PassArgs;
using mdfft::PassKernel;
using mdfft::detail::Pass;
namespace pl = mdfft::planner;

namespace {
thread_local std::string g_err;
}  // namespace

namespace mdfft {
namespace detail {

mdfft_status fail(mdfft_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

mdfft_status cuda_fail(cudaError_t e, const char *what) {
    return fail(MDFFT_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace detail
}  // namespace mdfft

using mdfft::detail::cuda_fail;
using mdfft::detail::fail;

namespace {

// strides of every natural axis in layout L
void layout_strides(const pl::Layout &L, const int64_t *N, int64_t *stride) {
    int64_t s = 1;
    for (int i = L.M - 1; i >= 0; --i) {
        stride[L.axis[i]] = s;
        s *= N[L.axis[i]];
    }
}

// tile32 and the multiply-shift divisors of the tile decomposition (after any change of the tiling)
void set_tile_divisors(PassArgs &a, int64_t ctas) {
    a.fd_bg = mdfft::fastdiv_make((uint32_t)a.Bg);
    a.tile32 = ctas <= 0xffffffffLL;
    if (!a.tile32) return;
    a.fd_g = mdfft::fastdiv_make((uint32_t)a.gblocks);
    a.fd_h = mdfft::fastdiv_make((uint32_t)a.hblocks);
    for (int i = 0; i < a.nrest; ++i) a.fd_rest[i] = mdfft::fastdiv_make((uint32_t)a.rest_count[i]);
}

mdfft::OwnerMap owner_map(int M, const int64_t *N, int64_t P, const pl::Layout &L) {
    int64_t d[pl::kMaxDims];
    pl::layout_dims(L, N, d);
    int k = pl::regime(M, d, P);
    mdfft::OwnerMap m{1, 1, P, nullptr, 0, 1};
    for (int i = 0; i < M; ++i) (i < k ? m.lead : m.tail) *= d[i];
    return m;
}

// Owner tables of a comparison method (OwnerMap::blk): table t < M is layout
// t with the ownership of step t, table M the natural layout with the
// ownership of the last step; each holds d, q, ps per layout position.
std::vector<int64_t> owner_tables(const mdfft_plan_s *p) {
    std::vector<int64_t> tab;
    if (p->bd.kind == pl::kRowwise) return tab;
    const int M = p->M;
    tab.resize((size_t)(M + 1) * 3 * M);
    for (int t = 0; t <= M; ++t) {
        const int step = t < M ? t : M - 1;
        int64_t q[pl::kMaxDims], ps[pl::kMaxDims];
        pl::block_axis_grid(p->bd, M, step, q, ps);
        int64_t *row = &tab[(size_t)t * 3 * M];
        for (int i = 0; i < M; ++i) {
            const int ax = t < M ? p->order[t].axis[i] : i;
            row[i] = p->N[ax], row[M + i] = q[ax], row[2 * M + i] = ps[ax];
        }
    }
    return tab;
}

// Points the pass kernels' count mode at the owner tables (device copy at tab).
void set_block_owners(mdfft_plan_s *p, const int64_t *tab) {
    const int M = p->M;
    for (int s = 0; s < M; ++s) {
        PassArgs &a = p->pass[s].args;
        int64_t q[pl::kMaxDims], ps[pl::kMaxDims];
        pl::block_axis_grid(p->bd, M, s, q, ps);
        const int f = p->order[s].axis[M - 1];
        a.own_in = mdfft::OwnerMap{1, 1, p->P, tab + (size_t)s * 3 * M, M, q[f] > 1 ? ps[f] : 1};
        a.own_out = mdfft::OwnerMap{1, 1, p->P, tab + (size_t)(s + 1) * 3 * M, M, 1};
    }
}

// Kernel for a line length: the tensor-core dtypes use the tensor-core
// variant when the length is a multiple of 16 (radix-16 stages exist) and the
// FP32 SIMT kernel otherwise.
bool lookup(mdfft_dtype dt, int64_t n, PassKernel *k) {
    if (dt == MDFFT_C64) return mdfft::find_pass_kernel_c64(n, k);
    if (dt == MDFFT_C128) return mdfft::find_pass_kernel_c128(n, k);
    if (dt == MDFFT_C64_TC_FP16 || dt == MDFFT_C64_TC_BF16) {
        const int tc = dt == MDFFT_C64_TC_FP16 ? mdfft::kTcFp16 : mdfft::kTcBf16;
        if (mdfft::find_pass_kernel_tc(n, tc, k)) return true;
        return mdfft::find_pass_kernel_c64(n, k);
    }
    return false;
}

// Tile shape: Bg lines along g times Bh along h, at most `lines`, scored by
// the fraction of useful lines and by the length of the contiguous runs the
// store writes (a run of Bg elements; 128 bytes and more count as full).
void choose_tile(int lines, int64_t Ng, int64_t Nh, size_t elem, int *Bg, int *Bh) {
    double best = -1;
    for (int bg = 1; bg <= lines && bg <= Ng; ++bg) {
        int bh = (int)std::min<int64_t>(Nh, lines / bg);
        if (bh < 1) continue;
        double ug = (double)Ng / (double)(((Ng + bg - 1) / bg) * bg);
        double uh = (double)Nh / (double)(((Nh + bh - 1) / bh) * bh);
        double fill = (double)(bg * bh) / (double)lines;
        double coal = std::min(1.0, (double)bg * (double)elem / 128.0);
        double score = ug * uh * fill * coal;
        if (score > best + 1e-12) best = score, *Bg = bg, *Bh = bh;
    }
}

// Small grids: shrinks the tile of a built pass (along h first, then along g
// down to 128-byte store runs) until the pass fills about one resident wave of
// CTAs; idle lanes in a CTA cost less than idle SMs.  Updates the tile counts
// and ps.ctas (not the divisors); returns the wave.  No heap use.
int64_t shrink_to_wave(Pass &ps, size_t elem, bool line_store) {
    PassArgs &a = ps.args;
    const int64_t rest = ps.ctas / (a.gblocks * a.hblocks);
    const int64_t wave = mdfft::detail::wave_ctas(ps.k);
    const int min_bg = std::max(1, (int)(128 / elem));
    while (ps.ctas < wave && (a.Bh > 1 || (!line_store && a.Bg > min_bg))) {
        if (a.Bh > 1)
            a.Bh = (a.Bh + 1) / 2;
        else
            a.Bg = std::max(min_bg, (a.Bg + 1) / 2);
        a.gblocks = (a.Ng + a.Bg - 1) / a.Bg;
        a.hblocks = (a.Nh + a.Bh - 1) / a.Bh;
        ps.ctas = a.gblocks * a.hblocks * rest;
    }
    return wave;
}

// Launch arguments of pass s with the tile order `mapping` (kernel ps.k kept
// if set, else the default kernel of the length):
//  0  tiles of Bg lines consecutive along g, the output layout's fastest axis
//     (other than f), and Bh along h, its next axis; the rest of the axes
//     follow the output layout -- the store writes runs of Bg elements;
//  1  input-chunk order: g and h are the input layout's second and third
//     fastest axes and the rest follow the input layout, so consecutive
//     tiles are consecutive lines of layout s and a tile of whole f_MD chunks
//     (1-D and 2-D regimes) is exactly one chunk (CTA t owns chunk t); the
//     store then writes elements Bg apart by g's output stride.
// A pass that keeps f fastest in its output (lines stored whole) has only
// tile order 0.
mdfft_status layout_pass(const mdfft_plan_s *p, int s, int mapping, Pass &ps, bool keep_kernel = false) {
    const int M = p->M;
    const pl::Layout &L = p->order[s];
    pl::Layout nat;
    nat.M = M;
    for (int i = 0; i < M; ++i) nat.axis[i] = i;
    // the last pass stores natural order, or layout L_M itself (MDFFT_PLAN_OUT_LAST_LAYOUT)
    const pl::Layout &Lo = (s + 1 < M) ? p->order[s + 1] : (p->flags & MDFFT_PLAN_OUT_LAST_LAYOUT) ? L : nat;
    ps.f = L.axis[M - 1];
    ps.g = Lo.axis[M - 1];
    const bool line_store = ps.g == ps.f;  // output keeps f fastest: lines stored whole
    if (line_store && s + 1 < M) return fail(MDFFT_E_ORDER, "output layout keeps the transformed axis fastest");
    if (line_store && mapping != 0) return fail(MDFFT_E_ARG, "a pass that stores whole lines has tile order 0 only");
    if (mapping != 0 && mapping != 1) return fail(MDFFT_E_ARG, "tile order must be 0 or 1");
    if (line_store) ps.g = Lo.axis[M - 2];  // tile lines along the next axes of the layout
    const pl::Layout &Lt = mapping == 1 ? L : Lo;  // the layout the tiles follow
    if (mapping == 1) ps.g = M >= 2 ? L.axis[M - 2] : ps.f;
    ps.h = -1;
    for (int i = M - 2; i >= 0; --i)
        if (Lt.axis[i] != ps.f && Lt.axis[i] != ps.g) {
            ps.h = Lt.axis[i];
            break;
        }
    ps.mapping = mapping;
    ps.n = p->N[ps.f];
    if (!keep_kernel && !lookup(p->dt, ps.n, &ps.k))
        return fail(MDFFT_E_UNSUPPORTED, "line length " + std::to_string(ps.n) + " is not built for this dtype");

    int64_t sin_[pl::kMaxDims], sout[pl::kMaxDims];
    layout_strides(L, p->N, sin_);
    layout_strides(Lo, p->N, sout);
    PassArgs &a = ps.args;
    std::memset(&a, 0, sizeof(a));
    const int64_t Ng = p->N[ps.g], Nh = ps.h >= 0 ? p->N[ps.h] : 1;
    int Bg = 1, Bh = 1;
    choose_tile(ps.k.lines, Ng, Nh, p->elem, &Bg, &Bh);
    a.Bg = Bg, a.Bh = Bh, a.Ng = Ng, a.Nh = Nh;
    a.gblocks = (Ng + Bg - 1) / Bg;
    a.hblocks = (Nh + Bh - 1) / Bh;
    a.in_sg = sin_[ps.g];
    a.in_sh = ps.h >= 0 ? sin_[ps.h] : 0;
    a.out_sh = ps.h >= 0 ? sout[ps.h] : 0;
    a.out_sf = sout[ps.f];
    a.out_sg = sout[ps.g];
    a.line_store = line_store ? 1 : 0;
    if ((line_store ? sout[ps.f] : mapping == 0 ? sout[ps.g] : 1) != 1 || sin_[ps.f] != 1)
        return fail(MDFFT_E_ORDER, "internal: layout strides");
    // remaining axes, fastest first in the layout the tiles follow
    a.nrest = 0;
    ps.ctas = a.gblocks * a.hblocks;
    for (int i = M - 1; i >= 0; --i) {
        int ax = Lt.axis[i];
        if (ax == ps.f || ax == ps.g || ax == ps.h) continue;
        a.rest_count[a.nrest] = p->N[ax];
        a.rest_in[a.nrest] = sin_[ax];
        a.rest_out[a.nrest] = sout[ax];
        a.nrest++;
        ps.ctas *= p->N[ax];
    }
    if (p->batch > 1) {  // the transforms of a batch: one more axis, outermost, stride T in and out
        a.rest_count[a.nrest] = p->batch;
        a.rest_in[a.nrest] = p->T;
        a.rest_out[a.nrest] = p->T;
        a.nrest++;
        ps.ctas *= p->batch;
    }
    const int64_t wave = shrink_to_wave(ps, p->elem, line_store);
    set_tile_divisors(a, ps.ctas);
    a.own_in = owner_map(M, p->N, p->P, L);
    a.own_out = owner_map(M, p->N, p->P, Lo);
    a.scale = 1.0;
    a.scaled = 0;
    ps.grid = ps.k.persistent ? std::min<int64_t>(ps.ctas, wave) : ps.ctas;
    return MDFFT_OK;
}

mdfft_status build_pass(mdfft_plan_s *p, int s) { return layout_pass(p, s, 0, p->pass[s]); }

// Pass s run by kernel k with tile order m and tiles of Bg x Bh lines (the
// autotuner's candidates and stored tunings); the count mode's owner maps
// are those of the built pass.
mdfft_status candidate_pass(const mdfft_plan_s *p, int s, const PassKernel &k, int m, int Bg, int Bh, Pass &out) {
    Pass c = p->pass[s];
    c.k = k;
    mdfft_status st = layout_pass(p, s, m, c, true);
    if (st != MDFFT_OK) return st;
    PassArgs &a = c.args;
    a.own_in = p->pass[s].args.own_in;
    a.own_out = p->pass[s].args.own_out;
    if (Bg < 1 || Bh < 1 || (int64_t)Bg * Bh > k.lines || Bg > a.Ng || Bh > a.Nh)
        return fail(MDFFT_E_ARG, "tile shape does not fit the kernel or the pass");
    a.Bg = Bg, a.Bh = Bh;
    a.gblocks = (a.Ng + Bg - 1) / Bg;
    a.hblocks = (a.Nh + Bh - 1) / Bh;
    c.ctas = a.gblocks * a.hblocks;
    for (int i = 0; i < a.nrest; ++i) c.ctas *= a.rest_count[i];
    set_tile_divisors(a, c.ctas);
    c.grid = k.persistent ? std::min<int64_t>(c.ctas, mdfft::detail::wave_ctas(k)) : c.ctas;
    out = c;
    return MDFFT_OK;
}

// Twiddle table of one pass (layout of tw_offset in fft_pass.cuh): entry
// r * NS + k of stage s >= 1 is w_N^e, e = k r N / (NS R), w_N = exp(-2 pi i/N),
// computed in FP64 with sincospi and rounded to the pass precision.
}  // namespace

// Resident CTAs of kernel k on the whole GPU (the runtime's occupancy
// figure).  A persistent kernel launches exactly this many CTAs, so it asks
// for the largest shared-memory carveout (a property of the function) and the
// count is also worked out from its registers and shared memory against the
// SM's limits; the larger figure is used.  (The runtime reported one CTA per
// SM for the tensor-core kernels, whose limits allow three.)
int64_t mdfft::detail::wave_ctas(const PassKernel &k) {
    int dev = 0, sms = 1, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (k.smem > 48 * 1024) cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
    if (k.persistent && k.smem > 48 * 1024)
        cudaFuncSetAttribute(k.fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k.fn, k.threads, k.smem) != cudaSuccess) per = 0;
    if (!k.persistent) return (int64_t)sms * std::max(per, 1);
    cudaFuncAttributes fa;
    int smem_sm = 0, regs_sm = 0, thr_sm = 0, reserved = 0;
    if (cudaFuncGetAttributes(&fa, k.fn) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) {
        const int warps = (k.threads + 31) / 32;
        const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
        const int by_smem = smem_sm / (int)(k.smem + fa.sharedSizeBytes + reserved);
        const int by_regs = regs_warp > 0 ? regs_sm / (regs_warp * warps) : 32;
        const int by_thr = thr_sm / k.threads;
        per = std::max(per, std::min(by_smem, std::min(by_regs, by_thr)));
    }
    if (k.per_sm > 0) per = std::min(per, k.per_sm);
    return (int64_t)sms * std::max(per, 1);
}

void mdfft::detail::retile_pass(const mdfft_plan_s *p, int s, int lines, PassArgs *out, int64_t *ctas) {
    const Pass &ps = p->pass[s];
    PassArgs a = ps.args;
    int Bg = 1, Bh = 1;
    choose_tile(lines, a.Ng, a.Nh, p->elem, &Bg, &Bh);
    a.Bg = Bg, a.Bh = Bh;
    a.gblocks = (a.Ng + Bg - 1) / Bg;
    a.hblocks = (a.Nh + Bh - 1) / Bh;
    int64_t n = a.gblocks * a.hblocks;
    for (int i = 0; i < a.nrest; ++i) n *= a.rest_count[i];
    set_tile_divisors(a, n);
    *out = a;
    *ctas = n;
}

namespace {

__global__ void twiddle_kernel(void *dst, int64_t n, mdfft::RadixPlan plan, int dbl) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= mdfft::tw_entries(plan)) return;
    int64_t off = 0, ns = plan.R[0];
    for (int s = 1; s < plan.S; ++s) {
        const int64_t R = plan.R[s];
        if (q < off + ns * R) {
            const int64_t r = (q - off) / ns, k = (q - off) % ns;
            const int64_t e = (k * r * (n / (ns * R))) % n;
            double sv, cv;
            sincospi(-2.0 * (double)e / (double)n, &sv, &cv);
            if (dbl) reinterpret_cast<double2 *>(dst)[q] = make_double2(cv, sv);
            else reinterpret_cast<float2 *>(dst)[q] = make_float2((float)cv, (float)sv);
            return;
        }
        off += ns * R;
        ns *= R;
    }
}

// Twiddle table of pass s for radix plan `plan` (the plan of the pass's
// kernel), made on `st`.
void make_twiddles(const mdfft_plan_s *p, int s, const mdfft::RadixPlan &plan, cudaStream_t st) {
    const int entries = std::max(1, mdfft::tw_entries(plan));
    twiddle_kernel<<<(unsigned)((entries + 255) / 256), 256, 0, st>>>((char *)p->tw + p->pass[s].tw_offset,
                                                                      p->pass[s].n, plan, p->dt == MDFFT_C128);
}

bool same_plan(const mdfft::RadixPlan &a, const mdfft::RadixPlan &b) {
    if (a.S != b.S) return false;
    for (int i = 0; i < a.S; ++i)
        if (a.R[i] != b.R[i]) return false;
    return true;
}

mdfft_status parse_order(int M, const int *order, std::vector<pl::Layout> &out) {
    out.clear();
    for (int s = 0; s < M; ++s) {
        pl::Layout L;
        L.M = M;
        for (int i = 0; i < M; ++i) L.axis[i] = order[s * M + i];
        out.push_back(L);
    }
    std::string msg = pl::check_order(M, out);
    if (!msg.empty()) return fail(MDFFT_E_ORDER, msg);
    return MDFFT_OK;
}

void release(mdfft_plan_s *p) {
    if (!p) return;
    if (p->tw) cudaFree(p->tw);
    if (p->ws) cudaFree(p->ws);
    if (p->ws2) cudaFree(p->ws2);
    for (cudaEvent_t e : p->ev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t h : p->hs)
        if (h) cudaStreamDestroy(h);
    for (cudaEvent_t e : p->hev)
        if (e) cudaEventDestroy(e);
    for (auto &g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (p->capture) cudaStreamDestroy(p->capture);
    for (auto &b : p->dist_boxes)
        if (b.dev) cudaFree(b.dev);
    delete p;
}

bool overlaps(const void *a, const void *b, size_t n) {
    auto x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + n && y < x + n;
}

mdfft_status launch_passes(mdfft_plan_t p, const void *in, void *out, int dir, int normalize, cudaStream_t st,
                           int64_t *counts, int64_t v, bool allow_timing = true);

// Argument checks of an execution on device arrays (E_ARG with a message).
mdfft_status check_exec(mdfft_plan_t p, const void *in, const void *out, int dir, int normalize, const int64_t *counts) {
    if (!p) return fail(MDFFT_E_ARG, "null plan");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan cannot execute");
    if (p->external_ws) return fail(MDFFT_E_ARG, "plan has no workspace of its own");
    if (!in || !out) return fail(MDFFT_E_ARG, "null data pointer");
    if (dir != -1 && dir != 1) return fail(MDFFT_E_ARG, "dir must be -1 (forward) or +1 (inverse)");
    if (normalize != 0 && !(normalize == 1 && dir == 1))
        return fail(MDFFT_E_ARG, "normalize = 1 is only defined for the inverse");
    size_t align = p->dt == MDFFT_C128 ? 16 : 8;
    if ((uintptr_t)in % align || (uintptr_t)out % align) return fail(MDFFT_E_ARG, "misaligned data pointer");
    const size_t bytes = (size_t)p->T * p->batch * p->elem;
    const bool inplace = in == out;
    if (inplace && !(p->flags & MDFFT_PLAN_INPLACE))
        return fail(MDFFT_E_ARG, "in == out needs a plan made with MDFFT_PLAN_INPLACE");
    if (!inplace && overlaps(in, out, bytes)) return fail(MDFFT_E_ARG, "in and out overlap partially");
    if (counts && ((uintptr_t)counts % 8)) return fail(MDFFT_E_ARG, "misaligned counts pointer");
    for (int s = 0; s < p->M; ++s)  // pipelined passes copy whole 16-byte units
        if (p->pass[s].k.bulk && (((uintptr_t)in % 16) || ((uintptr_t)out % 16)))
            return fail(MDFFT_E_ARG, "tuned pass kernels read whole 16-byte units: align in and out to 16 bytes");
    return MDFFT_OK;
}

mdfft_status exec_impl(mdfft_plan_t p, const void *in, void *out, int dir, int normalize, mdfft_stream_t stream,
                       int64_t *counts) {
    mdfft_status cs = check_exec(p, in, out, dir, normalize, counts);
    if (cs != MDFFT_OK) return cs;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (counts) {
        cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * 2 * p->M, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    return launch_passes(p, in, out, dir, normalize, st, counts, -1);
}

// The M passes on `st`: of the whole batch (v < 0) or of transform v alone
// (the batch axis dropped, every array offset by v T elements; no timing).
mdfft_status launch_passes(mdfft_plan_t p, const void *in, void *out, int dir, int normalize, cudaStream_t st,
                           int64_t *counts, int64_t v, bool allow_timing) {
    const int M = p->M;
    const bool one = v >= 0 && p->batch > 1;
    const size_t off = v >= 0 ? (size_t)v * (size_t)p->T * p->elem : 0;
    auto at = [off](const void *b) { return b ? (void *)((char *)b + off) : nullptr; };
    // destination of every pass: the last one is `out`; going backwards the
    // buffers alternate so that no pass reads and writes the same array and
    // `in` is never written (unless in == out)
    void *dst[MDFFT_MAX_DIMS];
    dst[M - 1] = at(out);
    for (int s = M - 2; s >= 0; --s) dst[s] = (dst[s + 1] == at(out)) ? at(p->ws) : at(out);
    if (dst[0] == at(in)) dst[0] = at(p->ws2);  // in-place with an odd number of passes
    const void *src = at(in);
    const bool timed = p->timing && v < 0 && allow_timing;
    const int64_t slot = p->timed % MDFFT_TIMING_SLOTS;
    for (int s = 0; s < M; ++s) {
        Pass &ps = p->pass[s];
        PassArgs a = ps.args;
        int64_t grid = ps.grid;
        a.ntiles = ps.ctas;
        if (one) {  // the batch is the outermost tile axis
            a.nrest--;
            a.ntiles = ps.ctas / p->batch;
            grid = std::min<int64_t>(grid, a.ntiles);
        }
        a.in = src;
        a.out = dst[s];
        a.tw = (const char *)p->tw + ps.tw_offset;
        a.err = p->err;
        a.conj = dir == 1 ? (s == 0 ? 1 : 0) | (s == M - 1 ? 2 : 0) : 0;
        a.scale = (s == M - 1 && normalize) ? 1.0 / (double)p->T : 1.0;
        a.scaled = a.scale != 1.0;
        if (counts) {
            a.moved = reinterpret_cast<unsigned long long *>(counts + s);
            a.split = reinterpret_cast<unsigned long long *>(counts + M + s);
        }
        if (timed) cudaEventRecord(p->ev[slot * (M + 1) + s], st);
        void *args[] = {&a};
        cudaError_t e = cudaLaunchKernel(ps.k.fn, dim3((unsigned)grid), dim3(ps.k.threads), args, ps.k.smem, st);
        if (e != cudaSuccess) return cuda_fail(e, "pass launch");
        src = dst[s];
    }
    if (timed) {
        cudaEventRecord(p->ev[slot * (M + 1) + M], st);
        p->timed++;
    }
    return MDFFT_OK;
}

// mdfft_exec_host for a batch: transform v's copy in, passes and copy out go
// to three streams of the plan, so the copies of neighbouring transforms
// overlap each other and the passes (both copy directions and the SMs busy at
// once).  The transforms touch disjoint parts of every array; the caller's
// stream is forked at the start and joined at the end.
mdfft_status exec_host_pipelined(mdfft_plan_t p, const void *in_host, void *out_host, void *dev_in, void *dev_out,
                                 int dir, int normalize, cudaStream_t st) {
    mdfft_status cs = check_exec(p, dev_in, dev_out, dir, normalize, nullptr);
    if (cs != MDFFT_OK) return cs;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        if (!p->hs[i]) e = cudaStreamCreateWithFlags(&p->hs[i], cudaStreamNonBlocking);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        if (!p->hev[i]) e = cudaEventCreateWithFlags(&p->hev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline streams");
    cudaStream_t h2d = p->hs[0], comp = p->hs[1], d2h = p->hs[2];
    cudaEvent_t fork = p->hev[0], copied = p->hev[1], computed = p->hev[2], done = p->hev[3];
    const size_t vb = (size_t)p->T * p->elem;
    e = cudaEventRecord(fork, st);
    for (cudaStream_t h : p->hs)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h, fork, 0);
    for (int64_t v = 0; v < p->batch && e == cudaSuccess; ++v) {
        const size_t o = (size_t)v * vb;
        e = cudaMemcpyAsync((char *)dev_in + o, (const char *)in_host + o, vb, cudaMemcpyHostToDevice, h2d);
        if (e == cudaSuccess) e = cudaEventRecord(copied, h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(comp, copied, 0);
        if (e != cudaSuccess) break;
        mdfft_status r = launch_passes(p, dev_in, dev_out, dir, normalize, comp, nullptr, v);
        if (r != MDFFT_OK) return r;
        e = cudaEventRecord(computed, comp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(d2h, computed, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char *)out_host + o, (const char *)dev_out + o, vb, cudaMemcpyDeviceToHost, d2h);
    }
    if (e == cudaSuccess) e = cudaEventRecord(done, d2h);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, done, 0);
    if (e != cudaSuccess) return cuda_fail(e, "pipelined host execution");
    return MDFFT_OK;
}

// Drops the captured graphs of a plan (its launch arguments changed).
void drop_graphs(mdfft_plan_s *p) {
    for (auto &g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    p->graphs.clear();
}

constexpr size_t kMaxGraphs = 8;

mdfft_status exec_graph_impl(mdfft_plan_t p, const void *in, void *out, int dir, int normalize, cudaStream_t st) {
    mdfft_status cs = check_exec(p, in, out, dir, normalize, nullptr);
    if (cs != MDFFT_OK) return cs;
    mdfft_plan_s::GraphEntry *hit = nullptr;
    for (auto &g : p->graphs)
        if (g.in == in && g.out == out && g.dir == dir && g.normalize == normalize) hit = &g;
    if (!hit) {
        cudaError_t e = cudaSuccess;
        if (!p->capture) e = cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "capture stream");
        e = cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        mdfft_status r = launch_passes(p, in, out, dir, normalize, p->capture, nullptr, -1, false);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(p->capture, &graph);  // ends the capture whatever happened inside
        if (r != MDFFT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        if (p->graphs.size() >= kMaxGraphs) {  // replace the least recently used
            auto lru = p->graphs.begin();
            for (auto it = p->graphs.begin(); it != p->graphs.end(); ++it)
                if (it->used < lru->used) lru = it;
            cudaGraphExecDestroy(lru->exec);
            p->graphs.erase(lru);
        }
        mdfft_plan_s::GraphEntry g;
        g.in = in, g.out = out, g.dir = dir, g.normalize = normalize, g.exec = exec;
        p->graphs.push_back(g);
        hit = &p->graphs.back();
    }
    hit->used = ++p->graph_tick;
    cudaError_t e = cudaGraphLaunch(hit->exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return MDFFT_OK;
}

}  // namespace

extern "C" {

const char *mdfft_last_error(void) { return g_err.c_str(); }

mdfft_status mdfft_exec_graph(mdfft_plan_t p, const void *in, void *out, int dir, int normalize,
                              mdfft_stream_t stream) {
    return exec_graph_impl(p, in, out, dir, normalize, reinterpret_cast<cudaStream_t>(stream));
}

int mdfft_supported_length(int64_t n, mdfft_dtype dt) {
    PassKernel k;
    return lookup(dt, n, &k) ? 1 : 0;
}

mdfft_status mdfft_plan(mdfft_plan_t *out, int M, const int64_t N[], int64_t P, const int *order, mdfft_dtype dt,
                        unsigned flags) {
    return mdfft::detail::plan_create(out, M, N, P, order, dt, flags, true, 1);
}

mdfft_status mdfft_plan_batched(mdfft_plan_t *out, int M, const int64_t N[], int64_t P, const int *order,
                                mdfft_dtype dt, unsigned flags, int64_t batch) {
    return mdfft::detail::plan_create(out, M, N, P, order, dt, flags, true, batch);
}

}  // extern "C"

mdfft_status mdfft::detail::plan_create(mdfft_plan_t *out, int M, const int64_t N[], int64_t P, const int *order,
                                        mdfft_dtype dt, unsigned flags, bool with_workspace, int64_t batch) {
    g_err.clear();
    if (!out || !N) return fail(MDFFT_E_ARG, "null argument");
    *out = nullptr;
    if (batch < 1) return fail(MDFFT_E_ARG, "batch must be >= 1");
    if (M < 2 || M > MDFFT_MAX_DIMS) return fail(MDFFT_E_UNSUPPORTED, "M must be in [2, 8]");
    constexpr unsigned kDecomp = MDFFT_PLAN_DECOMP_SLAB | MDFFT_PLAN_DECOMP_PENCIL | MDFFT_PLAN_DECOMP_VOLUMETRIC;
    if (flags & ~(MDFFT_PLAN_HOST_ONLY | MDFFT_PLAN_INPLACE | MDFFT_PLAN_PERSISTENT | MDFFT_PLAN_OUT_LAST_LAYOUT |
                  MDFFT_PLAN_TUNE_RADIX |
                  kDecomp))
        return fail(MDFFT_E_ARG, "unknown flag");
    const unsigned decomp = flags & kDecomp;
    if (decomp & (decomp - 1)) return fail(MDFFT_E_ARG, "at most one MDFFT_PLAN_DECOMP_* flag");
    if (dt != MDFFT_C64 && dt != MDFFT_C128 && dt != MDFFT_C64_TC_FP16 && dt != MDFFT_C64_TC_BF16)
        return fail(MDFFT_E_ARG, "unknown dtype");
    mdfft_plan_s *p = new (std::nothrow) mdfft_plan_s;
    if (!p) return fail(MDFFT_E_NOMEM, "host allocation");
    p->M = M, p->P = P, p->dt = dt, p->flags = flags;
    p->elem = dt == MDFFT_C128 ? 16 : 8;
    unsigned __int128 T = 1;
    for (int i = 0; i < M; ++i) {
        if (N[i] < 1) {
            release(p);
            return fail(MDFFT_E_ARG, "dims must be >= 1");
        }
        p->N[i] = N[i];
        T *= (unsigned __int128)N[i];
    }
    if (T > ((unsigned __int128)1 << 40)) {
        release(p);
        return fail(MDFFT_E_ARG, "grid too large");
    }
    p->T = (int64_t)T;
    p->batch = batch;
    if (T * (unsigned __int128)batch > ((unsigned __int128)1 << 40)) {
        release(p);
        return fail(MDFFT_E_ARG, "batch too large");
    }
    if (P < 1 || P > p->T) {
        release(p);
        return fail(MDFFT_E_RANGE, "P must be in [1, N_1 ... N_M]");
    }
    mdfft_status st;
    if (order) {
        if ((st = parse_order(M, order, p->order)) != MDFFT_OK) {
            release(p);
            return st;
        }
    } else {
        int64_t total;
        std::string err;
        // the exact search up to 6 dims (6: when affordable), else the balanced-split heuristic
        bool ok = M <= 6 && pl::search_order(M, p->N, P, false, p->order, total, err);
        if (!ok && M == 6 && err.rfind("the exact order search is too large", 0) == 0) err.clear();
        if (!ok && err.empty()) ok = pl::heuristic_order(M, p->N, P, p->order, total, err);
        if (!ok) {
            release(p);
            return fail(MDFFT_E_UNSUPPORTED, "order search: " + err);
        }
    }
    if (decomp) {
        const int kind = decomp == MDFFT_PLAN_DECOMP_SLAB     ? pl::kSlab
                         : decomp == MDFFT_PLAN_DECOMP_PENCIL ? pl::kPencil
                                                              : pl::kVolumetric;
        std::string err;
        if (!pl::block_decomposition(M, p->N, P, kind, p->order, p->bd, err)) {
            release(p);
            return fail(MDFFT_E_RANGE, err);
        }
    }
    const bool host_only = flags & MDFFT_PLAN_HOST_ONLY;
    if (!host_only) {
        // every axis is transformed once: its line length must be built
        for (int i = 0; i < M; ++i) {
            PassKernel k;
            const int64_t n = p->N[i];
            if (!lookup(dt, n, &k)) {
                release(p);
                return fail(MDFFT_E_UNSUPPORTED, "line length " + std::to_string(n) + " is not built");
            }
        }
        for (int s = 0; s < M; ++s)
            if ((st = build_pass(p, s)) != MDFFT_OK) {
                release(p);
                return st;
            }
        if ((flags & MDFFT_PLAN_PERSISTENT) && dt == MDFFT_C64)
            for (int s = 0; s < M; ++s) {  // same tile shape: the pipelined kernel has the default's lines
                PassKernel k;
                if (mdfft::find_pass_kernel_pipe(p->pass[s].n, 1, &k) && k.lines == p->pass[s].k.lines) {
                    p->pass[s].k = k;
                    p->pass[s].grid = std::min<int64_t>(p->pass[s].ctas, mdfft::detail::wave_ctas(k));
                }
            }
        // twiddle tables: one per pass, 256-byte aligned inside one allocation,
        // each with room for the table of any radix plan of its length (fewer
        // than 2 n entries) so that autotuning can switch plans
        size_t off = 0;
        for (int s = 0; s < M; ++s) {
            p->pass[s].tw_offset = off;
            const size_t entries = std::max<size_t>(2 * (size_t)p->pass[s].n, mdfft::tw_entries(p->pass[s].k.plan));
            off += (entries * p->elem + 255) / 256 * 256;
        }
        p->tw_bytes = off;
        // + the device error flag, + the owner tables of a comparison method
        const std::vector<int64_t> owners = owner_tables(p);
        cudaError_t e = cudaMalloc(&p->tw, off + 256 + owners.size() * sizeof(int64_t));
        if (e != cudaSuccess) {
            release(p);
            return cuda_fail(e, "cudaMalloc twiddles");
        }
        p->err = reinterpret_cast<int *>((char *)p->tw + off);
        cudaMemset(p->err, 0, sizeof(int));
        if (!owners.empty()) {
            const int64_t *tab = reinterpret_cast<const int64_t *>((char *)p->tw + off + 256);
            e = cudaMemcpy((void *)tab, owners.data(), owners.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                release(p);
                return cuda_fail(e, "owner tables");
            }
            set_block_owners(p, tab);
        }
        for (int s = 0; s < M; ++s) make_twiddles(p, s, p->pass[s].k.plan, nullptr);
        const size_t bytes = (size_t)p->T * p->batch * p->elem;
        p->external_ws = !with_workspace;
        if (with_workspace && (e = cudaMalloc(&p->ws, bytes)) != cudaSuccess) {
            release(p);
            return cuda_fail(e, "cudaMalloc workspace");
        }
        if (with_workspace && (flags & MDFFT_PLAN_INPLACE) && (M % 2 == 1)) {
            if ((e = cudaMalloc(&p->ws2, bytes)) != cudaSuccess) {
                release(p);
                return cuda_fail(e, "cudaMalloc second workspace");
            }
        }
        for (int s = 0; s < M; ++s) {
            const PassKernel &k = p->pass[s].k;
            if (k.smem > 48 * 1024) {
                e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
                if (e != cudaSuccess) {
                    release(p);
                    return cuda_fail(e, "cudaFuncSetAttribute");
                }
            }
        }
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) {  // twiddles ready for any stream
            release(p);
            return cuda_fail(e, "twiddle generation");
        }
    }
    *out = p;
    return MDFFT_OK;
}

extern "C" {

mdfft_status mdfft_exec(mdfft_plan_t p, const void *in, void *out, int dir, int normalize, mdfft_stream_t stream) {
    return exec_impl(p, in, out, dir, normalize, stream, nullptr);
}

mdfft_status mdfft_exec_counted(mdfft_plan_t p, const void *in, void *out, int dir, int normalize,
                                mdfft_stream_t stream, int64_t *counts_dev) {
    if (!counts_dev) return fail(MDFFT_E_ARG, "null counts pointer");
    return exec_impl(p, in, out, dir, normalize, stream, counts_dev);
}

mdfft_status mdfft_comm_volume(mdfft_plan_t p, mdfft_comm *out) {
    if (!p || !out) return fail(MDFFT_E_ARG, "null argument");
    if (!p->comm_ready) {
        mdfft_comm c;
        std::memset(&c, 0, sizeof(c));
        const int M = p->M;
        pl::Layout nat;
        nat.M = M;
        for (int i = 0; i < M; ++i) nat.axis[i] = i;
        const bool rowwise = p->bd.kind == pl::kRowwise;
        for (int s = 0; s + 1 < M; ++s) {
            c.per_transition[s] = rowwise ? pl::transition_amount(M, p->N, p->P, p->order[s], p->order[s + 1])
                                          : pl::block_transition_amount(M, p->N, p->P, p->bd, s);
            c.total += c.per_transition[s];
        }
        c.final_to_natural = rowwise && !(p->flags & MDFFT_PLAN_OUT_LAST_LAYOUT)
                                 ? pl::transition_amount(M, p->N, p->P, p->order[M - 1], nat)
                                 : 0;
        c.paper_total = c.total;
        for (int s = 0; s < M; ++s) {
            c.split_line[s] = rowwise ? pl::split_line_amount(M, p->N, p->P, p->order[s])
                                      : pl::block_split_amount(M, p->N, p->bd, p->order, s);
            c.paper_total += c.split_line[s];
            int64_t d[pl::kMaxDims];
            pl::layout_dims(p->order[s], p->N, d);
            c.regime[s] = rowwise ? pl::regime(M, d, p->P) : p->bd.k;
        }
        // Sec. 4 closed forms for the same T and Np
        const double T = (double)p->T, P = (double)p->P, nan = std::nan("");
        bool cubic = true;
        for (int i = 1; i < M; ++i) cubic = cubic && p->N[i] == p->N[0];
        const double n = (double)p->N[0];
        c.amount_slab = T - T / P;
        c.amount_pencil = (cubic && M == 3) ? 2.0 * n * n * n - 2.0 * P * std::pow(n * n / P, 1.5) : nan;
        c.amount_volumetric = cubic ? (double)M * T * (n / std::pow(T / P, 1.0 / (double)M) - 1.0) : nan;
        p->comm = c;
        p->comm_ready = true;
    }
    *out = p->comm;
    return MDFFT_OK;
}

mdfft_status mdfft_chunk(mdfft_plan_t p, int step, int64_t pid, int64_t *xs, int64_t *xe, int64_t start_coord[],
                         int64_t end_coord[]) {
    if (!p || !xs || !xe) return fail(MDFFT_E_ARG, "null argument");
    if (step < 0 || step > p->M) return fail(MDFFT_E_ARG, "step out of range");
    if (pid < 0 || pid >= p->P) return fail(MDFFT_E_ARG, "pid out of range");
    if (p->bd.kind != pl::kRowwise) return fail(MDFFT_E_ARG, "f_MD chunks belong to row-wise plans");
    pl::Layout L;
    L.M = p->M;
    for (int i = 0; i < p->M; ++i) L.axis[i] = step < p->M ? p->order[step].axis[i] : i;
    int64_t d[pl::kMaxDims];
    pl::layout_dims(L, p->N, d);
    *xs = pl::fmd(p->M, d, p->P, pid);
    *xe = pl::fmd(p->M, d, p->P, pid + 1) - 1;
    if (start_coord) pl::digits(p->M, d, *xs, start_coord);
    if (end_coord) pl::digits(p->M, d, *xe, end_coord);
    return MDFFT_OK;
}

mdfft_status mdfft_exchange_counts(mdfft_plan_t p, int step, int G, int64_t *counts) {
    if (!p || !counts) return fail(MDFFT_E_ARG, "null argument");
    if (step < 0 || step >= p->M) return fail(MDFFT_E_ARG, "step out of range");
    if (G < 1 || G > p->P) return fail(MDFFT_E_ARG, "G must be in [1, P]");
    if (p->bd.kind != pl::kRowwise) return fail(MDFFT_E_ARG, "exchange counts are for row-wise plans");
    pl::Layout nat;
    nat.M = p->M;
    for (int i = 0; i < p->M; ++i) nat.axis[i] = i;
    const pl::Layout &A = p->order[step];
    const pl::Layout &B = step + 1 < p->M ? p->order[step + 1] : nat;
    pl::exchange_counts(p->M, p->N, p->P, A, B, G, counts);
    return MDFFT_OK;
}

mdfft_status mdfft_block_grid(mdfft_plan_t p, int step, int64_t *q_axis) {
    if (!p || !q_axis) return fail(MDFFT_E_ARG, "null argument");
    if (p->bd.kind == pl::kRowwise) return fail(MDFFT_E_ARG, "row-wise plan: no block grid");
    if (step < 0 || step >= p->M) return fail(MDFFT_E_ARG, "step out of range");
    int64_t ps[pl::kMaxDims];
    pl::block_axis_grid(p->bd, p->M, step, q_axis, ps);
    return MDFFT_OK;
}

mdfft_status mdfft_plan_order(mdfft_plan_t p, int *order_out) {
    if (!p || !order_out) return fail(MDFFT_E_ARG, "null argument");
    for (int s = 0; s < p->M; ++s)
        for (int i = 0; i < p->M; ++i) order_out[s * p->M + i] = p->order[s].axis[i];
    return MDFFT_OK;
}

mdfft_status mdfft_order_search(int M, const int64_t N[], int64_t P, int want_worst, int *order_out, int64_t *total) {
    if (!N || !order_out || !total) return fail(MDFFT_E_ARG, "null argument");
    if (M < 2 || M > 6) return fail(MDFFT_E_UNSUPPORTED, "order search supports 2 <= M <= 6");
    int64_t T = 1;
    for (int i = 0; i < M; ++i) {
        if (N[i] < 1) return fail(MDFFT_E_ARG, "dims must be >= 1");
        T *= N[i];
    }
    if (P < 1 || P > T) return fail(MDFFT_E_RANGE, "P must be in [1, N_1 ... N_M]");
    std::vector<pl::Layout> order;
    std::string err;
    if (!pl::search_order(M, N, P, want_worst != 0, order, *total, err))
        return fail(err.rfind("the exact order search is too large", 0) == 0 ? MDFFT_E_UNSUPPORTED : MDFFT_E_ARG, err);
    for (int s = 0; s < M; ++s)
        for (int i = 0; i < M; ++i) order_out[s * M + i] = order[s].axis[i];
    return MDFFT_OK;
}

mdfft_status mdfft_order_heuristic(int M, const int64_t N[], int64_t P, int *order_out, int64_t *total) {
    if (!N || !order_out || !total) return fail(MDFFT_E_ARG, "null argument");
    std::vector<pl::Layout> order;
    std::string err;
    if (M < 2 || M > MDFFT_MAX_DIMS) return fail(MDFFT_E_UNSUPPORTED, "M must be in [2, 8]");
    int64_t T = 1;
    for (int i = 0; i < M; ++i) {
        if (N[i] < 1) return fail(MDFFT_E_ARG, "dims must be >= 1");
        T *= N[i];
    }
    if (P < 1 || P > T) return fail(MDFFT_E_RANGE, "P must be in [1, N_1 ... N_M]");
    if (!pl::heuristic_order(M, N, P, order, *total, err)) return fail(MDFFT_E_ARG, err);
    for (int s = 0; s < M; ++s)
        for (int i = 0; i < M; ++i) order_out[s * M + i] = order[s].axis[i];
    return MDFFT_OK;
}

mdfft_status mdfft_pass_timing(mdfft_plan_t p, int enable) {
    if (!p) return fail(MDFFT_E_ARG, "null plan");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan");
    if (enable && p->ev.empty()) {
        p->ev.assign((size_t)MDFFT_TIMING_SLOTS * (p->M + 1), nullptr);
        for (cudaEvent_t &e : p->ev) {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return cuda_fail(err, "cudaEventCreate");
        }
    }
    p->timing = enable != 0;
    if (enable) p->timed = 0;
    return MDFFT_OK;
}

mdfft_status mdfft_pass_times(mdfft_plan_t p, float *ms_out, int cap, int *n_execs) {
    if (!p || !ms_out) return fail(MDFFT_E_ARG, "null argument");
    if (p->timed == 0) return fail(MDFFT_E_ARG, "no timed execution recorded");
    const int M = p->M;
    const int64_t n = std::min<int64_t>(p->timed, MDFFT_TIMING_SLOTS);
    const int64_t last = (p->timed - 1) % MDFFT_TIMING_SLOTS;
    cudaError_t e = cudaEventSynchronize(p->ev[last * (M + 1) + M]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    std::vector<double> sum(M, 0.0);
    for (int64_t slot = 0; slot < n; ++slot)
        for (int s = 0; s < M; ++s) {
            float ms = 0;
            e = cudaEventElapsedTime(&ms, p->ev[slot * (M + 1) + s], p->ev[slot * (M + 1) + s + 1]);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
            sum[s] += ms;
        }
    for (int s = 0; s < M && s < cap; ++s) ms_out[s] = (float)(sum[s] / (double)n);
    if (n_execs) *n_execs = (int)n;
    return MDFFT_OK;
}

mdfft_status mdfft_exec_host(mdfft_plan_t p, const void *in_host, void *out_host, void *dev_in, void *dev_out,
                             int dir, int normalize, mdfft_stream_t stream) {
    if (!p) return fail(MDFFT_E_ARG, "null plan");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan cannot execute");
    if (!in_host || !out_host || !dev_in || !dev_out) return fail(MDFFT_E_ARG, "null pointer");
    const size_t bytes = (size_t)p->T * p->batch * p->elem;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->batch > 1) return exec_host_pipelined(p, in_host, out_host, dev_in, dev_out, dir, normalize, st);
    cudaError_t e = cudaMemcpyAsync(dev_in, in_host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    mdfft_status r = exec_impl(p, dev_in, dev_out, dir, normalize, stream, nullptr);
    if (r != MDFFT_OK) return r;
    e = cudaMemcpyAsync(out_host, dev_out, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    return MDFFT_OK;
}

namespace {

// The ring-of-slots kernels the autotuner tries (slots, resident CTAs per SM,
// radix plan): two or three slots at two to four CTAs per SM, where two to
// four tiles' loads in flight per SM measured best for 24-point lines; the
// alternative radix plan only when the plan asks for radix search.
struct RingVariant {
    int slots, per_sm, rp;
};
constexpr RingVariant kRing[] = {{2, 3, 0}, {3, 2, 0}, {2, 4, 0}, {2, 2, 0}, {2, 3, 1}, {3, 2, 1}};
constexpr int kRingVariants = (int)(sizeof(kRing) / sizeof(kRing[0]));
bool ring_variant(int64_t n, int rv, bool tune_radix, PassKernel *k) {
    if (rv < 0 || rv >= kRingVariants || (kRing[rv].rp && !tune_radix)) return false;
    return mdfft::find_pass_kernel_ring(n, kRing[rv].slots, kRing[rv].per_sm, kRing[rv].rp, k);
}

// The one-thread-per-line kernels (radix plan, warps per CTA): 4 warps, 2
// warps, and the alternative radix plan when the plan asks for radix search.
struct LineVariant {
    int rp, warps;
};
constexpr LineVariant kLine[] = {{0, 4}, {0, 2}, {1, 4}};
constexpr int kLineVariants = (int)(sizeof(kLine) / sizeof(kLine[0]));
bool line_variant(int64_t n, int lv, bool tune_radix, PassKernel *k) {
    if (lv < 0 || lv >= kLineVariants || (kLine[lv].rp && !tune_radix)) return false;
    return mdfft::find_pass_kernel_line(n, kLine[lv].rp, kLine[lv].warps, k);
}

}  // namespace

mdfft_status mdfft_plan_autotune(mdfft_plan_t p, const void *in, void *out, int reps, mdfft_stream_t stream,
                                 float *ms_before, float *ms_after) {
    if (!p || !in || !out) return fail(MDFFT_E_ARG, "null argument");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan");
    if (reps < 1) return fail(MDFFT_E_ARG, "reps must be >= 1");
    const size_t bytes = (size_t)p->T * p->batch * p->elem;
    if (overlaps(in, out, bytes)) return fail(MDFFT_E_ARG, "in and out overlap");
    drop_graphs(p);  // captured launches would keep the old launch shapes
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(MDFFT_E_CUDA, "cudaEventCreate");
    mdfft_status result = MDFFT_OK;
    for (int s = 0; s < p->M && result == MDFFT_OK; ++s) {
        Pass &ps = p->pass[s];
        std::vector<PassKernel> variants{ps.k};
        PassKernel k;
        if (p->dt == MDFFT_C64) {
            for (int thr : {256, 512, 192, 384})
                if (mdfft::find_pass_kernel_c64_thr(ps.n, thr, &k) && k.threads != ps.k.threads) variants.push_back(k);
            const bool al16 = (uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0;
            for (int nbuf : {1, 2})
                if (mdfft::find_pass_kernel_pipe(ps.n, nbuf, &k) && al16) variants.push_back(k);
            for (int rv = 0; rv < kRingVariants; ++rv)
                if (ring_variant(ps.n, rv, (p->flags & MDFFT_PLAN_TUNE_RADIX) != 0, &k) && al16) variants.push_back(k);
            for (int lv = 0; lv < kLineVariants; ++lv)
                if (line_variant(ps.n, lv, (p->flags & MDFFT_PLAN_TUNE_RADIX) != 0, &k) && al16) variants.push_back(k);
            for (int rp = 0; rp < ((p->flags & MDFFT_PLAN_TUNE_RADIX) ? 2 : 1); ++rp)
                if (mdfft::find_pass_kernel_line2(ps.n, rp, &k) && al16) variants.push_back(k);
            if ((p->flags & MDFFT_PLAN_TUNE_RADIX) && mdfft::find_pass_kernel_c64_alt(ps.n, &k)) variants.push_back(k);
            if (mdfft::find_pass_kernel_c64_occ(ps.n, &k)) variants.push_back(k);
            if (mdfft::find_pass_kernel_c64_shfl(ps.n, &k)) variants.push_back(k);
            for (int rp = 0; rp < ((p->flags & MDFFT_PLAN_TUNE_RADIX) ? 2 : 1); ++rp)
                for (int minb : {2, 4})
                    if (mdfft::find_pass_kernel_c64_pf(ps.n, rp, minb, &k)) variants.push_back(k);
        }
        if (p->dt == MDFFT_C64_TC_FP16 || p->dt == MDFFT_C64_TC_BF16) {
            const int tc = p->dt == MDFFT_C64_TC_FP16 ? mdfft::kTcFp16 : mdfft::kTcBf16;
            if (mdfft::find_pass_kernel_tc_thr(ps.n, tc, 128, &k) && k.fn != ps.k.fn) variants.push_back(k);
            for (bool land : {true, false})
                if (mdfft::find_pass_kernel_tcg(ps.n, tc, land, &k) && k.fn != ps.k.fn) variants.push_back(k);
        }
        float best_ms = -1.f, default_ms = -1.f;
        Pass best = ps;
        mdfft::RadixPlan table = ps.k.plan;  // the plan the pass's twiddle table is made for
        for (size_t v = 0; v < variants.size() && result == MDFFT_OK; ++v) {
            const PassKernel &kv = variants[v];
            if (kv.smem > 48 * 1024 &&
                cudaFuncSetAttribute(kv.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kv.smem) != cudaSuccess) {
                result = fail(MDFFT_E_CUDA, "cudaFuncSetAttribute");
                break;
            }
            if (!same_plan(kv.plan, table)) {  // timing with the twiddles of the variant's own radix plan
                make_twiddles(p, s, kv.plan, st);
                table = kv.plan;
            }
            // tile orders: output-coalesced, and input-chunk order (not for
            // the pipelined kernels, and not when the pass stores whole lines)
            const int orders = (kv.persistent || ps.args.line_store) ? 1 : 2;
            for (int m = 0; m < orders && result == MDFFT_OK; ++m) {
                Pass base;
                if (candidate_pass(p, s, kv, m, 1, 1, base) != MDFFT_OK) continue;
                // tile shapes: the default choice and powers of two along g
                std::vector<std::pair<int, int>> tiles;
                int bg0 = 1, bh0 = 1;
                choose_tile(kv.lines, base.args.Ng, base.args.Nh, p->elem, &bg0, &bh0);
                tiles.push_back({bg0, bh0});
                for (int bg = kv.lines; bg >= 4; bg /= 2) {
                    if (bg > base.args.Ng) continue;
                    const int bh = (int)std::min<int64_t>(base.args.Nh, kv.lines / bg);
                    if (std::find(tiles.begin(), tiles.end(), std::make_pair(bg, bh)) == tiles.end())
                        tiles.push_back({bg, bh});
                }
                for (size_t ti = 0; ti < tiles.size(); ++ti) {
                    Pass cand;
                    if (candidate_pass(p, s, kv, m, tiles[ti].first, tiles[ti].second, cand) != MDFFT_OK) continue;
                    PassArgs a = cand.args;
                    a.in = in;
                    a.out = out;
                    a.tw = (const char *)p->tw + ps.tw_offset;
                    a.scale = 1.0;
                    a.scaled = 0;
                    a.ntiles = cand.ctas;
                    a.err = p->err;
                    void *args[] = {&a};
                    cudaError_t e = cudaSuccess;
                    for (int w = 0; w < 2 && e == cudaSuccess; ++w)
                        e = cudaLaunchKernel(kv.fn, dim3((unsigned)cand.grid), dim3(kv.threads), args, kv.smem, st);
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < reps && e == cudaSuccess; ++r)
                        e = cudaLaunchKernel(kv.fn, dim3((unsigned)cand.grid), dim3(kv.threads), args, kv.smem, st);
                    cudaEventRecord(e1, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) {
                        result = cuda_fail(e, "autotune launch");
                        break;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= (float)reps;
                    if (v == 0 && m == 0 && ti == 0) default_ms = ms;
                    if (best_ms < 0.f || ms < best_ms) best_ms = ms, best = cand;
                }
            }
        }
        if (!same_plan(best.k.plan, table)) make_twiddles(p, s, best.k.plan, st);  // the chosen kernel's table
        if (result != MDFFT_OK) break;
        best.args.in = nullptr, best.args.out = nullptr, best.args.tw = nullptr, best.args.err = nullptr;
        ps = best;
        if (ms_before) ms_before[s] = default_ms;
        if (ms_after) ms_after[s] = best_ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

namespace {

// The launch variants the autotuner chooses among, by code:
// 0 default, 1 / 2 fixed 256 / 512-thread CTAs, 3 / 4 pipelined with 1 / 2 landing buffers,
// 5 tensor-core kernel with 128-thread CTAs, 6 / 7 fixed 192 / 384-thread CTAs,
// 8 the alternative radix plan (default CTA shape rule), 9 a register cap for
// 6 CTAs per SM, 10 / 11 the tensor-core kernel with independent 128-thread
// groups, with landing buffers / with first-stage loads from HBM, 12 / 13 the
// persistent kernel with the next tile's loads in registers (2 / 4 CTAs per
// SM), 14 / 15 the same with the alternative radix plan, 16 the 256-point
// kernel with a warp-shuffle exchange between its two stages, 17-22 the
// ring-of-slots kernel (kRing[variant - 17]: slots, CTAs per SM, radix plan),
// 23-25 one thread per line with the stages in registers (kLine[variant - 23]),
// 26 / 27 two threads per line (default / alternative radix plan).
constexpr int kLineVariant = 17 + kRingVariants;
constexpr int kLine2Variant = kLineVariant + kLineVariants;
constexpr int kTuningVariants = kLine2Variant + 2;
bool tuning_kernel(const mdfft_plan_s *p, int s, int variant, PassKernel *k) {
    const int64_t n = p->pass[s].n;
    if (variant >= 17 && variant < kLineVariant) return p->dt == MDFFT_C64 && ring_variant(n, variant - 17, true, k);
    if (variant >= kLineVariant && variant < kLine2Variant)
        return p->dt == MDFFT_C64 && line_variant(n, variant - kLineVariant, true, k);
    if (variant >= kLine2Variant && variant < kTuningVariants)
        return p->dt == MDFFT_C64 && mdfft::find_pass_kernel_line2(n, variant - kLine2Variant, k);
    switch (variant) {
        case 16:
            return p->dt == MDFFT_C64 && mdfft::find_pass_kernel_c64_shfl(n, k);
        case 12:
        case 13:
        case 14:
        case 15:
            return p->dt == MDFFT_C64 &&
                   mdfft::find_pass_kernel_c64_pf(n, variant >= 14 ? 1 : 0, (variant & 1) ? 4 : 2, k);
        case 10:
        case 11:
            return (p->dt == MDFFT_C64_TC_FP16 || p->dt == MDFFT_C64_TC_BF16) &&
                   mdfft::find_pass_kernel_tcg(n, p->dt == MDFFT_C64_TC_FP16 ? mdfft::kTcFp16 : mdfft::kTcBf16,
                                               variant == 10, k);
        case 9:
            return p->dt == MDFFT_C64 && mdfft::find_pass_kernel_c64_occ(n, k);
        case 8:
            return p->dt == MDFFT_C64 && mdfft::find_pass_kernel_c64_alt(n, k);
        case 6:
        case 7:
            return p->dt == MDFFT_C64 && mdfft::find_pass_kernel_c64_thr(n, variant == 6 ? 192 : 384, k);
        case 5:
            return (p->dt == MDFFT_C64_TC_FP16 || p->dt == MDFFT_C64_TC_BF16) &&
                   mdfft::find_pass_kernel_tc_thr(n, p->dt == MDFFT_C64_TC_FP16 ? mdfft::kTcFp16 : mdfft::kTcBf16,
                                                  128, k);
        case 0:
            return lookup(p->dt, n, k);
        case 1:
        case 2:
            return p->dt == MDFFT_C64 && mdfft::find_pass_kernel_c64_thr(n, variant == 1 ? 256 : 512, k);
        case 3:
        case 4:
            return p->dt == MDFFT_C64 && mdfft::find_pass_kernel_pipe(n, variant - 2, k);
        default:
            return false;
    }
}

}  // namespace

mdfft_status mdfft_plan_tuning(mdfft_plan_t p, int32_t *out, int cap) {
    if (!p || !out) return fail(MDFFT_E_ARG, "null argument");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan has no passes");
    if (cap < 4 * p->M) return fail(MDFFT_E_ARG, "cap must be at least 4 M");
    for (int s = 0; s < p->M; ++s) {
        const Pass &ps = p->pass[s];
        int variant = -1;
        for (int v = 0; v < kTuningVariants && variant < 0; ++v) {
            PassKernel k;
            if (tuning_kernel(p, s, v, &k) && k.fn == ps.k.fn && k.per_sm == ps.k.per_sm) variant = v;
        }
        if (variant < 0) return fail(MDFFT_E_CUDA, "internal: unknown pass kernel");
        out[4 * s] = variant, out[4 * s + 1] = ps.args.Bg, out[4 * s + 2] = ps.args.Bh, out[4 * s + 3] = ps.mapping;
    }
    return MDFFT_OK;
}

mdfft_status mdfft_plan_set_tuning(mdfft_plan_t p, const int32_t *in, int n) {
    if (!p || !in) return fail(MDFFT_E_ARG, "null argument");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan has no passes");
    if (n != 4 * p->M) return fail(MDFFT_E_ARG, "expected 4 M entries");
    Pass next[MDFFT_MAX_DIMS];
    for (int s = 0; s < p->M; ++s) {  // validate everything before changing anything
        PassKernel k;
        const int variant = in[4 * s], Bg = in[4 * s + 1], Bh = in[4 * s + 2], mapping = in[4 * s + 3];
        if (!tuning_kernel(p, s, variant, &k)) return fail(MDFFT_E_ARG, "kernel variant not built for this pass");
        if ((variant == 3 || variant == 4) && k.lines != p->pass[s].k.lines)
            return fail(MDFFT_E_ARG, "pipelined variant needs the default tile lines");
        if (mapping != 0 && (k.persistent || mapping != 1))
            return fail(MDFFT_E_ARG, "tile order must be 0, or 1 with a non-persistent kernel");
        if (k.smem > 48 * 1024 &&
            cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) != cudaSuccess)
            return fail(MDFFT_E_CUDA, "cudaFuncSetAttribute");
        mdfft_status st = candidate_pass(p, s, k, mapping, Bg, Bh, next[s]);
        if (st != MDFFT_OK) return st;
    }
    for (int s = 0; s < p->M; ++s)
        if (!same_plan(next[s].k.plan, p->pass[s].k.plan)) make_twiddles(p, s, next[s].k.plan, nullptr);
    cudaError_t e = cudaDeviceSynchronize();  // the new tables ready for any stream
    if (e != cudaSuccess) return cuda_fail(e, "twiddle generation");
    for (int s = 0; s < p->M; ++s) p->pass[s] = next[s];
    drop_graphs(p);
    return MDFFT_OK;
}

mdfft_status mdfft_pass_describe(mdfft_plan_t p, int s, mdfft_pass_info *out) {
    if (!p || !out) return fail(MDFFT_E_ARG, "null argument");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan has no passes");
    if (s < 0 || s >= p->M) return fail(MDFFT_E_ARG, "pass index out of range");
    const Pass &ps = p->pass[s];
    out->line_length = ps.n;
    out->tile_g = ps.args.Bg;
    out->tile_h = ps.args.Bh;
    out->threads = ps.k.threads;
    out->smem_bytes = (int)ps.k.smem;
    out->ctas = ps.ctas;
    out->fft_axis = ps.f;
    out->store_axis = ps.g;
    out->grid = ps.grid;
    out->persistent = ps.k.persistent;
    out->stages = ps.k.plan.S;
    for (int i = 0; i < 12; ++i) out->radix[i] = i < ps.k.plan.S ? ps.k.plan.R[i] : 0;
    out->tile_order = ps.mapping;
    return MDFFT_OK;
}

namespace {
// The tiling a probe of pass s moves: the pass's own tiles (as built or
// autotuned) when they fit a CTA of `lines` lines, else the default tiling.
void probe_tiling(const mdfft_plan_s *p, int s, int lines, PassArgs *a, int64_t *ctas) {
    const Pass &ps = p->pass[s];
    if ((int64_t)ps.args.Bg * ps.args.Bh <= lines) {
        *a = ps.args;
        *ctas = ps.ctas;
        set_tile_divisors(*a, ps.ctas);
    } else {
        mdfft::detail::retile_pass(p, s, lines, a, ctas);
    }
}
}  // namespace

mdfft_status mdfft_pattern_probe(mdfft_plan_t p, int s, const void *in, void *out, int reps, mdfft_stream_t stream,
                                 float *ms) {
    if (!p || !in || !out || !ms) return fail(MDFFT_E_ARG, "null argument");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan");
    if (s < 0 || s >= p->M || reps < 1) return fail(MDFFT_E_ARG, "bad pass index or reps");
    if (p->dt != MDFFT_C64) return fail(MDFFT_E_UNSUPPORTED, "complex64 plans only");
    const Pass &ps = p->pass[s];
    if (ps.args.line_store) return fail(MDFFT_E_UNSUPPORTED, "the pass stores whole lines: no transpose to probe");
    PassKernel k;
    if (!mdfft::find_move_kernel_c64(ps.n, &k)) return fail(MDFFT_E_UNSUPPORTED, "no probe for this line length");
    PassArgs a;
    int64_t ctas = 0;
    probe_tiling(p, s, k.lines, &a, &ctas);
    a.in = in, a.out = out, a.scale = 1.0, a.scaled = 0, a.conj = 0, a.moved = nullptr, a.split = nullptr;
    if (k.smem > 48 * 1024 &&
        cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) != cudaSuccess)
        return fail(MDFFT_E_CUDA, "cudaFuncSetAttribute");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    void *args[] = {&a};
    cudaError_t e = cudaLaunchKernel(k.fn, dim3((unsigned)ctas), dim3(k.threads), args, k.smem, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = cudaLaunchKernel(k.fn, dim3((unsigned)ctas), dim3(k.threads), args, k.smem, st);
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "probe launch");
    *ms = t / (float)reps;
    return MDFFT_OK;
}

mdfft_status mdfft_movement_probe(mdfft_plan_t p, int s, int slots, int per_sm, const void *in, void *out, int reps,
                                  mdfft_stream_t stream, float *ms) {
    if (!p || !in || !out || !ms) return fail(MDFFT_E_ARG, "null argument");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan");
    if (s < 0 || s >= p->M || reps < 1) return fail(MDFFT_E_ARG, "bad pass index or reps");
    if (per_sm < 1 || per_sm > 8) return fail(MDFFT_E_ARG, "per_sm must be in [1, 8]");
    if ((uintptr_t)in % 16 || (uintptr_t)out % 16) return fail(MDFFT_E_ARG, "in and out must be 16-byte aligned");
    if (p->dt != MDFFT_C64) return fail(MDFFT_E_UNSUPPORTED, "complex64 plans only");
    const Pass &ps = p->pass[s];
    if (ps.args.line_store) return fail(MDFFT_E_UNSUPPORTED, "the pass stores whole lines: no transpose to probe");
    PassKernel k;
    if (!mdfft::find_move_ring_kernel_c64(ps.n, slots, &k))
        return fail(MDFFT_E_UNSUPPORTED, "no ring probe for this line length or slot count");
    k.per_sm = per_sm;
    PassArgs a;
    int64_t ctas = 0;
    probe_tiling(p, s, k.lines, &a, &ctas);
    a.in = in, a.out = out, a.scale = 1.0, a.scaled = 0, a.conj = 0, a.moved = nullptr, a.split = nullptr;
    a.ntiles = ctas;
    const int64_t grid = std::min<int64_t>(ctas, mdfft::detail::wave_ctas(k));  // sets the shared-memory limit
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    void *args[] = {&a};
    cudaError_t e = cudaLaunchKernel(k.fn, dim3((unsigned)grid), dim3(k.threads), args, k.smem, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = cudaLaunchKernel(k.fn, dim3((unsigned)grid), dim3(k.threads), args, k.smem, st);
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "probe launch");
    *ms = t / (float)reps;
    return MDFFT_OK;
}

mdfft_status mdfft_plan_check(mdfft_plan_t p) {
    if (!p) return fail(MDFFT_E_ARG, "null plan");
    if (!p->err) return MDFFT_OK;
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, p->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
    if (flag) {
        cudaMemset(p->err, 0, sizeof(int));
        return fail(MDFFT_E_TIMEOUT, "a pass kernel's bounded wait gave up; its output is incomplete");
    }
    return MDFFT_OK;
}

mdfft_status mdfft_workspace_size(mdfft_plan_t p, size_t *bytes) {
    if (!p || !bytes) return fail(MDFFT_E_ARG, "null argument");
    *bytes = 0;
    if (p->ws) *bytes += (size_t)p->T * p->batch * p->elem;
    if (p->ws2) *bytes += (size_t)p->T * p->batch * p->elem;
    return MDFFT_OK;
}

mdfft_status mdfft_launches_per_exec(mdfft_plan_t p, int *launches) {
    if (!p || !launches) return fail(MDFFT_E_ARG, "null argument");
    *launches = p->M;
    return MDFFT_OK;
}

mdfft_status mdfft_destroy(mdfft_plan_t p) {
    release(p);
    return MDFFT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mdfft_exec_noalloc: the transform without any device allocation.
//
// The scratch it needs (twiddle tables and the array the passes ping-pong
// through) is this file-scope device array.  Every GPU that loads the library
// holds it until the process exits.  Host code must not use the symbol's
// address directly (on the host it names a stand-in); the device address is
// taken once per device with cudaGetSymbolAddress and cached.  The cache
// does not survive cudaDeviceReset (the module is loaded again and the array
// may move): a process that resets a device must not call this entry point
// on that device afterwards.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[MDFFT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr size_t kNoallocTwiddleBytes = 256 * 1024;  // M <= 8 tables of at most 2048 x 16 bytes
constexpr size_t kNoallocTwiddleStride = 2048;       // entries reserved per pass (tw_entries < 2 N <= 2048)
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_addr[kNoallocMaxDevices] = {nullptr};

mdfft_status noalloc_fail(mdfft_status st, const char *msg) {
    g_err = msg;  // the message is recorded like every other entry point's
    return st;
}

// Device address of the scratch array on the current device (looked up once).
mdfft_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices) return noalloc_fail(MDFFT_E_UNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_noalloc_addr[dev];
    return MDFFT_OK;
}

// Pass s of the order held in the fixed-size array L (no heap use): the same
// launch configuration mdfft_plan builds (tile shape, small-grid shrink),
// without the owner maps of the count mode.
mdfft_status noalloc_pass(int M, const int64_t *N, const pl::Layout *L, mdfft_dtype dt, size_t elem, int s,
                          Pass &ps) {
    pl::Layout nat;
    nat.M = M;
    for (int i = 0; i < M; ++i) nat.axis[i] = i;
    const pl::Layout &Li = L[s];
    const pl::Layout &Lo = (s + 1 < M) ? L[s + 1] : nat;
    ps.f = Li.axis[M - 1];
    ps.g = Lo.axis[M - 1];
    ps.h = -1;
    for (int i = M - 2; i >= 0; --i)
        if (Lo.axis[i] != ps.f) {
            ps.h = Lo.axis[i];
            break;
        }
    ps.n = N[ps.f];
    if (!lookup(dt, ps.n, &ps.k)) return noalloc_fail(MDFFT_E_UNSUPPORTED, "a line length is not built for this dtype");
    int64_t sin_[pl::kMaxDims], sout[pl::kMaxDims];
    layout_strides(Li, N, sin_);
    layout_strides(Lo, N, sout);
    PassArgs &a = ps.args;
    std::memset(&a, 0, sizeof(a));
    const int64_t Ng = N[ps.g], Nh = ps.h >= 0 ? N[ps.h] : 1;
    int Bg = 1, Bh = 1;
    choose_tile(ps.k.lines, Ng, Nh, elem, &Bg, &Bh);
    a.Bg = Bg, a.Bh = Bh, a.Ng = Ng, a.Nh = Nh;
    a.gblocks = (Ng + Bg - 1) / Bg;
    a.hblocks = (Nh + Bh - 1) / Bh;
    a.in_sg = sin_[ps.g];
    a.in_sh = ps.h >= 0 ? sin_[ps.h] : 0;
    a.out_sh = ps.h >= 0 ? sout[ps.h] : 0;
    a.out_sf = sout[ps.f];
    a.out_sg = 1;
    ps.ctas = a.gblocks * a.hblocks;
    for (int i = M - 1; i >= 0; --i) {
        int ax = Lo.axis[i];
        if (ax == ps.f || ax == ps.g || ax == ps.h) continue;
        a.rest_count[a.nrest] = N[ax];
        a.rest_in[a.nrest] = sin_[ax];
        a.rest_out[a.nrest] = sout[ax];
        a.nrest++;
        ps.ctas *= N[ax];
    }
    shrink_to_wave(ps, elem, false);  // the small-grid tiles of mdfft_plan
    set_tile_divisors(a, ps.ctas);
    a.scale = 1.0;
    a.scaled = 0;
    return MDFFT_OK;
}

}  // namespace

extern "C" mdfft_status mdfft_exec_noalloc(int M, const int64_t N[], const int *order, mdfft_dtype dt,
                                           const void *in, void *out, int dir, int normalize,
                                           mdfft_stream_t stream) {
    if (!N || !order || !in || !out) return noalloc_fail(MDFFT_E_ARG, "null argument (the order is required)");
    if (M < 2 || M > MDFFT_MAX_DIMS) return noalloc_fail(MDFFT_E_UNSUPPORTED, "M must be in [2, 8]");
    if (dt != MDFFT_C64 && dt != MDFFT_C128) return noalloc_fail(MDFFT_E_UNSUPPORTED, "dtype must be C64 or C128");
    if (dir != -1 && dir != 1) return noalloc_fail(MDFFT_E_ARG, "dir must be -1 (forward) or +1 (inverse)");
    if (normalize != 0 && !(normalize == 1 && dir == 1))
        return noalloc_fail(MDFFT_E_ARG, "normalize = 1 is only defined for the inverse");
    const size_t elem = dt == MDFFT_C128 ? 16 : 8;
    unsigned __int128 T = 1;
    for (int i = 0; i < M; ++i) {
        if (N[i] < 1) return noalloc_fail(MDFFT_E_ARG, "dims must be >= 1");
        T *= (unsigned __int128)N[i];
    }
    if (T * elem > (unsigned __int128)MDFFT_NOALLOC_MAX_ARRAY_BYTES)
        return noalloc_fail(MDFFT_E_UNSUPPORTED,
                            "array larger than MDFFT_NOALLOC_MAX_ARRAY_BYTES; use mdfft_plan + mdfft_exec");
    const size_t bytes = (size_t)T * elem;
    if ((uintptr_t)in % elem || (uintptr_t)out % elem) return noalloc_fail(MDFFT_E_ARG, "misaligned data pointer");
    if (overlaps(in, out, bytes)) return noalloc_fail(MDFFT_E_ARG, "in and out must not overlap");
    // the order, validated without heap use
    pl::Layout L[MDFFT_MAX_DIMS];
    unsigned used_last = 0;
    for (int s = 0; s < M; ++s) {
        L[s].M = M;
        unsigned seen = 0;
        for (int i = 0; i < M; ++i) {
            int a = order[s * M + i];
            if (a < 0 || a >= M || (seen & (1u << a))) return noalloc_fail(MDFFT_E_ORDER, "a layout is not a permutation");
            if (s == 0 && a != i) return noalloc_fail(MDFFT_E_ORDER, "layout 0 must be the natural order");
            seen |= 1u << a;
            L[s].axis[i] = a;
        }
        unsigned last = 1u << L[s].axis[M - 1];
        if (used_last & last) return noalloc_fail(MDFFT_E_ORDER, "a layout transforms an axis twice");
        used_last |= last;
    }
    Pass pass[MDFFT_MAX_DIMS];
    for (int s = 0; s < M; ++s) {
        mdfft_status st = noalloc_pass(M, N, L, dt, elem, s, pass[s]);
        if (st != MDFFT_OK) return st;
    }
    unsigned char *scratch = nullptr;
    mdfft_status st = noalloc_scratch(&scratch);
    if (st != MDFFT_OK) return st;
    unsigned char *ws = scratch + kNoallocTwiddleBytes;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    // twiddles of every pass, rewritten by every call in stream order
    for (int s = 0; s < M; ++s) {
        const int entries = std::max(1, mdfft::tw_entries(pass[s].k.plan));
        twiddle_kernel<<<(unsigned)((entries + 255) / 256), 256, 0, cs>>>(
            scratch + (size_t)s * kNoallocTwiddleStride * elem, pass[s].n, pass[s].k.plan, dt == MDFFT_C128);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "twiddle launch");
    void *dst[MDFFT_MAX_DIMS];
    dst[M - 1] = out;
    for (int s = M - 2; s >= 0; --s) dst[s] = (dst[s + 1] == out) ? (void *)ws : out;
    const void *src = in;
    for (int s = 0; s < M; ++s) {
        const PassKernel &k = pass[s].k;
        if (k.smem > 48 * 1024) {
            e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        }
        PassArgs a = pass[s].args;
        a.in = src;
        a.out = dst[s];
        a.tw = scratch + (size_t)s * kNoallocTwiddleStride * elem;
        a.conj = dir == 1 ? (s == 0 ? 1 : 0) | (s == M - 1 ? 2 : 0) : 0;
        a.scale = (s == M - 1 && normalize) ? 1.0 / (double)T : 1.0;
        a.scaled = a.scale != 1.0;
        void *args[] = {&a};
        e = cudaLaunchKernel(k.fn, dim3((unsigned)pass[s].ctas), dim3(k.threads), args, k.smem, cs);
        if (e != cudaSuccess) return cuda_fail(e, "pass launch");
        src = dst[s];
    }
    return MDFFT_OK;
}
