// dist.cu -- the data plane of the distributed setting (Sec. 1; the
// "Transpose" steps of Fig. 4) when the P virtual processes sit on G devices.
//
// Device g holds the processes floor(gP/G) .. floor((g+1)P/G) - 1, i.e. one
// contiguous row-major range of every layout.  Step s of a transform on G
// devices is:
//   1. mdfft_dist_lines   the 1-D DFTs along the last axis of layout s over
//                         the device's range (whole lines: no transpose);
//   2. mdfft_dist_pack    the range's points, grouped by the device that owns
//                         them in layout s+1 (natural order after the last
//                         step), each group contiguous in a send buffer;
//   3. (the caller's transport: an all-to-all-v with mdfft_exchange_counts)
//   4. mdfft_dist_unpack  the received groups into the device's range of
//                         layout s+1.
// The order of a group's points is fixed by the planner's boxes: the source
// range's boxes (layout s) are intersected with the destination range's boxes
// (layout s+1) in a fixed order, and the points of each intersection are
// listed in layout s+1's row-major order.  Sender and receiver derive the same
// list, so only the values travel.  The pack reads the source range in that
// order (the transpose); the unpack reads and writes contiguous runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "plan_internal.h"

using mdfft::PassArgs;
using mdfft::detail::cuda_fail;
using mdfft::detail::fail;
namespace pl = mdfft::planner;

namespace mdfft {
namespace dist {

// One intersection box of a copy: point r (0 .. count) of the box has the
// coordinates of r over ext (slowest first) and goes from src_base +
// sum c_i src_stride_i to dst_base + sum c_i dst_stride_i.
struct CopyBox {
    int64_t start;  // first point of the box in the copy's numbering
    int64_t src_base, dst_base;
    int64_t ext[kMaxTileDims], src_stride[kMaxTileDims], dst_stride[kMaxTileDims];
};

// Each CTA copies one contiguous range of the copy's points, its threads
// striding through it, so a thread's box only moves forward: one search at
// the start, then a step to the next box when its point passes the current
// one's end.  Coordinates are split in 32-bit arithmetic when every box is
// smaller than 2^32 points (small32), else in 64-bit.  A thread works on
// kUnroll points at a time: all their loads are in flight before the stores.
template <typename C> struct BoxWalk {
    const CopyBox *boxes;
    int nboxes, M, small32, cur;
    int64_t total, next;
    __device__ __forceinline__ void seek(int64_t e) {
        int lo = 0, hi = nboxes - 1;  // last box starting at or before e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (boxes[mid].start <= e) lo = mid;
            else hi = mid - 1;
        }
        cur = lo;
        next = cur + 1 < nboxes ? boxes[cur + 1].start : total;
    }
    // source and destination index of point e (e only grows between calls)
    __device__ __forceinline__ void at(int64_t e, int64_t &s, int64_t &d) {
        while (e >= next) {
            ++cur;
            next = cur + 1 < nboxes ? boxes[cur + 1].start : total;
        }
        const CopyBox &b = boxes[cur];
        s = b.src_base, d = b.dst_base;
        if (small32) {
            uint32_t r = (uint32_t)(e - b.start);
            for (int i = M - 1; i >= 0 && r; --i) {
                const uint32_t x = (uint32_t)b.ext[i], c = r % x;
                r /= x;
                s += (int64_t)c * b.src_stride[i];
                d += (int64_t)c * b.dst_stride[i];
            }
        } else {
            int64_t r = e - b.start;
            for (int i = M - 1; i >= 0 && r; --i) {
                const int64_t c = r % b.ext[i];
                r /= b.ext[i];
                s += c * b.src_stride[i];
                d += c * b.dst_stride[i];
            }
        }
    }
};

constexpr int kUnroll = 4;

template <typename C>
__global__ void __launch_bounds__(256) box_copy_kernel(const C *__restrict__ src, C *__restrict__ dst,
                                                      const CopyBox *__restrict__ boxes, int nboxes, int M,
                                                      int64_t total, int64_t per_cta, int small32) {
    const int64_t e0 = (int64_t)blockIdx.x * per_cta;
    const int64_t e1 = e0 + per_cta < total ? e0 + per_cta : total;
    int64_t e = e0 + threadIdx.x;
    if (e >= e1) return;
    BoxWalk<C> w{boxes, nboxes, M, small32, 0, total, 0};
    w.seek(e);
    const int64_t step = blockDim.x;
    for (; e < e1; e += kUnroll * step) {
        int64_t si[kUnroll], di[kUnroll];
        C v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (e + u * step < e1) w.at(e + u * step, si[u], di[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (e + u * step < e1) v[u] = src[si[u]];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (e + u * step < e1) dst[di[u]] = v[u];
    }
}

}  // namespace dist
}  // namespace mdfft

using mdfft::dist::CopyBox;

namespace {

pl::Layout layout_at(const mdfft_plan_s *p, int step) {
    pl::Layout L;
    L.M = p->M;
    for (int i = 0; i < p->M; ++i) L.axis[i] = step < p->M ? p->order[step].axis[i] : i;
    return L;
}

// Range [x0, x1) of device g of G in layout `step` (step M: natural order).
void device_range(const mdfft_plan_s *p, int step, int G, int g, int64_t *x0, int64_t *x1) {
    const pl::Layout L = layout_at(p, step);
    int64_t d[pl::kMaxDims];
    pl::layout_dims(L, p->N, d);
    *x0 = pl::fmd(p->M, d, p->P, (int64_t)g * p->P / G);
    *x1 = pl::fmd(p->M, d, p->P, (int64_t)(g + 1) * p->P / G);
}

void strides_of(const pl::Layout &L, const int64_t *N, int64_t *st) {
    int64_t s = 1;
    for (int i = L.M - 1; i >= 0; --i) st[L.axis[i]] = s, s *= N[L.axis[i]];
}

// The boxes of the copy of step `step` between device `me` and all others:
// pack = the points of me's range in layout step, group by group (destination
// h = 0 .. G-1); unpack = the points of me's range in layout step+1, group by
// group (source g = 0 .. G-1).  Both number the points of group (g -> h) the
// same way.
mdfft_status make_boxes(const mdfft_plan_s *p, int step, int G, int me, bool pack, std::vector<CopyBox> &out,
                        int64_t *total) {
    const int M = p->M;
    const pl::Layout A = layout_at(p, step), B = layout_at(p, step + 1);
    int64_t sa[pl::kMaxDims], sb[pl::kMaxDims];
    strides_of(A, p->N, sa);
    strides_of(B, p->N, sb);
    int64_t my0, my1;
    device_range(p, pack ? step : step + 1, G, me, &my0, &my1);
    out.clear();
    int64_t pos = 0;
    for (int other = 0; other < G; ++other) {
        const int g = pack ? me : other, h = pack ? other : me;
        int64_t a0, a1, b0, b1;
        device_range(p, step, G, g, &a0, &a1);
        device_range(p, step + 1, G, h, &b0, &b1);
        std::vector<pl::Box> ba, bb;
        pl::range_boxes(A, p->N, a0, a1, ba);
        pl::range_boxes(B, p->N, b0, b1, bb);
        for (const pl::Box &x : ba)
            for (const pl::Box &y : bb) {
                int64_t lo[pl::kMaxDims], hi[pl::kMaxDims], count = 1;
                for (int i = 0; i < M; ++i) {
                    lo[i] = std::max(x.lo[i], y.lo[i]);
                    hi[i] = std::min(x.hi[i], y.hi[i]);
                    count *= std::max<int64_t>(0, hi[i] - lo[i]);
                }
                if (count == 0) continue;
                CopyBox cb;
                std::memset(&cb, 0, sizeof(cb));
                cb.start = pos;
                // points in layout step+1's row-major order over the box
                int64_t run = 1, boxstride[pl::kMaxDims];
                for (int i = M - 1; i >= 0; --i) {
                    const int ax = B.axis[i];
                    cb.ext[i] = hi[ax] - lo[ax];
                    boxstride[i] = run;
                    run *= cb.ext[i];
                }
                int64_t in_a = 0, in_b = 0;
                for (int ax = 0; ax < M; ++ax) in_a += lo[ax] * sa[ax], in_b += lo[ax] * sb[ax];
                for (int i = 0; i < M; ++i) {
                    const int ax = B.axis[i];
                    if (pack) {  // local layout-step array -> send buffer
                        cb.src_stride[i] = sa[ax];
                        cb.dst_stride[i] = boxstride[i];
                    } else {  // receive buffer -> local layout-step+1 array
                        cb.src_stride[i] = boxstride[i];
                        cb.dst_stride[i] = sb[ax];
                    }
                }
                cb.src_base = pack ? in_a - my0 : pos;
                cb.dst_base = pack ? pos : in_b - my0;
                out.push_back(cb);
                pos += count;
            }
    }
    *total = pos;
    return MDFFT_OK;
}

mdfft_status check_dist(const mdfft_plan_s *p, int step, int G, int g) {
    if (!p) return fail(MDFFT_E_ARG, "null plan");
    if (p->flags & MDFFT_PLAN_HOST_ONLY) return fail(MDFFT_E_ARG, "host-only plan cannot execute");
    if (p->bd.kind != pl::kRowwise) return fail(MDFFT_E_ARG, "the distributed data plane is for row-wise plans");
    if (p->flags & MDFFT_PLAN_OUT_LAST_LAYOUT) return fail(MDFFT_E_ARG, "distributed steps end in natural order");
    if (p->batch != 1) return fail(MDFFT_E_ARG, "distributed steps take plans of one transform");
    if (step < 0 || step >= p->M) return fail(MDFFT_E_ARG, "step out of range");
    if (G < 1 || G > p->P) return fail(MDFFT_E_ARG, "G must be in [1, P]");
    if (g < 0 || g >= G) return fail(MDFFT_E_ARG, "device index out of range");
    return MDFFT_OK;
}

// Copy boxes of (step, G, device, pack) in device memory, made on first use.
mdfft_status device_boxes(mdfft_plan_s *p, int step, int G, int me, bool pack, const CopyBox **dev, int *n,
                          int64_t *total) {
    const std::vector<int64_t> key{step, G, me, pack ? 1 : 0};
    for (auto &c : p->dist_boxes)
        if (c.key == key) {
            *dev = static_cast<const CopyBox *>(c.dev), *n = c.n, *total = c.total;
            return MDFFT_OK;
        }
    std::vector<CopyBox> boxes;
    int64_t tot = 0;
    mdfft_status st = make_boxes(p, step, G, me, pack, boxes, &tot);
    if (st != MDFFT_OK) return st;
    mdfft_plan_s::DistBoxes c;
    c.key = key;
    c.n = (int)boxes.size();
    c.total = tot;
    if (c.n > 0) {
        cudaError_t e = cudaMalloc(&c.dev, boxes.size() * sizeof(CopyBox));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc copy boxes");
        e = cudaMemcpy(c.dev, boxes.data(), boxes.size() * sizeof(CopyBox), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(c.dev);
            return cuda_fail(e, "copy boxes");
        }
    }
    p->dist_boxes.push_back(c);
    *dev = static_cast<const CopyBox *>(c.dev), *n = c.n, *total = tot;
    return MDFFT_OK;
}

mdfft_status run_copy(mdfft_plan_s *p, int step, int G, int me, bool pack, const void *src, void *dst,
                      cudaStream_t st) {
    if (!src || !dst) return fail(MDFFT_E_ARG, "null data pointer");
    if ((uintptr_t)src % p->elem || (uintptr_t)dst % p->elem) return fail(MDFFT_E_ARG, "misaligned data pointer");
    const CopyBox *boxes = nullptr;
    int n = 0;
    int64_t total = 0;
    mdfft_status s = device_boxes(p, step, G, me, pack, &boxes, &n, &total);
    if (s != MDFFT_OK || total == 0) return s;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // contiguous ranges of whole 256-point rounds, about 8 resident waves of CTAs
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((total + 1023) / 1024, (int64_t)sms * 64));
    const int64_t per_cta = ((total + blocks - 1) / blocks + 255) / 256 * 256;
    const int small32 = total < (int64_t(1) << 32) ? 1 : 0;  // every box holds fewer than 2^32 points
    if (p->dt == MDFFT_C128)
        mdfft::dist::box_copy_kernel<double2><<<(unsigned)blocks, 256, 0, st>>>(
            static_cast<const double2 *>(src), static_cast<double2 *>(dst), boxes, n, p->M, total, per_cta, small32);
    else
        mdfft::dist::box_copy_kernel<float2><<<(unsigned)blocks, 256, 0, st>>>(
            static_cast<const float2 *>(src), static_cast<float2 *>(dst), boxes, n, p->M, total, per_cta, small32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, pack ? "pack launch" : "unpack launch");
    return MDFFT_OK;
}

}  // namespace

extern "C" {

mdfft_status mdfft_dist_local_range(mdfft_plan_t p, int step, int G, int g, int64_t *x0, int64_t *x1) {
    if (!p || !x0 || !x1) return fail(MDFFT_E_ARG, "null argument");
    if (step < 0 || step > p->M) return fail(MDFFT_E_ARG, "step out of range");
    if (G < 1 || G > p->P || g < 0 || g >= G) return fail(MDFFT_E_ARG, "G must be in [1, P] and g in [0, G)");
    device_range(p, step, G, g, x0, x1);
    return MDFFT_OK;
}

mdfft_status mdfft_dist_lines(mdfft_plan_t p, int step, int G, int g, const void *in_local, void *out_local,
                              int dir, int normalize, mdfft_stream_t stream) {
    mdfft_status cs = check_dist(p, step, G, g);
    if (cs != MDFFT_OK) return cs;
    if (!in_local || !out_local) return fail(MDFFT_E_ARG, "null data pointer");
    if (dir != -1 && dir != 1) return fail(MDFFT_E_ARG, "dir must be -1 (forward) or +1 (inverse)");
    if (normalize != 0 && !(normalize == 1 && dir == 1))
        return fail(MDFFT_E_ARG, "normalize = 1 is only defined for the inverse");
    const int M = p->M;
    const mdfft::detail::Pass &ps = p->pass[step];
    const int64_t n = ps.n;
    int64_t x0, x1;
    device_range(p, step, G, g, &x0, &x1);
    if (x0 % n || x1 % n)
        return fail(MDFFT_E_UNSUPPORTED, "a device boundary splits a line of this step (M-D regime): use fewer devices");
    const size_t bytes = (size_t)(x1 - x0) * p->elem;
    const uintptr_t a = (uintptr_t)in_local, b = (uintptr_t)out_local;
    if (a != b && a < b + bytes && b < a + bytes) return fail(MDFFT_E_ARG, "in and out overlap partially");
    const size_t align = ps.k.bulk ? 16 : p->elem;
    if (a % align || b % align) return fail(MDFFT_E_ARG, "misaligned data pointer");
    // the device's lines as a [lines x n] array: one pass that keeps the
    // transformed axis fastest (lines stored whole, no transpose)
    PassArgs args;
    std::memset(&args, 0, sizeof(args));
    const int64_t lines = (x1 - x0) / n;
    int Bg = std::max(1, std::min<int>(ps.k.lines, (int)std::min<int64_t>(lines, 1 << 20)));
    args.Bg = Bg, args.Bh = 1, args.Ng = lines, args.Nh = 1;
    args.fd_bg = mdfft::fastdiv_make((uint32_t)Bg);
    args.gblocks = (lines + Bg - 1) / Bg;
    args.hblocks = 1;
    args.in_sg = n, args.out_sg = n, args.out_sf = 1;
    args.line_store = 1;
    args.ntiles = args.gblocks;
    args.tile32 = args.gblocks <= 0xffffffffLL;
    if (args.tile32) {
        args.fd_g = mdfft::fastdiv_make((uint32_t)args.gblocks);
        args.fd_h = mdfft::fastdiv_make(1);
    }
    args.in = in_local;
    args.out = out_local;
    args.tw = (const char *)p->tw + ps.tw_offset;
    args.err = p->err;
    args.conj = dir == 1 ? (step == 0 ? 1 : 0) | (step == M - 1 ? 2 : 0) : 0;
    args.scale = (step == M - 1 && normalize) ? 1.0 / (double)p->T : 1.0;
    args.scaled = args.scale != 1.0;
    args.own_in = args.own_out = mdfft::OwnerMap{1, 1, 1, nullptr, 0, 1};
    const int64_t grid = ps.k.persistent ? std::min<int64_t>(args.gblocks, mdfft::detail::wave_ctas(ps.k)) : args.gblocks;
    void *kargs[] = {&args};
    cudaError_t e = cudaLaunchKernel(ps.k.fn, dim3((unsigned)grid), dim3(ps.k.threads), kargs, ps.k.smem,
                                     reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "line pass launch");
    return MDFFT_OK;
}

mdfft_status mdfft_dist_pack(mdfft_plan_t p, int step, int G, int g, const void *local, void *sendbuf,
                             mdfft_stream_t stream) {
    mdfft_status cs = check_dist(p, step, G, g);
    if (cs != MDFFT_OK) return cs;
    return run_copy(p, step, G, g, true, local, sendbuf, reinterpret_cast<cudaStream_t>(stream));
}

mdfft_status mdfft_dist_unpack(mdfft_plan_t p, int step, int G, int h, const void *recvbuf, void *local,
                               mdfft_stream_t stream) {
    mdfft_status cs = check_dist(p, step, G, h);
    if (cs != MDFFT_OK) return cs;
    return run_copy(p, step, G, h, false, recvbuf, local, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
