// serve.cu -- batched serving of M-D FFT requests of different shapes.
//
// Continuous batching at pass granularity.  Every step launches, in one
// persistent kernel, the next pass (Fig. 4 step + transpose, as in
// mdfft_exec) of every request in flight, whatever its shape; a request that
// arrives while others are on the GPU joins at the next step, as soon as the
// HBM budget and a slot allow, and leaves after its last pass.  One step is
// one launch of a CUDA graph (copy of the step's work table from pinned host
// memory, then the persistent kernel), captured once per table slot.  The
// persistent kernel walks the tiles of all items with a grid stride; a CTA
// finds the item of a tile by binary search over the items' first tiles and
// runs the tile code of that item's line length.  Passes of lines of 16 to
// 64 points (16-byte aligned arrays) go instead to a second persistent
// kernel of the same graph, launched after the first, whose warps each take
// whole 32-line tiles and run the one-thread-per-line code of fft_line.cuh.
// There is no device-side waiting: passes of one request are in consecutive
// steps, ordered by the stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "fft_line.cuh"
#include "plan_internal.h"

using mdfft::PassArgs;
using mdfft::detail::cuda_fail;
using mdfft::detail::fail;

namespace mdfft {
namespace serve {

constexpr int kMaxItems = 512;  // passes per step
constexpr int kSlots = 8;       // tables (and graphs) in flight
constexpr int kThreads = 256;   // CTA size of the persistent kernel (every length uses all of it)

// line lengths the persistent kernel carries (complex64); other lengths run
// as separate launches of their own pass kernel within the same step
#define MDFFT_SERVE_LENGTHS(X) X(0, 16) X(1, 24) X(2, 32) X(3, 48) X(4, 64) X(5, 96) X(6, 128) X(7, 160) X(8, 192) X(9, 256)
#define MDFFT_COUNT_KIND(i, N) +1
constexpr int kKinds = 0 MDFFT_SERVE_LENGTHS(MDFFT_COUNT_KIND);
#undef MDFFT_COUNT_KIND
static_assert(kKinds == 10, "serving kinds are numbered 0 .. kKinds - 1 in MDFFT_SERVE_LENGTHS");

struct Item {
    PassArgs args;
    int64_t start;  // first tile of this item in the step's tile numbering
    int kind;       // index into MDFFT_SERVE_LENGTHS
    int pad;
};

struct Table {
    int n;          // items of the grouped kernel: items[0, n)
    int chunk;      // consecutive tiles dealt to a CTA at a time
    int64_t total;  // tiles in the step
    // items of the line kernels, group g after those of the groups before:
    // items[n + n_line[0] + .. + n_line[g-1], + n_line[g]), tiles numbered from 0 in each group
    int n_line[2];
    int chunk_line[2];  // consecutive 32-line tiles dealt to a warp at a time
    int64_t total_line[2];
    Item items[kMaxItems];
};

// line lengths of the one-thread-per-line serving kernels: kind kLineKind + i;
// group 0 (16, 24, 32: up to 90 registers a thread in the standalone
// kernel) and group 1 (48, 64: up to 190) are separate kernels, so that the
// short lengths keep more warps per SM
#define MDFFT_SERVE_LINE_LENGTHS(X) X(0, 16) X(1, 24) X(2, 32) X(3, 48) X(4, 64)
#define MDFFT_SERVE_LINE_GROUP0(X) X(0, 16) X(1, 24) X(2, 32)
#define MDFFT_SERVE_LINE_GROUP1(X) X(3, 48) X(4, 64)
constexpr int kLineKind = 100;
constexpr int kLineThreads = 128, kLineWarps = kLineThreads / 32;
constexpr int line_group(int kind) { return kind - kLineKind >= 3 ? 1 : 0; }
constexpr size_t kArgsBytes = (sizeof(PassArgs) + 15) / 16 * 16;
constexpr size_t cmax2(size_t a, size_t b) { return a > b ? a : b; }
#define MDFFT_LINE_RS_MAX(i, N) cmax2((size_t)LineCfg<N>::RS,
#define MDFFT_LINE_CLOSE(i, N) )
// staging row stride of each group: its longest line's
constexpr size_t kLineRs[2] = {MDFFT_SERVE_LINE_GROUP0(MDFFT_LINE_RS_MAX) 0 MDFFT_SERVE_LINE_GROUP0(MDFFT_LINE_CLOSE),
                               MDFFT_SERVE_LINE_GROUP1(MDFFT_LINE_RS_MAX) 0 MDFFT_SERVE_LINE_GROUP1(MDFFT_LINE_CLOSE)};
// per warp: the item's arguments, 32 staging rows, 32 line offsets
constexpr size_t line_warp_smem(int g) { return kArgsBytes + 32 * kLineRs[g] * sizeof(float2) + 32 * sizeof(int64_t); }
constexpr size_t kLineSmem[2] = {kLineWarps * line_warp_smem(0), kLineWarps * line_warp_smem(1)};

int line_kind_of(int64_t n) {
    switch (n) {
#define MDFFT_KIND(i, N) \
    case N:              \
        return kLineKind + i;
        MDFFT_SERVE_LINE_LENGTHS(MDFFT_KIND)
#undef MDFFT_KIND
        default:
            return -1;
    }
}

template <int N> using ServeCfg = PassCfg<float, N, 0, kThreads>;
template <int N> constexpr size_t smem_of() { return ServeCfg<N>::SMEM; }
template <int N> constexpr int threads_of() { return ServeCfg<N>::THREADS; }
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
#define MDFFT_SMEM_MAX(i, N) cmax(smem_of<N>(),
#define MDFFT_CLOSE(i, N) )
constexpr size_t kSmem = MDFFT_SERVE_LENGTHS(MDFFT_SMEM_MAX) 0 MDFFT_SERVE_LENGTHS(MDFFT_CLOSE);
#define MDFFT_THR_OK(i, N) static_assert(threads_of<N>() <= kThreads, "serve CTA too small");
MDFFT_SERVE_LENGTHS(MDFFT_THR_OK)

// tile lines of the serving configuration of each kind
int lines_of_kind(int kind) {
    switch (kind) {
#define MDFFT_LINES(i, N) \
    case i:               \
        return ServeCfg<N>::LINES;
        MDFFT_SERVE_LENGTHS(MDFFT_LINES)
#undef MDFFT_LINES
        default:
            return 0;
    }
}

int kind_of(int64_t n) {
    switch (n) {
#define MDFFT_KIND(i, N) \
    case N:              \
        return i;
        MDFFT_SERVE_LENGTHS(MDFFT_KIND)
#undef MDFFT_KIND
        default:
            return -1;
    }
}

__global__ void __launch_bounds__(kThreads, 4) serve_kernel(const Table *tab) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PassArgs args;
    const int n = tab->n;
    const int64_t total = tab->total;
    // chunks of kChunk consecutive tiles, dealt to the CTAs in turn: tiles of
    // different line lengths even out across CTAs, and consecutive tiles of
    // a chunk mostly belong to one item, so item lookups and argument copies
    // are rare (items are in increasing tile order, so lookups only advance)
    const int kChunk = tab->chunk;
    int cur = 0;
    int64_t cur_start = 0, cur_end = n > 1 ? tab->items[1].start : total;  // item 0 starts at tile 0
    int kind = -1;
    for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < total; c0 += (int64_t)gridDim.x * kChunk)
        for (int64_t t = c0; t < c0 + kChunk && t < total; ++t) {
        if (t >= cur_end || kind < 0) {
            if (t >= cur_end) {  // binary search over the items after cur: last one starting <= t
                int lo = cur + 1, hi = n - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (tab->items[mid].start <= t) lo = mid;
                    else hi = mid - 1;
                }
                cur = lo;
                cur_start = tab->items[cur].start;
                cur_end = cur + 1 < n ? tab->items[cur + 1].start : total;
            }
            __syncthreads();  // every thread is done with the previous arguments
            const int *src = reinterpret_cast<const int *>(&tab->items[cur].args);
            int *dst = reinterpret_cast<int *>(&args);
            for (int w = threadIdx.x; w < (int)(sizeof(PassArgs) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
            kind = tab->items[cur].kind;
            __syncthreads();
        }
        const int64_t local = t - cur_start;
        switch (kind) {
#define MDFFT_RUN(i, N)                                                  \
    case i:                                                              \
        pass_tile<float, N, 0, kThreads>(args, local, smem, threadIdx.x); \
        break;
            MDFFT_SERVE_LENGTHS(MDFFT_RUN)
#undef MDFFT_RUN
            default:
                break;
        }
        __syncthreads();  // shared memory is reused by the next tile
    }
}

// A line kernel (group G): warp w of the grid takes chunks of
// chunk_line[G] consecutive 32-line tiles of the group's items in turn; it
// copies an item's arguments to its own shared memory when it reaches the
// item's tiles (items are in increasing tile order, so lookups only
// advance).  No CTA barrier.  Registers: group 0 fits 4 CTAs per SM, group 1 2.
template <int G>
__global__ void __launch_bounds__(kLineThreads, G == 0 ? 4 : 2) serve_line_kernel(const Table *tab) {
    extern __shared__ __align__(16) unsigned char line_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wsm = line_smem + warp * line_warp_smem(G);
    PassArgs &args = *reinterpret_cast<PassArgs *>(wsm);
    float2 *stage = reinterpret_cast<float2 *>(wsm + kArgsBytes);
    int64_t *lbase = reinterpret_cast<int64_t *>(stage + 32 * kLineRs[G]);
    const Item *items = tab->items + tab->n + (G == 1 ? tab->n_line[0] : 0);
    const int n = tab->n_line[G];
    const int64_t total = tab->total_line[G];
    const int64_t chunk = tab->chunk_line[G];
    const int64_t gw = (int64_t)blockIdx.x * kLineWarps + warp, nw = (int64_t)gridDim.x * kLineWarps;
    int cur = -1, kind = -1;
    int64_t cur_start = 0, cur_end = 0;
    for (int64_t c0 = gw * chunk; c0 < total; c0 += nw * chunk)
        for (int64_t t = c0; t < c0 + chunk && t < total; ++t) {
            if (t >= cur_end) {  // the last item after cur starting at or before t
                int lo = cur + 1, hi = n - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (items[mid].start <= t) lo = mid;
                    else hi = mid - 1;
                }
                cur = lo;
                cur_start = items[cur].start;
                cur_end = cur + 1 < n ? items[cur + 1].start : total;
                __syncwarp();  // every lane is done with the previous arguments
                const int *src = reinterpret_cast<const int *>(&items[cur].args);
                int *dst = reinterpret_cast<int *>(&args);
                for (int w = lane; w < (int)(sizeof(PassArgs) / sizeof(int)); w += 32) dst[w] = src[w];
                kind = items[cur].kind;
                __syncwarp();
            }
            const TileCoord c = tile_coords(args, t - cur_start);
#define MDFFT_RUN(i, N)                                           \
    case kLineKind + i:                                           \
        line_warp<N>(args, c, 0, stage, lbase, lane);             \
        break;
            if constexpr (G == 0) {
                switch (kind) {
                    MDFFT_SERVE_LINE_GROUP0(MDFFT_RUN)
                    default:
                        break;
                }
            } else {
                switch (kind) {
                    MDFFT_SERVE_LINE_GROUP1(MDFFT_RUN)
                    default:
                        break;
                }
            }
#undef MDFFT_RUN
        }
}

// first-fit allocator over one device arena (offsets 256-byte aligned)
class Arena {
  public:
    void reset(size_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

struct Request {
    int64_t id = 0;
    mdfft_plan_t plan = nullptr;
    const void *in = nullptr;
    void *out = nullptr;
    int dir = -1, normalize = 0;
    size_t bytes = 0;     // budget charge: input + output + workspace
    size_t ws_off = 0;
    bool has_ws = false;
    int next_pass = 0;
    bool admitted = false, finished = false;
    double done_ms = -1.0;  // completion on the server clock
    int slot = -1;          // slot of the step that ran the last pass
    int last_slot = -1;     // slot of the latest step that ran one of its passes
    bool cancelled = false;
};

struct Slot {
    Table *host = nullptr;  // pinned
    Table *dev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy = nullptr;  // the table copy node (its size follows the step's item count)
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool direct = false;  // the step ran plain pass launches (low load)
    std::vector<Request *> finishing;
};

}  // namespace serve
}  // namespace mdfft

using namespace mdfft::serve;

struct ServePass {  // a plan's pass re-tiled for the persistent kernels
    PassArgs args;      // for the grouped kernel (kind >= 0)
    int64_t ctas;
    int kind;
    PassArgs line_args;  // for the line kernel (line_kind >= 0): 32-line tiles
    int64_t line_tiles;
    int line_kind;
};

struct mdfft_server_s {
    size_t budget = 0, in_use = 0;
    std::map<mdfft_plan_t, std::vector<ServePass>> retiled;
    int max_inflight = 0;
    int64_t P = 64;
    cudaStream_t stream = nullptr, capture = nullptr;
    int grid = 0;
    void *arena_mem = nullptr;
    size_t arena_bytes = 0;
    Arena arena;
    std::map<std::vector<int64_t>, mdfft_plan_t> plans;
    std::deque<Request *> queue;
    std::vector<Request *> inflight;
    std::unordered_map<int64_t, Request *> requests;
    int64_t next_id = 1;
    int depth = 2;  // steps in flight on the GPU at most; arrivals in between join the next step
    int chunk = 4;  // at most this many consecutive tiles dealt to a CTA at a time
    int direct = 4;  // low load: at most this many requests with passes left run them as plain launches
    int lines = 1;   // passes of 16 to 64 points go to the line kernels
    int line_grid[2] = {0, 0};
    cudaStream_t capture2[2] = {nullptr, nullptr};            // the line kernels' branches of the step graph
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};  // branches start after the table copy, the step ends after all
    Slot slots[kSlots];
    int next_slot = 0;
    cudaEvent_t t0 = nullptr;
    mdfft_server_stats stats{};
};

namespace {

mdfft_status capture_graphs(mdfft_server_t s) {
    for (Slot &sl : s->slots) {
        if (sl.exec) cudaGraphExecDestroy(sl.exec), sl.exec = nullptr;
        if (sl.graph) cudaGraphDestroy(sl.graph), sl.graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        cudaMemcpyAsync(sl.dev, sl.host, sizeof(Table), cudaMemcpyHostToDevice, s->capture);
        // the two kernels are parallel branches: the line kernel's CTAs take
        // SMs as the grouped kernel's CTAs finish, and the other way round
        cudaEventRecord(s->fork, s->capture);
        cudaStreamWaitEvent(s->capture2[0], s->fork, 0);
        cudaStreamWaitEvent(s->capture2[1], s->fork, 0);
        serve_kernel<<<s->grid, kThreads, kSmem, s->capture>>>(sl.dev);
        serve_line_kernel<0><<<s->line_grid[0], kLineThreads, kLineSmem[0], s->capture2[0]>>>(sl.dev);
        serve_line_kernel<1><<<s->line_grid[1], kLineThreads, kLineSmem[1], s->capture2[1]>>>(sl.dev);
        for (int g = 0; g < 2; ++g) {
            cudaEventRecord(s->join[g], s->capture2[g]);
            cudaStreamWaitEvent(s->capture, s->join[g], 0);
        }
        e = cudaStreamEndCapture(s->capture, &sl.graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&sl.exec, sl.graph, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        size_t nn = 0;
        cudaGraphGetNodes(sl.graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(sl.graph, nodes.data(), &nn);
        sl.copy = nullptr;
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeMemcpy) sl.copy = nd;
        }
    }
    return MDFFT_OK;
}

// Requests of a slot whose step has completed: record completion, free memory.
void resolve_slot(mdfft_server_t s, Slot &sl) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->t0, sl.done);
    for (Request *r : sl.finishing) {
        r->finished = true;
        r->done_ms = r->cancelled ? -1.0 : ms;
        if (r->has_ws) s->arena.release(r->ws_off, (size_t)r->plan->T * r->plan->elem);
        r->has_ws = false;
        s->in_use -= r->bytes;
        (r->cancelled ? s->stats.cancelled : s->stats.completed)++;
        s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), r));
    }
    sl.finishing.clear();
    sl.busy = false;
}

void poll_slots(mdfft_server_t s) {
    for (Slot &sl : s->slots)
        if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) resolve_slot(s, sl);
}

mdfft_status get_plan(mdfft_server_t s, int M, const int64_t *N, mdfft_plan_t *out) {
    std::vector<int64_t> key(N, N + M);
    auto it = s->plans.find(key);
    if (it != s->plans.end()) {
        *out = it->second;
        return MDFFT_OK;
    }
    int64_t T = 1;
    for (int i = 0; i < M; ++i) T *= N[i];
    mdfft_plan_t p = nullptr;
    mdfft_status st = mdfft::detail::plan_create(&p, M, N, std::min<int64_t>(s->P, T), nullptr, MDFFT_C64, 0, false, 1);
    if (st != MDFFT_OK) return st;
    s->plans[key] = p;
    std::vector<ServePass> rt(M);
    for (int q = 0; q < M; ++q) {
        rt[q].kind = kind_of(p->pass[q].n);
        rt[q].ctas = 0;
        if (rt[q].kind >= 0) mdfft::detail::retile_pass(p, q, lines_of_kind(rt[q].kind), &rt[q].args, &rt[q].ctas);
        rt[q].line_kind = line_kind_of(p->pass[q].n);
        rt[q].line_tiles = 0;
        if (rt[q].line_kind >= 0) mdfft::detail::retile_pass(p, q, 32, &rt[q].line_args, &rt[q].line_tiles);
    }
    s->retiled[p] = rt;
    *out = p;
    return MDFFT_OK;
}

// Pass s of request r as launch arguments (buffers as in mdfft_exec: the
// last pass writes out, earlier ones alternate with the request's workspace).
PassArgs pass_args(mdfft_server_t s, const Request *r, int pass) {
    const mdfft_plan_s *p = r->plan;
    const int M = p->M;
    void *ws = (char *)s->arena_mem + r->ws_off;
    const void *src = r->in;
    void *dst = nullptr;
    for (int q = 0; q <= pass; ++q) {
        // destination of pass q going backwards from out
        dst = ((M - 1 - q) % 2 == 0) ? r->out : ws;
        if (q < pass) src = dst;
    }
    PassArgs a = p->pass[pass].args;
    a.in = src;
    a.out = dst;
    a.tw = (const char *)p->tw + p->pass[pass].tw_offset;
    a.conj = r->dir == 1 ? (pass == 0 ? 1 : 0) | (pass == M - 1 ? 2 : 0) : 0;
    a.scale = (pass == M - 1 && r->normalize) ? 1.0 / (double)p->T : 1.0;
    a.scaled = a.scale != 1.0;
    return a;
}

}  // namespace

extern "C" {

mdfft_status mdfft_server_create(mdfft_server_t *out, size_t budget_bytes, int max_inflight, int64_t P,
                                 mdfft_stream_t stream) {
    if (!out) return fail(MDFFT_E_ARG, "null argument");
    *out = nullptr;
    if (budget_bytes < 4096 || max_inflight < 1 || max_inflight > kMaxItems || P < 1)
        return fail(MDFFT_E_ARG, "budget >= 4096 bytes, 1 <= max_inflight <= 512, P >= 1");
    mdfft_server_s *s = new (std::nothrow) mdfft_server_s;
    if (!s) return fail(MDFFT_E_NOMEM, "host allocation");
    s->budget = budget_bytes;
    s->max_inflight = max_inflight;
    s->P = P;
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    s->stats.budget_bytes = budget_bytes;
    auto bail = [&](mdfft_status st) {
        mdfft_server_destroy(s);
        return st;
    };
    cudaError_t e;
    // workspaces: one T-element array per request in flight; each request is
    // charged input + output + workspace, so workspaces use at most a third
    s->arena_bytes = (budget_bytes / 3 + 255) / 256 * 256;
    if ((e = cudaMalloc(&s->arena_mem, s->arena_bytes)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc arena"));
    s->arena.reset(s->arena_bytes);
    if ((e = cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s->capture2[0], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s->capture2[1], cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaStreamCreate"));
    if ((e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s->join[0], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s->join[1], cudaEventDisableTiming)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)) !=
        cudaSuccess)
        return bail(cuda_fail(e, "cudaFuncSetAttribute"));
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, kThreads, kSmem);
    s->grid = std::max(1, sms * std::max(1, per_sm));
    const void *line_fn[2] = {(const void *)serve_line_kernel<0>, (const void *)serve_line_kernel<1>};
    for (int g = 0; g < 2; ++g) {
        if ((e = cudaFuncSetAttribute(line_fn[g], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLineSmem[g])) !=
            cudaSuccess)
            return bail(cuda_fail(e, "cudaFuncSetAttribute"));
        int line_per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&line_per_sm, line_fn[g], kLineThreads, kLineSmem[g]);
        s->line_grid[g] = std::max(1, sms * std::max(1, line_per_sm));
    }
    for (Slot &sl : s->slots) {
        if ((e = cudaHostAlloc((void **)&sl.host, sizeof(Table), cudaHostAllocDefault)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaHostAlloc table"));
        std::memset(sl.host, 0, sizeof(Table));
        if ((e = cudaMalloc((void **)&sl.dev, sizeof(Table))) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMalloc table"));
        if ((e = cudaEventCreate(&sl.done)) != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    }
    mdfft_status st = capture_graphs(s);
    if (st != MDFFT_OK) return bail(st);
    s->stats.grid_ctas = s->grid;
    if ((e = cudaEventCreate(&s->t0)) != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    cudaEventRecord(s->t0, s->stream);
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return bail(cuda_fail(e, "cudaStreamSynchronize"));
    *out = s;
    return MDFFT_OK;
}

mdfft_status mdfft_server_submit(mdfft_server_t s, int M, const int64_t N[], const void *in_dev, void *out_dev,
                                 int dir, int normalize, int64_t *request_id) {
    if (!s || !N || !in_dev || !out_dev || !request_id) return fail(MDFFT_E_ARG, "null argument");
    if (dir != -1 && dir != 1) return fail(MDFFT_E_ARG, "dir must be -1 or +1");
    if (normalize != 0 && !(normalize == 1 && dir == 1)) return fail(MDFFT_E_ARG, "normalize only on the inverse");
    if ((uintptr_t)in_dev % 8 || (uintptr_t)out_dev % 8) return fail(MDFFT_E_ARG, "misaligned data pointer");
    mdfft_plan_t p = nullptr;
    mdfft_status st = get_plan(s, M, N, &p);
    if (st != MDFFT_OK) return st;
    const size_t bytes = (size_t)p->T * p->elem;
    const uintptr_t a = (uintptr_t)in_dev, b = (uintptr_t)out_dev;
    if (a < b + bytes && b < a + bytes) return fail(MDFFT_E_ARG, "in and out overlap");
    if (3 * bytes > s->budget) return fail(MDFFT_E_RANGE, "request larger than the whole HBM budget");
    Request *r = new (std::nothrow) Request;
    if (!r) return fail(MDFFT_E_NOMEM, "host allocation");
    r->id = s->next_id++;
    r->plan = p;
    r->in = in_dev;
    r->out = out_dev;
    r->dir = dir;
    r->normalize = normalize;
    r->bytes = 3 * bytes;
    s->requests[r->id] = r;
    s->queue.push_back(r);
    s->stats.submitted++;
    *request_id = r->id;
    return MDFFT_OK;
}

mdfft_status mdfft_server_step(mdfft_server_t s, int *launched) {
    if (!s) return fail(MDFFT_E_ARG, "null server");
    if (launched) *launched = 0;
    poll_slots(s);
    // admission: first come first served, within the budget, the slots and the arena
    while (!s->queue.empty() && (int)s->inflight.size() < s->max_inflight) {
        Request *r = s->queue.front();
        if (s->in_use + r->bytes > s->budget) break;
        size_t off = 0;
        if (!s->arena.alloc((size_t)r->plan->T * r->plan->elem, &off)) break;
        r->ws_off = off;
        r->has_ws = true;
        r->admitted = true;
        s->in_use += r->bytes;
        s->inflight.push_back(r);
        s->queue.pop_front();
        s->stats.admitted++;
    }
    std::vector<Request *> todo;
    for (Request *r : s->inflight)
        if (r->next_pass < r->plan->M) todo.push_back(r);
    if (todo.empty()) return MDFFT_OK;
    // low load: nothing queued and few requests with passes left -- they run
    // at once; the depth limit, which lets arrivals gather into fuller
    // steps, holds them back only while batched steps are in flight
    const bool direct = (int)todo.size() <= s->direct && s->queue.empty();
    int busy = 0, busy_batched = 0;
    for (const Slot &b : s->slots) busy += b.busy, busy_batched += b.busy && !b.direct;
    if (busy >= s->depth && (!direct || busy_batched > 0)) return MDFFT_OK;  // let more work gather
    Slot &sl = s->slots[s->next_slot];
    if (sl.busy) {  // its table may still be in use: wait for that step
        cudaError_t e = cudaEventSynchronize(sl.done);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        resolve_slot(s, sl);
    }
    cudaError_t e = cudaSuccess;
    if (direct) {
        // low load: every remaining pass of these requests, oldest first, as
        // plain pass launches (stream order keeps each request's passes in order)
        for (Request *r : todo) {
            for (int pass = r->next_pass; pass < r->plan->M; ++pass) {
                const mdfft::detail::Pass &ps = r->plan->pass[pass];
                PassArgs a = pass_args(s, r, pass);
                a.ntiles = ps.ctas;
                void *args[] = {&a};
                e = cudaLaunchKernel(ps.k.fn, dim3((unsigned)ps.grid), dim3(ps.k.threads), args, ps.k.smem, s->stream);
                if (e != cudaSuccess) return cuda_fail(e, "pass launch");
                s->stats.kernel_launches++;
            }
            r->next_pass = r->plan->M;
            r->last_slot = r->slot = s->next_slot;
            sl.finishing.push_back(r);
            s->stats.direct_requests++;
        }
        e = cudaEventRecord(sl.done, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        sl.busy = true;
        sl.direct = true;
        s->next_slot = (s->next_slot + 1) % kSlots;
        s->stats.steps++;
        if (launched) *launched = 1;
        return MDFFT_OK;
    }
    Table *tab = sl.host;
    int n = 0, n_line[2] = {0, 0};
    int64_t total = 0, total_line[2] = {0, 0};
    std::vector<std::pair<Request *, PassArgs>> separate;  // lengths the persistent kernels do not carry
    std::vector<Item> line_items[2];
    for (Request *r : todo) {
        if (n + n_line[0] + n_line[1] >= kMaxItems) break;
        const int pass = r->next_pass;
        const PassArgs a = pass_args(s, r, pass);
        const ServePass &sp = s->retiled[r->plan][pass];
        const bool al16 = (uintptr_t)a.in % 16 == 0 && (uintptr_t)a.out % 16 == 0;
        if (s->lines && sp.line_kind >= 0 && al16) {  // the same pass in 32-line tiles for a line kernel
            const int g = line_group(sp.line_kind);
            line_items[g].emplace_back();
            Item &it = line_items[g].back();
            it.args = sp.line_args;
            it.args.in = a.in, it.args.out = a.out, it.args.tw = a.tw;
            it.args.conj = a.conj, it.args.scale = a.scale, it.args.scaled = a.scaled;
            it.start = total_line[g];
            it.kind = sp.line_kind;
            total_line[g] += sp.line_tiles;
            n_line[g]++;
        } else if (sp.kind < 0) {
            separate.push_back({r, a});
        } else {  // the same pass re-tiled for the persistent kernel's CTA
            Item &it = tab->items[n++];
            it.args = sp.args;
            it.args.in = a.in, it.args.out = a.out, it.args.tw = a.tw;
            it.args.conj = a.conj, it.args.scale = a.scale, it.args.scaled = a.scaled;
            it.start = total;
            it.kind = sp.kind;
            total += sp.ctas;
        }
        r->next_pass++;
        r->last_slot = s->next_slot;
        if (r->next_pass == r->plan->M) {
            r->slot = s->next_slot;
            sl.finishing.push_back(r);
        }
    }
    tab->n = n;
    // the step's tiles spread over every CTA first: chunks of total / grid tiles, at most s->chunk
    tab->chunk = (int)std::max<int64_t>(1, std::min<int64_t>(s->chunk, total / std::max(1, s->grid)));
    tab->total = total;
    for (int g = 0, at = n; g < 2; ++g) {
        for (int i = 0; i < n_line[g]; ++i) tab->items[at++] = line_items[g][i];
        tab->n_line[g] = n_line[g];
        tab->chunk_line[g] = (int)std::max<int64_t>(
            1, std::min<int64_t>(s->chunk, total_line[g] / std::max<int64_t>(1, (int64_t)s->line_grid[g] * kLineWarps)));
        tab->total_line[g] = total_line[g];
    }
    const int n2 = n_line[0] + n_line[1];
    if (n + n2 > 0) {
        if (sl.copy) {  // copy only the header and the items of this step
            const size_t used = offsetof(Table, items) + (size_t)(n + n2) * sizeof(Item);
            e = cudaGraphExecMemcpyNodeSetParams1D(sl.exec, sl.copy, sl.dev, sl.host, used, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphExecMemcpyNodeSetParams1D");
        }
        e = cudaGraphLaunch(sl.exec, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        s->stats.graph_launches++;
        s->stats.kernel_launches++;
    }
    for (auto &pr : separate) {
        const mdfft::detail::Pass &ps = pr.first->plan->pass[pr.first->next_pass - 1];
        PassArgs a = pr.second;
        void *args[] = {&a};
        e = cudaLaunchKernel(ps.k.fn, dim3((unsigned)ps.ctas), dim3(ps.k.threads), args, ps.k.smem, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "pass launch");
        s->stats.kernel_launches++;
    }
    e = cudaEventRecord(sl.done, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    sl.busy = true;
    sl.direct = false;
    s->next_slot = (s->next_slot + 1) % kSlots;
    s->stats.steps++;
    if (launched) *launched = 1;
    return MDFFT_OK;
}

mdfft_status mdfft_server_run(mdfft_server_t s, int max_steps, int *steps) {
    if (!s) return fail(MDFFT_E_ARG, "null server");
    int n = 0;
    for (; n < max_steps; ++n) {
        int launched = 0;
        mdfft_status st = mdfft_server_step(s, &launched);
        if (st != MDFFT_OK) return st;
        if (!launched) break;
    }
    if (steps) *steps = n;
    return MDFFT_OK;
}

mdfft_status mdfft_server_poll(mdfft_server_t s, int64_t request_id, int *done, double *done_ms) {
    if (!s || !done) return fail(MDFFT_E_ARG, "null argument");
    auto it = s->requests.find(request_id);
    if (it == s->requests.end()) return fail(MDFFT_E_ARG, "unknown request id");
    Request *r = it->second;
    if (!r->finished && r->slot >= 0) {
        Slot &sl = s->slots[r->slot];
        if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) resolve_slot(s, sl);
    }
    *done = r->finished ? 1 : 0;
    if (done_ms) *done_ms = r->finished ? r->done_ms : -1.0;
    return MDFFT_OK;
}

mdfft_status mdfft_server_release(mdfft_server_t s, int64_t request_id) {
    if (!s) return fail(MDFFT_E_ARG, "null server");
    auto it = s->requests.find(request_id);
    if (it == s->requests.end()) return fail(MDFFT_E_ARG, "unknown request id");
    if (!it->second->finished) return fail(MDFFT_E_ARG, "request not finished");
    delete it->second;
    s->requests.erase(it);
    return MDFFT_OK;
}

mdfft_status mdfft_server_cancel(mdfft_server_t s, int64_t request_id) {
    if (!s) return fail(MDFFT_E_ARG, "null server");
    auto it = s->requests.find(request_id);
    if (it == s->requests.end()) return fail(MDFFT_E_ARG, "unknown request id");
    Request *r = it->second;
    if (r->finished || r->cancelled) return fail(MDFFT_E_ARG, "request already finished or cancelled");
    if (!r->admitted) {  // still queued: it never reached the GPU
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
        r->cancelled = r->finished = true;
        r->done_ms = -1.0;
        s->stats.cancelled++;
        return MDFFT_OK;
    }
    if (r->next_pass == r->plan->M) return MDFFT_OK;  // its last pass is on the GPU: it completes
    r->cancelled = true;
    r->next_pass = r->plan->M;  // no further passes are scheduled
    Slot *last = r->last_slot >= 0 ? &s->slots[r->last_slot] : nullptr;
    if (last && last->busy) {  // resources come back when its latest step has run
        r->slot = r->last_slot;
        last->finishing.push_back(r);
    } else {  // nothing of it is on the GPU
        r->finished = true;
        r->done_ms = -1.0;
        if (r->has_ws) s->arena.release(r->ws_off, (size_t)r->plan->T * r->plan->elem);
        r->has_ws = false;
        s->in_use -= r->bytes;
        s->stats.cancelled++;
        s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), r));
    }
    return MDFFT_OK;
}

mdfft_status mdfft_server_drain(mdfft_server_t s) {
    if (!s) return fail(MDFFT_E_ARG, "null server");
    while (!s->queue.empty() || !s->inflight.empty()) {
        int launched = 0;
        mdfft_status st = mdfft_server_step(s, &launched);
        if (st != MDFFT_OK) return st;
        if (!launched) {  // nothing to launch until a step completes: wait for the oldest one only
            for (int k = 0; k < kSlots; ++k) {
                Slot &sl = s->slots[(s->next_slot + k) % kSlots];
                if (!sl.busy) continue;
                cudaError_t e = cudaEventSynchronize(sl.done);
                if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
                resolve_slot(s, sl);
                break;
            }
        }
    }
    return MDFFT_OK;
}

mdfft_status mdfft_server_reset_clock(mdfft_server_t s) {
    if (!s) return fail(MDFFT_E_ARG, "null server");
    cudaEventRecord(s->t0, s->stream);
    cudaError_t e = cudaEventSynchronize(s->t0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    return MDFFT_OK;
}

mdfft_status mdfft_server_set_grid(mdfft_server_t s, int ctas) {
    if (!s || ctas < 1) return fail(MDFFT_E_ARG, "bad argument");
    for (Slot &sl : s->slots)
        if (sl.busy) {
            cudaError_t e = cudaEventSynchronize(sl.done);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
            resolve_slot(s, sl);
        }
    s->grid = ctas;
    s->stats.grid_ctas = ctas;
    return capture_graphs(s);
}

mdfft_status mdfft_server_set_line_kernel(mdfft_server_t s, int enable) {
    if (!s || (enable != 0 && enable != 1)) return fail(MDFFT_E_ARG, "enable must be 0 or 1");
    s->lines = enable;
    return MDFFT_OK;
}

mdfft_status mdfft_server_set_chunk(mdfft_server_t s, int chunk) {
    if (!s || chunk < 1 || chunk > 64) return fail(MDFFT_E_ARG, "chunk must be in [1, 64]");
    s->chunk = chunk;
    return MDFFT_OK;
}

mdfft_status mdfft_server_set_direct(mdfft_server_t s, int max_requests) {
    if (!s || max_requests < 0 || max_requests > 64) return fail(MDFFT_E_ARG, "direct threshold must be in [0, 64]");
    s->direct = max_requests;
    return MDFFT_OK;
}

mdfft_status mdfft_server_set_depth(mdfft_server_t s, int depth) {
    if (!s || depth < 1 || depth > kSlots) return fail(MDFFT_E_ARG, "depth must be in [1, 8]");
    s->depth = depth;
    return MDFFT_OK;
}

mdfft_status mdfft_server_get_stats(mdfft_server_t s, mdfft_server_stats *out) {
    if (!s || !out) return fail(MDFFT_E_ARG, "null argument");
    s->stats.inflight = (int64_t)s->inflight.size();
    s->stats.queued = (int64_t)s->queue.size();
    s->stats.bytes_in_use = s->in_use;
    *out = s->stats;
    return MDFFT_OK;
}

mdfft_status mdfft_server_destroy(mdfft_server_t s) {
    if (!s) return MDFFT_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Slot &sl : s->slots) {
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.graph) cudaGraphDestroy(sl.graph);
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (s->t0) cudaEventDestroy(s->t0);
    if (s->capture) cudaStreamDestroy(s->capture);
    for (int g = 0; g < 2; ++g) {
        if (s->capture2[g]) cudaStreamDestroy(s->capture2[g]);
        if (s->join[g]) cudaEventDestroy(s->join[g]);
    }
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->arena_mem) cudaFree(s->arena_mem);
    for (auto &kv : s->plans) mdfft_destroy(kv.second);
    for (auto &kv : s->requests) delete kv.second;
    delete s;
    return MDFFT_OK;
}

}  // extern "C"
