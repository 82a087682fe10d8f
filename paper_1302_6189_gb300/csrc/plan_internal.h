// plan_internal.h -- the plan object and helpers shared by the translation
// units of libmdfft (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mdfft.h"
#include "passes.h"
#include "planner.h"

namespace mdfft {
namespace detail {

struct Pass {
    int f = 0, g = 0, h = -1;  // transformed axis, output's fastest axis, next tile axis
    int64_t n = 0;             // line length N_f
    PassKernel k{};
    PassArgs args{};           // everything but in/out/tw/conj/scale/count pointers
    int64_t ctas = 0;          // tiles
    int64_t grid = 0;          // CTAs launched (= ctas, or one wave for persistent kernels)
    size_t tw_offset = 0;      // byte offset of this pass's twiddle table (room for 2 n entries: any radix plan)
    int mapping = 0;           // tile order: 0 output-coalesced, 1 input-chunk order (see layout_pass)
};

// CTAs of one wave of kernel k on the current device (at least 1).
int64_t wave_ctas(const PassKernel &k);

// Records the message for mdfft_last_error() on this thread; returns st.
mdfft_status fail(mdfft_status st, const std::string &msg);
mdfft_status cuda_fail(cudaError_t e, const char *what);

// mdfft_plan without the plan's own workspace (its owner supplies one per
// execution, as the server does).  exec on such a plan is refused.
mdfft_status plan_create(mdfft_plan_t *out, int M, const int64_t N[], int64_t P, const int *order, mdfft_dtype dt,
                         unsigned flags, bool with_workspace, int64_t batch);

}  // namespace detail
}  // namespace mdfft

struct mdfft_plan_s;

namespace mdfft {
namespace detail {
// Launch arguments of pass s re-tiled for a CTA of `lines` lines (same
// arithmetic per line, so the same results); *ctas receives the tile count.
void retile_pass(const mdfft_plan_s *p, int s, int lines, PassArgs *a, int64_t *ctas);
}  // namespace detail
}  // namespace mdfft

struct mdfft_plan_s {
    int M = 0;
    int64_t N[MDFFT_MAX_DIMS] = {0};
    int64_t P = 0, T = 0;
    int64_t batch = 1;            // transforms per execution, volume v at element offset v T
    mdfft_dtype dt = MDFFT_C64;
    unsigned flags = 0;
    size_t elem = 8;
    std::vector<mdfft::planner::Layout> order;
    mdfft::detail::Pass pass[MDFFT_MAX_DIMS];
    void *tw = nullptr, *ws = nullptr, *ws2 = nullptr;
    int *err = nullptr;           // device flag set by a persistent kernel whose bounded wait gave up
    bool external_ws = false;     // made by plan_create(..., with_workspace = false)
    size_t tw_bytes = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // MDFFT_TIMING_SLOTS x (M + 1) events, made on first enable
    int64_t timed = 0;            // executions recorded since the last enable
    bool comm_ready = false;
    mdfft_comm comm{};
    mdfft::planner::BlockDecomp bd;  // comparison method of the counted amounts (kind kRowwise: f_MD chunks)
    // pipelined host execution of a batch (made on first use): streams for
    // host-to-device copies, passes and device-to-host copies, and events
    // (fork, copied in, computed, done)
    cudaStream_t hs[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t hev[4] = {nullptr, nullptr, nullptr, nullptr};
    // mdfft_exec_graph: the passes captured per (in, out, dir, normalize), least recently used replaced
    struct GraphEntry {
        const void *in = nullptr;
        void *out = nullptr;
        int dir = 0, normalize = 0;
        cudaGraphExec_t exec = nullptr;
        uint64_t used = 0;
    };
    std::vector<GraphEntry> graphs;
    uint64_t graph_tick = 0;
    cudaStream_t capture = nullptr;  // private stream the passes are captured on
    // distributed data plane: copy boxes per (step, G, device, pack) in device memory, made on first use
    struct DistBoxes {
        std::vector<int64_t> key;
        void *dev = nullptr;
        int n = 0;
        int64_t total = 0;
    };
    std::vector<DistBoxes> dist_boxes;
};
