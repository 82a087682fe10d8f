// planner.h -- host-side row-wise decomposition planner (integer maths only).
//
// Layouts are permutations of axis ids listed slowest -> fastest.  The
// chunks of a layout are the f_MD chunks (Sec. 3.2) of the dims permuted into
// that layout.  Amounts are in data points.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace mdfft {
namespace planner {

constexpr int kMaxDims = 8;

struct Layout {
    int M = 0;
    int axis[kMaxDims] = {0};
};

// Number of leading dims the chunks are cut on (smallest k with
// P <= d_0 ... d_{k-1}); -1 if P < 1 or P > product(d).
int regime(int M, const int64_t *d, int64_t P);

// f_MD of Sec. 3.2 over dims d (already in layout order); pid in [0, P].
int64_t fmd(int M, const int64_t *d, int64_t P, int64_t pid);

// Mixed-radix digits of x over dims d.
void digits(int M, const int64_t *d, int64_t x, int64_t *c);

// Dims of N permuted into layout L.
void layout_dims(const Layout &L, const int64_t *N, int64_t *d);

// Half-open axis-aligned box in natural axis coordinates.
struct Box {
    int64_t lo[kMaxDims];
    int64_t hi[kMaxDims];
};

// Boxes (natural coordinates) covering layout-L row-major indices [a, b).
void range_boxes(const Layout &L, const int64_t *N, int64_t a, int64_t b, std::vector<Box> &out);

// Points whose owner differs between the chunks of layouts A and B.
int64_t transition_amount(int M, const int64_t *N, int64_t P, const Layout &A, const Layout &B);

// Split-line amount of layout L: sum over lines along its last axis of
// N_axis * (owners - 1).
int64_t split_line_amount(int M, const int64_t *N, int64_t P, const Layout &L);

// Owner of row-major index x of layout L (closed form inverse of f_MD).
int64_t owner_of(int M, const int64_t *N, int64_t P, const Layout &L, int64_t x);

// Validates an order of M layouts: first natural, each a permutation, last
// axes all distinct.  Returns "" or a message.
std::string check_order(int M, const std::vector<Layout> &order);

// Dynamic-programming order search (M <= 6).  want_worst selects max.
// Ties: lexicographically smallest sequence of layouts.
bool search_order(int M, const int64_t *N, int64_t P, bool want_worst, std::vector<Layout> &order,
                  int64_t &total, std::string &err);

// All-to-all-v counts of the transition A -> B when the P processes are laid
// onto G devices in contiguous blocks (device g holds processes
// floor(g P / G) .. floor((g+1) P / G) - 1, a contiguous row-major range):
// counts[g * G + h] = points held by g in A and by h in B.
void exchange_counts(int M, const int64_t *N, int64_t P, const Layout &A, const Layout &B, int G, int64_t *counts);

// Balanced-split heuristic for any M >= 2 (the form the paper suggests for
// higher dimensions, Sec. 3.3): axes split X | Y; first every axis of Y is
// transformed with X in front (layouts X . perm(Y)), then a permutation of Y
// moves to the front and the axes of X are transformed (layouts perm(Y) .
// perm(X)).  Each next layout is the one of that family with the smallest
// amount from the current layout (ties: lexicographically smallest); both
// splits |X| = floor(M/2) and ceil(M/2) are tried and the smaller total kept.
bool heuristic_order(int M, const int64_t *N, int64_t P, std::vector<Layout> &order, int64_t &total,
                     std::string &err);

// The comparison methods of Sec. 4 as block decompositions.  k axes are cut
// at a time (1: the 1-D or slab method, 2: the 2-D or pencil method, M: the
// volumetric M-D methods); step s transforms the last axis of order[s].
// With k < M the transformed axis is never cut: when the next step's axis is
// cut, that cut moves to the axis just transformed (the methods' transposes).
// Readings: the first step cuts the k slowest axes; P is split over the cuts
// as evenly as possible (prime factors, largest first, each to the cut with
// the smallest product, the first on ties); cut 0 varies slowest in the
// process id; a cut of n points into q blocks gives block j the points
// [floor(j n / q), floor((j + 1) n / q)) and needs q <= n.
enum BlockKind { kRowwise = 0, kSlab = 1, kPencil = 2, kVolumetric = 3 };

struct BlockDecomp {
    int kind = kRowwise;
    int k = 0;                           // cut axes per step
    int64_t q[kMaxDims] = {0};           // blocks of cut j
    int cut[kMaxDims][kMaxDims] = {{0}}; // [step][j]: natural axis of cut j
};

bool block_decomposition(int M, const int64_t *N, int64_t P, int kind, const std::vector<Layout> &order,
                         BlockDecomp &bd, std::string &err);

// Blocks along every natural axis in step s (1: not cut) and the process-id
// stride of that axis (0: not cut).
void block_axis_grid(const BlockDecomp &bd, int M, int s, int64_t *q_axis, int64_t *ps_axis);

// Points whose owner differs between steps s and s+1 (box intersection per process).
int64_t block_transition_amount(int M, const int64_t *N, int64_t P, const BlockDecomp &bd, int s);

// Lines of step s shared by several owners, each gathering the whole line:
// sum over lines of N_axis (owners - 1) = T (q - 1) when the axis is cut.
int64_t block_split_amount(int M, const int64_t *N, const BlockDecomp &bd, const std::vector<Layout> &order, int s);

}  // namespace planner
}  // namespace mdfft
