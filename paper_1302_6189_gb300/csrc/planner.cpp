// planner.cpp -- row-wise adaptive decomposition planner (host, integers).
//
// Follows Sec. 3.1-3.2 of Duy and Ozaki (arXiv:1302.6189): the f_MD chunk
// function, its start/end coordinates, the communication amount of a
// transpose (points whose owner changes; the rest are reused, Sec. 1 and the
// text on Fig. 2) and the order count of the C_MD equation.  Amounts are
// computed by intersecting the boxes that make up each chunk, and the order
// search is a dynamic programme over (step, layout, axes already
// transformed) that does not enumerate orders (on grids of up to 2^16 points
// it compares owner arrays, one per ownership class of layouts).
#include "planner.h"

#include <algorithm>
#include <cstring>

namespace mdfft {
namespace planner {

typedef unsigned __int128 u128;

int regime(int M, const int64_t *d, int64_t P) {
    if (M < 1 || M > kMaxDims || P < 1) return -1;
    u128 prod = 1;
    for (int k = 0; k < M; ++k) {
        if (d[k] < 1) return -1;
        prod *= (u128)d[k];
        if ((u128)P <= prod) return k + 1;
    }
    return -1;
}

int64_t fmd(int M, const int64_t *d, int64_t P, int64_t pid) {
    int k = regime(M, d, P);
    if (k < 0 || pid < 0 || pid > P) return -1;
    u128 lead = 1, tail = 1;
    for (int i = 0; i < M; ++i) (i < k ? lead : tail) *= (u128)d[i];
    return (int64_t)(((lead * (u128)pid) / (u128)P) * tail);
}

void digits(int M, const int64_t *d, int64_t x, int64_t *c) {
    for (int i = M - 1; i >= 0; --i) {
        c[i] = x % d[i];
        x /= d[i];
    }
}

void layout_dims(const Layout &L, const int64_t *N, int64_t *d) {
    for (int i = 0; i < L.M; ++i) d[i] = N[L.axis[i]];
}

int64_t owner_of(int M, const int64_t *N, int64_t P, const Layout &L, int64_t x) {
    int64_t d[kMaxDims];
    layout_dims(L, N, d);
    int k = regime(M, d, P);
    u128 lead = 1, tail = 1;
    for (int i = 0; i < M; ++i) (i < k ? lead : tail) *= (u128)d[i];
    u128 q = (u128)x / tail;  // index over the k leading dims
    // largest p with floor(lead * p / P) <= q
    return (int64_t)(((q + 1) * (u128)P - 1) / lead);
}

// Row-major range [a, b) over dims d (layout order) -> boxes in layout
// coordinates, recursing from the slowest dim: a partial head slab, a run of
// whole slabs, a partial tail slab.
static void boxes_rec(int M, const int64_t *d, int level, int64_t a, int64_t b, int64_t *lo, int64_t *hi,
                      std::vector<Box> &out, const int *axis) {
    if (a >= b) return;
    int64_t stride = 1;
    for (int i = level + 1; i < M; ++i) stride *= d[i];
    if (level == M - 1) {
        lo[level] = a, hi[level] = b;
        Box bx;
        for (int i = 0; i < M; ++i) bx.lo[axis[i]] = lo[i], bx.hi[axis[i]] = hi[i];
        out.push_back(bx);
        return;
    }
    int64_t qa = a / stride, ra = a % stride, qb = b / stride, rb = b % stride;
    if (qa == qb) {
        lo[level] = qa, hi[level] = qa + 1;
        boxes_rec(M, d, level + 1, ra, rb, lo, hi, out, axis);
        return;
    }
    if (ra != 0) {
        lo[level] = qa, hi[level] = qa + 1;
        boxes_rec(M, d, level + 1, ra, stride, lo, hi, out, axis);
        ++qa;
    }
    if (qa < qb) {
        lo[level] = qa, hi[level] = qb;
        for (int i = level + 1; i < M; ++i) lo[i] = 0, hi[i] = d[i];
        Box bx;
        for (int i = 0; i < M; ++i) bx.lo[axis[i]] = lo[i], bx.hi[axis[i]] = hi[i];
        out.push_back(bx);
    }
    if (rb != 0) {
        lo[level] = qb, hi[level] = qb + 1;
        boxes_rec(M, d, level + 1, 0, rb, lo, hi, out, axis);
    }
}

void range_boxes(const Layout &L, const int64_t *N, int64_t a, int64_t b, std::vector<Box> &out) {
    int64_t d[kMaxDims], lo[kMaxDims], hi[kMaxDims];
    layout_dims(L, N, d);
    boxes_rec(L.M, d, 0, a, b, lo, hi, out, L.axis);
}

static int64_t overlap(int M, const Box &x, const Box &y) {
    int64_t v = 1;
    for (int i = 0; i < M; ++i) {
        int64_t lo = std::max(x.lo[i], y.lo[i]), hi = std::min(x.hi[i], y.hi[i]);
        if (hi <= lo) return 0;
        v *= hi - lo;
    }
    return v;
}

int64_t transition_amount(int M, const int64_t *N, int64_t P, const Layout &A, const Layout &B) {
    int64_t da[kMaxDims], db[kMaxDims], T = 1;
    layout_dims(A, N, da);
    layout_dims(B, N, db);
    for (int i = 0; i < M; ++i) T *= N[i];
    int64_t kept = 0;
    std::vector<Box> ba, bb;
    for (int64_t p = 0; p < P; ++p) {
        ba.clear(), bb.clear();
        range_boxes(A, N, fmd(M, da, P, p), fmd(M, da, P, p + 1), ba);
        range_boxes(B, N, fmd(M, db, P, p), fmd(M, db, P, p + 1), bb);
        for (const Box &x : ba)
            for (const Box &y : bb) kept += overlap(M, x, y);
    }
    return T - kept;
}

int64_t split_line_amount(int M, const int64_t *N, int64_t P, const Layout &L) {
    // A chunk boundary that is not a multiple of the line length falls
    // inside a line and gives that line one more owner (chunks are never
    // empty because P <= T).
    int64_t d[kMaxDims];
    layout_dims(L, N, d);
    int64_t nf = d[M - 1], cuts = 0;
    for (int64_t p = 1; p < P; ++p) cuts += (fmd(M, d, P, p) % nf) != 0;
    return nf * cuts;
}

void exchange_counts(int M, const int64_t *N, int64_t P, const Layout &A, const Layout &B, int G, int64_t *counts) {
    int64_t da[kMaxDims], db[kMaxDims];
    layout_dims(A, N, da);
    layout_dims(B, N, db);
    std::vector<std::vector<Box>> ba(G), bb(G);
    for (int g = 0; g < G; ++g) {
        const int64_t p0 = (int64_t)g * P / G, p1 = (int64_t)(g + 1) * P / G;
        range_boxes(A, N, fmd(M, da, P, p0), fmd(M, da, P, p1), ba[g]);
        range_boxes(B, N, fmd(M, db, P, p0), fmd(M, db, P, p1), bb[g]);
    }
    for (int g = 0; g < G; ++g)
        for (int h = 0; h < G; ++h) {
            int64_t c = 0;
            for (const Box &x : ba[g])
                for (const Box &y : bb[h]) c += overlap(M, x, y);
            counts[(size_t)g * G + h] = c;
        }
}

std::string check_order(int M, const std::vector<Layout> &order) {
    if ((int)order.size() != M) return "order must have M layouts";
    bool used_last[kMaxDims] = {false};
    for (int s = 0; s < M; ++s) {
        bool seen[kMaxDims] = {false};
        for (int i = 0; i < M; ++i) {
            int a = order[s].axis[i];
            if (a < 0 || a >= M || seen[a]) return "layout " + std::to_string(s) + " is not a permutation";
            seen[a] = true;
            if (s == 0 && a != i) return "layout 0 must be the natural order";
        }
        int last = order[s].axis[M - 1];
        if (used_last[last]) return "layout " + std::to_string(s) + " transforms an axis twice";
        used_last[last] = true;
    }
    return "";
}

// ---------------------------------------------------------------- order search

namespace {

// The owner of a point in layout L depends only on the coordinates of L's
// first k axes (k = L's regime, Sec. 3.2): layouts with the same first k
// axes, in the same order, have the same ownership.  The search computes one
// amount per pair of such keys.  On small grids an amount is a count over
// the owner arrays of the two keys (T points), else box intersection.
struct SearchCtx {
    int M;
    const int64_t *N;
    int64_t P, T;
    bool worst;
    std::vector<Layout> perms;
    std::vector<int> key;                     // key id of every layout
    std::vector<int> key_rep;                 // a layout of every key
    std::vector<std::vector<int32_t>> owners; // owner array (natural index order) per key, on demand
    std::vector<int64_t> pair;     // lazily filled amounts per key pair, -1 = unknown
    std::vector<int64_t> memo;     // [layer][perm][mask], INT64_MIN = unknown
    int F, K, masks;
    static constexpr int64_t kOwnerArrayPoints = 1 << 16;

    const std::vector<int32_t> &owner_array(int k) {
        std::vector<int32_t> &o = owners[k];
        if (o.empty()) {
            const Layout &L = perms[key_rep[k]];
            int64_t st[kMaxDims], s = 1;  // stride in L of every natural axis
            for (int i = M - 1; i >= 0; --i) st[L.axis[i]] = s, s *= N[L.axis[i]];
            int64_t d[kMaxDims];
            layout_dims(L, N, d);
            const int kr = regime(M, d, P);
            int64_t lead = 1, tail = 1;
            for (int i = 0; i < M; ++i) (i < kr ? lead : tail) *= d[i];
            o.resize((size_t)T);
            int64_t c[kMaxDims];
            for (int64_t x = 0; x < T; ++x) {  // owner_of() of the point, its q = y / tail
                digits(M, N, x, c);
                int64_t y = 0;
                for (int i = 0; i < M; ++i) y += c[i] * st[i];
                o[(size_t)x] = (int32_t)(((y / tail + 1) * P - 1) / lead);
            }
        }
        return o;
    }

    int64_t amount(int f, int g) {
        const int a = key[f], b = key[g];
        int64_t &v = pair[(size_t)a * K + b];
        if (v < 0) {
            if (a == b) {
                v = 0;
            } else if (T <= kOwnerArrayPoints) {
                const std::vector<int32_t> &oa = owner_array(a);
                const std::vector<int32_t> &ob = owner_array(b);
                int64_t moved = 0;
                for (int64_t x = 0; x < T; ++x) moved += oa[(size_t)x] != ob[(size_t)x];
                v = moved;
            } else {
                v = transition_amount(M, N, P, perms[f], perms[g]);
            }
        }
        return v;
    }
    bool better(int64_t a, int64_t b) const { return worst ? a > b : a < b; }

    int64_t &slot(int layer, int f, unsigned mask) { return memo[((size_t)layer * F + f) * masks + mask]; }

    // optimal sum of transitions from layout f at `layer` to the last layer
    int64_t solve(int layer, int f, unsigned mask) {
        if (layer == M - 1) return 0;
        int64_t &m = slot(layer, f, mask);
        if (m != INT64_MIN) return m;
        bool have = false;
        int64_t best = 0;
        for (int g = 0; g < F; ++g) {
            int last = perms[g].axis[M - 1];
            if (mask & (1u << last)) continue;
            int64_t v = amount(f, g) + solve(layer + 1, g, mask | (1u << last));
            if (!have || better(v, best)) best = v, have = true;
        }
        m = best;
        return m;
    }
};

}  // namespace

bool search_order(int M, const int64_t *N, int64_t P, bool want_worst, std::vector<Layout> &order,
                  int64_t &total, std::string &err) {
    if (M < 2 || M > 6) {
        err = "order search supports 2 <= M <= 6";
        return false;
    }
    int64_t T = 1;
    for (int i = 0; i < M; ++i) {
        if (N[i] < 1) {
            err = "dims must be >= 1";
            return false;
        }
        T *= N[i];
    }
    if (P < 1 || P > T) {
        err = "P out of range";
        return false;
    }
    SearchCtx c;
    c.M = M, c.N = N, c.P = P, c.T = T, c.worst = want_worst;
    int ids[kMaxDims];
    for (int i = 0; i < M; ++i) ids[i] = i;
    std::vector<std::vector<int>> keys;
    do {  // lexicographic permutations; index 0 is the natural layout
        Layout L;
        L.M = M;
        std::memcpy(L.axis, ids, sizeof(int) * M);
        int64_t d[kMaxDims];
        layout_dims(L, N, d);
        std::vector<int> k(ids, ids + regime(M, d, P));
        const size_t id = std::find(keys.begin(), keys.end(), k) - keys.begin();
        if (id == keys.size()) keys.push_back(k), c.key_rep.push_back((int)c.perms.size());
        c.key.push_back((int)id);
        c.perms.push_back(L);
    } while (std::next_permutation(ids, ids + M));
    c.F = (int)c.perms.size();
    c.K = (int)keys.size();
    c.masks = 1 << M;
    // the exact search must stay affordable: amounts of every key pair
    const double per_pair = T <= SearchCtx::kOwnerArrayPoints ? (double)T : (double)P * 4.0 * M * M;
    if ((double)c.K * c.K * per_pair > 4e10) {
        err = "the exact order search is too large for this grid and P (use the heuristic)";
        return false;
    }
    c.owners.resize(c.K);
    c.pair.assign((size_t)c.K * c.K, -1);
    c.memo.assign((size_t)M * c.F * c.masks, INT64_MIN);

    unsigned mask = 1u << (M - 1);
    total = c.solve(0, 0, mask);
    order.clear();
    order.push_back(c.perms[0]);
    int f = 0;
    for (int layer = 0; layer + 1 < M; ++layer) {
        int64_t want = c.solve(layer, f, mask);
        for (int g = 0; g < c.F; ++g) {
            int last = c.perms[g].axis[M - 1];
            if (mask & (1u << last)) continue;
            if (c.amount(f, g) + c.solve(layer + 1, g, mask | (1u << last)) == want) {
                order.push_back(c.perms[g]);
                f = g;
                mask |= 1u << last;
                break;
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------- heuristic

namespace {

// permutations of v in lexicographic order
std::vector<std::vector<int>> perms_of(std::vector<int> v) {
    std::sort(v.begin(), v.end());
    std::vector<std::vector<int>> out;
    do out.push_back(v);
    while (std::next_permutation(v.begin(), v.end()));
    return out;
}

Layout cat(int M, const std::vector<int> &front, const std::vector<int> &back) {
    Layout L;
    L.M = M;
    int i = 0;
    for (int a : front) L.axis[i++] = a;
    for (int a : back) L.axis[i++] = a;
    return L;
}

bool lex_less(const Layout &a, const Layout &b) {
    for (int i = 0; i < a.M; ++i)
        if (a.axis[i] != b.axis[i]) return a.axis[i] < b.axis[i];
    return false;
}

int64_t split_order(int M, const int64_t *N, int64_t P, int p, std::vector<Layout> &order) {
    std::vector<int> X, Y;
    for (int i = 0; i < M; ++i) (i < p ? X : Y).push_back(i);
    const auto px = perms_of(X), py = perms_of(Y);
    order.clear();
    order.push_back(cat(M, X, Y));
    unsigned used = 1u << (M - 1);
    int64_t total = 0;
    auto pick = [&](const std::vector<Layout> &family) {
        const Layout &cur = order.back();
        bool have = false;
        int64_t best = 0;
        Layout bestL;
        for (const Layout &L : family) {
            const int last = L.axis[M - 1];
            if (used & (1u << last)) continue;
            const int64_t v = transition_amount(M, N, P, cur, L);
            if (!have || v < best || (v == best && lex_less(L, bestL))) have = true, best = v, bestL = L;
        }
        order.push_back(bestL);
        used |= 1u << bestL.axis[M - 1];
        total += best;
    };
    std::vector<Layout> fam1, fam2;
    for (const auto &y : py) fam1.push_back(cat(M, X, y));
    for (const auto &y : py)
        for (const auto &x : px) fam2.push_back(cat(M, y, x));
    for (size_t k = 1; k < Y.size(); ++k) pick(fam1);  // the rest of Y, X in front
    for (size_t k = 0; k < X.size(); ++k) pick(fam2);  // Y in front, the axes of X
    return total;
}

}  // namespace

bool heuristic_order(int M, const int64_t *N, int64_t P, std::vector<Layout> &order, int64_t &total,
                     std::string &err) {
    if (M < 2 || M > kMaxDims) {
        err = "heuristic supports 2 <= M <= 8";
        return false;
    }
    int64_t T = 1;
    for (int i = 0; i < M; ++i) {
        if (N[i] < 1) {
            err = "dims must be >= 1";
            return false;
        }
        T *= N[i];
    }
    if (P < 1 || P > T) {
        err = "P out of range";
        return false;
    }
    bool have = false;
    for (int p : {M / 2, (M + 1) / 2}) {
        if (p < 1 || p >= M) continue;
        std::vector<Layout> o;
        const int64_t t = split_order(M, N, P, p, o);
        if (!have || t < total) order = o, total = t, have = true;
    }
    return have;
}

bool block_decomposition(int M, const int64_t *N, int64_t P, int kind, const std::vector<Layout> &order,
                         BlockDecomp &bd, std::string &err) {
    bd = BlockDecomp();
    bd.kind = kind;
    if (kind == kRowwise) return true;
    if (kind != kSlab && kind != kPencil && kind != kVolumetric) {
        err = "unknown decomposition";
        return false;
    }
    const int k = kind == kVolumetric ? M : kind;
    if (k > M || (kind == kPencil && M < 3)) {
        err = "the pencil method needs M >= 3";
        return false;
    }
    bd.k = k;
    // P's prime factors, largest first, each to the cut with the smallest product
    std::vector<int64_t> primes;
    int64_t r = P;
    for (int64_t f = 2; f <= r / f; ++f)
        for (; r % f == 0; r /= f) primes.push_back(f);
    if (r > 1) primes.push_back(r);
    std::sort(primes.rbegin(), primes.rend());
    for (int j = 0; j < k; ++j) bd.q[j] = 1;
    for (int64_t f : primes) {
        int lo = 0;
        for (int j = 1; j < k; ++j)
            if (bd.q[j] < bd.q[lo]) lo = j;
        bd.q[lo] *= f;
    }
    static const char *names[] = {"", "slab", "pencil", "volumetric"};
    for (int s = 0; s < M; ++s) {
        const int f = order[s].axis[M - 1];
        for (int j = 0; j < k; ++j) {
            if (s == 0)
                bd.cut[0][j] = j;
            else {
                const int prev = bd.cut[s - 1][j];
                bd.cut[s][j] = (k < M && prev == f) ? order[s - 1].axis[M - 1] : prev;
            }
            if (k < M && bd.cut[s][j] == f) {
                err = std::string("the ") + names[kind] + " method cannot start by transforming a cut axis";
                return false;
            }
            if (bd.q[j] > N[bd.cut[s][j]]) {
                err = std::string("the ") + names[kind] + " method cuts an axis of " +
                      std::to_string(N[bd.cut[s][j]]) + " points into " + std::to_string(bd.q[j]) + " blocks";
                return false;
            }
        }
    }
    return true;
}

void block_axis_grid(const BlockDecomp &bd, int M, int s, int64_t *q_axis, int64_t *ps_axis) {
    for (int a = 0; a < M; ++a) q_axis[a] = 1, ps_axis[a] = 0;
    int64_t ps = 1;
    for (int j = bd.k - 1; j >= 0; --j) {
        q_axis[bd.cut[s][j]] = bd.q[j];
        ps_axis[bd.cut[s][j]] = ps;
        ps *= bd.q[j];
    }
}

int64_t block_transition_amount(int M, const int64_t *N, int64_t P, const BlockDecomp &bd, int s) {
    int64_t qa[kMaxDims], pa[kMaxDims], qb[kMaxDims], pb[kMaxDims];
    block_axis_grid(bd, M, s, qa, pa);
    block_axis_grid(bd, M, s + 1, qb, pb);
    int64_t T = 1;
    for (int a = 0; a < M; ++a) T *= N[a];
    int64_t kept = 0;
    for (int64_t p = 0; p < P; ++p) {
        int64_t v = 1;
        for (int a = 0; a < M && v; ++a) {
            // block of process p along axis a in either step; [lo, hi) points
            const int64_t ba = qa[a] > 1 ? (p / pa[a]) % qa[a] : 0, bb = qb[a] > 1 ? (p / pb[a]) % qb[a] : 0;
            const int64_t lo = std::max(ba * N[a] / qa[a], bb * N[a] / qb[a]);
            const int64_t hi = std::min((ba + 1) * N[a] / qa[a], (bb + 1) * N[a] / qb[a]);
            v *= hi > lo ? hi - lo : 0;
        }
        kept += v;
    }
    return T - kept;
}

int64_t block_split_amount(int M, const int64_t *N, const BlockDecomp &bd, const std::vector<Layout> &order, int s) {
    int64_t q[kMaxDims], ps[kMaxDims];
    block_axis_grid(bd, M, s, q, ps);
    int64_t T = 1;
    for (int a = 0; a < M; ++a) T *= N[a];
    return T * (q[order[s].axis[M - 1]] - 1);
}

}  // namespace planner
}  // namespace mdfft
