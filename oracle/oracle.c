/*
 * oracle.c -- plain, slow FP64 CPU reference ("the oracle") for the
 * multi-dimensional FFT with row-wise adaptive decomposition and
 * transpose-order awareness (Duy and Ozaki, "A decomposition method with
 * minimum communication amount for parallelization of multi-dimensional
 * FFTs", arXiv:1302.6189).
 *
 * TEST INFRASTRUCTURE ONLY.  The CUDA library never includes, links or calls
 * this file, and this file uses nothing of the library.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Conventions: complex values are interleaved (re, im) doubles; every index
 * is int64; axis ids are 0 = a, 1 = b, ...; a "layout" is a permutation of
 * the axis ids listed from the slowest to the fastest axis of a row-major
 * array, and its last axis is the one transformed in that step (Fig. 4).
 *
 * Parts, each following the passage it cites:
 *   1. 1-D DFT, recursive mixed-radix Cooley-Tukey   (Sec. 2, the 1-D DFT equation)
 *   2. M-D DFT as M single-axis passes               (Sec. 2, the M-D DFT equation and
 *                                                     the "M single steps" remark)
 *   3. naive O(T^2) M-D DFT                          (Sec. 2, the M-D DFT equation)
 *   4. row-wise map X_1, f_MD, chunk bounds and
 *      coordinate recovery                           (Sec. 3.1 and Sec. 3.2)
 *   5. owners and communication amounts, brute force (Sec. 3.1, Figs. 2-3; Sec. 3.3)
 *   6. enumeration of transpose orders               (Sec. 3.2, the C_MD equation; Table 1)
 *   7. the parallel algorithm of Fig. 4 with explicit per-rank chunk buffers
 *   8. closed-form amounts of the comparison methods (Sec. 4, A_1D ... A_5D)
 *   9. the comparison methods as owners of every point (Sec. 4), brute force
 *
 * Parity status: every part is pinned by the tests against values that do
 * not come from this file (naive DFT, numpy.fft, closed-form spectra, the
 * paper's Table 1, its printed ratios and its worked 2-D-regime statement,
 * and the closed forms A_1D ... A_5D of Sec. 4 for part 9).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXDIM 16
#define ORC_TWO_PI 6.283185307179586476925286766559

typedef struct { double re, im; } cx;

static inline cx cx_mul(cx a, cx b) {
    cx r;
    r.re = a.re * b.re - a.im * b.im;
    r.im = a.re * b.im + a.im * b.re;
    return r;
}

static inline cx cx_add(cx a, cx b) {
    cx r;
    r.re = a.re + b.re;
    r.im = a.im + b.im;
    return r;
}

/* ------------------------------------------------------------------------ */
/* 1. 1-D DFT (Sec. 2): Xbar(k) = sum_j w_N^{jk} X(j), w_N = exp(-2 pi i/N),  */
/*    no normalisation.  sign = -1 gives that forward transform, +1 the      */
/*    unnormalised inverse.                                                   */
/* ------------------------------------------------------------------------ */

/* roots[q] = exp(sign * 2 pi i q / n) for q in [0, n). */
static cx *make_roots(int64_t n, int sign) {
    cx *t = (cx *)malloc((size_t)n * sizeof(cx));
    if (!t) return NULL;
    for (int64_t q = 0; q < n; ++q) {
        double a = ORC_TWO_PI * (double)q / (double)n;
        t[q].re = cos(a);
        t[q].im = (double)sign * sin(a);
    }
    return t;
}

static int64_t smallest_factor(int64_t n) {
    for (int64_t p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/*
 * out[0..n) = DFT_n of (in[0], in[s], in[2s], ...).  Decimation in time by
 * the smallest prime factor p of n, n = p * m:
 *   X[k + m t] = sum_{q<p} w_n^{q (k + m t)} Y_q[k],
 *   Y_q = DFT_m of the samples in[(q + p u) s], u < m.
 * roots holds the n_top-th roots of unity (n divides n_top), tmp >= p entries.
 */
static void fft_rec(const cx *in, int64_t s, cx *out, int64_t n, const cx *roots, int64_t n_top,
                    cx *tmp) {
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int64_t p = smallest_factor(n), m = n / p;
    for (int64_t q = 0; q < p; ++q) fft_rec(in + q * s, s * p, out + q * m, m, roots, n_top, tmp);
    int64_t step = n_top / n; /* w_n^e = roots[(e mod n) * step] */
    for (int64_t k = 0; k < m; ++k) {
        for (int64_t q = 0; q < p; ++q) tmp[q] = out[q * m + k];
        for (int64_t t = 0; t < p; ++t) {
            cx acc = {0.0, 0.0};
            for (int64_t q = 0; q < p; ++q) {
                int64_t e = (q * (k + m * t)) % n;
                acc = cx_add(acc, cx_mul(roots[e * step], tmp[q]));
            }
            out[k + m * t] = acc;
        }
    }
}

/* In-place 1-D transform of n interleaved complex values.  0 on success. */
int orc_fft1d(double *x, int64_t n, int sign) {
    if (n < 1 || (sign != -1 && sign != 1)) return -1;
    cx *roots = make_roots(n, sign);
    cx *in = (cx *)malloc((size_t)n * sizeof(cx));
    cx *tmp = (cx *)malloc((size_t)n * sizeof(cx));
    if (!roots || !in || !tmp) {
        free(roots), free(in), free(tmp);
        return -4;
    }
    memcpy(in, x, (size_t)n * sizeof(cx));
    fft_rec(in, 1, (cx *)x, n, roots, n, tmp);
    free(roots), free(in), free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 2. M-D DFT as M single-axis steps on the natural layout (Sec. 2).         */
/* ------------------------------------------------------------------------ */

typedef struct {
    cx *data;
    int64_t n, stride, line_lo, line_hi;
    const cx *roots;
} axis_job;

static void *axis_worker(void *arg) {
    axis_job *j = (axis_job *)arg;
    cx *line = (cx *)malloc((size_t)j->n * sizeof(cx));
    cx *res = (cx *)malloc((size_t)j->n * sizeof(cx));
    cx *tmp = (cx *)malloc((size_t)j->n * sizeof(cx));
    if (!line || !res || !tmp) {
        free(line), free(res), free(tmp);
        return (void *)1;
    }
    for (int64_t l = j->line_lo; l < j->line_hi; ++l) {
        /* line l: all coordinates but this axis; its elements are base + i * stride */
        int64_t base = (l / j->stride) * (j->n * j->stride) + (l % j->stride);
        for (int64_t i = 0; i < j->n; ++i) line[i] = j->data[base + i * j->stride];
        fft_rec(line, 1, res, j->n, j->roots, j->n, tmp);
        for (int64_t i = 0; i < j->n; ++i) j->data[base + i * j->stride] = res[i];
    }
    free(line), free(res), free(tmp);
    return NULL;
}

/* In-place transform of one axis of a natural row-major array. */
int orc_fft_axis(double *x, int M, const int64_t *N, int axis, int sign, int nthreads) {
    if (M < 1 || M > ORC_MAXDIM || axis < 0 || axis >= M || (sign != -1 && sign != 1)) return -1;
    int64_t T = 1, stride = 1;
    for (int r = 0; r < M; ++r) {
        if (N[r] < 1) return -1;
        T *= N[r];
    }
    for (int r = axis + 1; r < M; ++r) stride *= N[r];
    int64_t n = N[axis], lines = T / n;
    cx *roots = make_roots(n, sign);
    if (!roots) return -4;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > lines) nthreads = (int)lines;
    axis_job jobs[256];
    pthread_t th[256];
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].data = (cx *)x;
        jobs[t].n = n;
        jobs[t].stride = stride;
        jobs[t].line_lo = lines * t / nthreads;
        jobs[t].line_hi = lines * (t + 1) / nthreads;
        jobs[t].roots = roots;
    }
    if (nthreads == 1) {
        if (axis_worker(&jobs[0])) rc = -4;
    } else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, axis_worker, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) {
            void *ret = NULL;
            pthread_join(th[t], &ret);
            if (ret) rc = -4;
        }
    }
    free(roots);
    return rc;
}

/* In-place M-D transform: one axis after another, last axis first (Sec. 2). */
int orc_fftnd(double *x, int M, const int64_t *N, int sign, int nthreads) {
    for (int axis = M - 1; axis >= 0; --axis) {
        int rc = orc_fft_axis(x, M, N, axis, sign, nthreads);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 3. Naive M-D DFT, the nested sum of Sec. 2 evaluated point by point.      */
/* ------------------------------------------------------------------------ */

int orc_dft_naive(const double *in, double *out, int M, const int64_t *N, int sign) {
    if (M < 1 || M > ORC_MAXDIM || (sign != -1 && sign != 1)) return -1;
    int64_t T = 1;
    for (int r = 0; r < M; ++r) T *= N[r];
    const cx *X = (const cx *)in;
    cx *Y = (cx *)out;
    int64_t kc[ORC_MAXDIM], jc[ORC_MAXDIM];
    for (int64_t kk = 0; kk < T; ++kk) {
        int64_t rem = kk;
        for (int r = M - 1; r >= 0; --r) kc[r] = rem % N[r], rem /= N[r];
        cx acc = {0.0, 0.0};
        for (int64_t jj = 0; jj < T; ++jj) {
            int64_t rj = jj;
            for (int r = M - 1; r >= 0; --r) jc[r] = rj % N[r], rj /= N[r];
            /* phase = sum_r (j_r k_r mod N_r) / N_r, reduced to [0, 1) */
            double frac = 0.0;
            for (int r = 0; r < M; ++r) frac += (double)((jc[r] * kc[r]) % N[r]) / (double)N[r];
            frac -= floor(frac);
            double a = ORC_TWO_PI * frac;
            cx w = {cos(a), (double)sign * sin(a)};
            acc = cx_add(acc, cx_mul(w, X[jj]));
        }
        Y[kk] = acc;
    }
    return 0;
}

/* One output point of the M-D DFT, Xbar(k) = sum_j prod_r w_{N_r}^{j_r k_r} X(j),
 * with the phase of axis r read from a vector of N_r values exp(sign 2 pi i
 * (j k_r mod N_r) / N_r).  Used for sampled checks of grids too large for a
 * full reference transform. */
int orc_dft_point(const double *in, int M, const int64_t *N, const int64_t *k, int sign, double *out) {
    if (M < 1 || M > ORC_MAXDIM || (sign != -1 && sign != 1)) return -1;
    cx *ph[ORC_MAXDIM] = {0};
    int64_t T = 1;
    int rc = 0;
    for (int r = 0; r < M; ++r) {
        T *= N[r];
        ph[r] = (cx *)malloc((size_t)N[r] * sizeof(cx));
        if (!ph[r]) {
            rc = -4;
            goto done;
        }
        for (int64_t j = 0; j < N[r]; ++j) {
            double a = ORC_TWO_PI * (double)((j * k[r]) % N[r]) / (double)N[r];
            ph[r][j].re = cos(a);
            ph[r][j].im = (double)sign * sin(a);
        }
    }
    {
        const cx *X = (const cx *)in;
        int64_t jc[ORC_MAXDIM] = {0};
        cx acc = {0.0, 0.0};
        for (int64_t jj = 0; jj < T; ++jj) {
            cx w = ph[0][jc[0]];
            for (int r = 1; r < M; ++r) w = cx_mul(w, ph[r][jc[r]]);
            acc = cx_add(acc, cx_mul(w, X[jj]));
            for (int r = M - 1; r >= 0; --r) { /* next j in row-major order */
                if (++jc[r] < N[r]) break;
                jc[r] = 0;
            }
        }
        out[0] = acc.re;
        out[1] = acc.im;
    }
done:
    for (int r = 0; r < M; ++r) free(ph[r]);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 4. Row-wise decomposition (Sec. 3.1, Sec. 3.2).                            */
/* ------------------------------------------------------------------------ */

typedef unsigned __int128 u128;

/* Regime: the number k of leading dims the chunks are cut on, i.e. the
 * smallest k with Np <= N_1 ... N_k (the case split of f_MD).  -1 if Np is
 * outside [1, N_1 ... N_M]. */
int orc_regime(int M, const int64_t *N, int64_t P) {
    if (M < 1 || M > ORC_MAXDIM || P < 1) return -1;
    u128 lead = 1;
    for (int r = 0; r < M; ++r) {
        if (N[r] < 1) return -1;
        lead *= (u128)N[r];
        if ((u128)P <= lead) return r + 1;
    }
    return -1;
}

/* f_MD(N_1..N_M, Np, myid) of Sec. 3.2: with k the regime,
 *   floor((N_1 ... N_k) * myid / Np) * (N_{k+1} ... N_M).
 * myid may be Np (gives T, the end bound).  -1 on bad arguments. */
int64_t orc_fmd(int M, const int64_t *N, int64_t P, int64_t myid) {
    int k = orc_regime(M, N, P);
    if (k < 0 || myid < 0 || myid > P) return -1;
    u128 lead = 1, rest = 1;
    for (int r = 0; r < k; ++r) lead *= (u128)N[r];
    for (int r = k; r < M; ++r) rest *= (u128)N[r];
    u128 v = (lead * (u128)myid / (u128)P) * rest;
    return (int64_t)v;
}

/* Coordinate recovery of Sec. 3.2: x_1 = floor(x / (N_2...N_M)), then each
 * following coordinate from what is left after subtracting the earlier ones. */
void orc_coords(int M, const int64_t *N, int64_t x, int64_t *c) {
    int64_t left = x;
    for (int r = 0; r < M; ++r) {
        int64_t w = 1;
        for (int i = r + 1; i < M; ++i) w *= N[i];
        c[r] = left / w;
        left -= c[r] * w;
    }
}

/* Row-wise linear index X_1 of Sec. 3.2. */
int64_t orc_linear(int M, const int64_t *N, const int64_t *c) {
    int64_t X = 0;
    for (int r = 0; r < M; ++r) {
        int64_t w = 1;
        for (int i = r + 1; i < M; ++i) w *= N[i];
        X += c[r] * w;
    }
    return X;
}

/* Chunk of rank myid: x^s = f(myid), x^e = f(myid+1) - 1 and their
 * coordinates (Sec. 3.1 and 3.2).  0 on success. */
int orc_chunk(int M, const int64_t *N, int64_t P, int64_t myid, int64_t *xs, int64_t *xe,
              int64_t *cs, int64_t *ce) {
    if (myid < 0 || myid >= P) return -1;
    int64_t a = orc_fmd(M, N, P, myid), b = orc_fmd(M, N, P, myid + 1);
    if (a < 0 || b < 0) return -1;
    *xs = a;
    *xe = b - 1;
    if (cs) orc_coords(M, N, a, cs);
    if (ce) orc_coords(M, N, b - 1, ce);
    return 0;
}

static int layout_ok(int M, const int *L) {
    int seen[ORC_MAXDIM] = {0};
    for (int i = 0; i < M; ++i) {
        if (L[i] < 0 || L[i] >= M || seen[L[i]]) return 0;
        seen[L[i]] = 1;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* 5. Owners and communication amounts by brute force.                       */
/*    A layout's chunks are the f_MD chunks of its row-major order, i.e. of  */
/*    the dims permuted into that layout (Sec. 3.1: other layouts follow    */
/*    by the same construction).  The amount of one transpose is the number  */
/*    of points whose owner changes; the rest is reused in place (Sec. 1,    */
/*    Sec. 3.1 on Fig. 2).                                                   */
/* ------------------------------------------------------------------------ */

/* owner[natural linear index] = rank holding that point in layout L. */
int orc_owner_array(int M, const int64_t *N, int64_t P, const int *L, int32_t *owner) {
    if (M < 1 || M > ORC_MAXDIM || !layout_ok(M, L)) return -1;
    int64_t Nl[ORC_MAXDIM], cl[ORC_MAXDIM], c[ORC_MAXDIM];
    for (int i = 0; i < M; ++i) Nl[i] = N[L[i]];
    if (orc_regime(M, Nl, P) < 0) return -3;
    for (int64_t p = 0; p < P; ++p) {
        int64_t xs = orc_fmd(M, Nl, P, p), xe = orc_fmd(M, Nl, P, p + 1) - 1;
        for (int64_t X = xs; X <= xe; ++X) {
            orc_coords(M, Nl, X, cl);
            for (int i = 0; i < M; ++i) c[L[i]] = cl[i];
            owner[orc_linear(M, N, c)] = (int32_t)p;
        }
    }
    return 0;
}

static int64_t count_differ(const int32_t *a, const int32_t *b, int64_t T) {
    int64_t v = 0;
    for (int64_t i = 0; i < T; ++i) v += (a[i] != b[i]);
    return v;
}

/* Split-line amount of layout L: lines along L's last axis cut between k
 * owners need N_axis * (k - 1) points exchanged (0 when no line is cut). */
int64_t orc_split_line(int M, const int64_t *N, int64_t P, const int *L) {
    int64_t Nl[ORC_MAXDIM], T = 1;
    for (int i = 0; i < M; ++i) Nl[i] = N[L[i]], T *= Nl[i];
    if (orc_regime(M, Nl, P) < 0) return -1;
    int64_t nf = Nl[M - 1], total = 0;
    int32_t *own = (int32_t *)malloc((size_t)T * sizeof(int32_t)); /* indexed by L-linear index */
    if (!own) return -4;
    for (int64_t p = 0; p < P; ++p)
        for (int64_t X = orc_fmd(M, Nl, P, p); X < orc_fmd(M, Nl, P, p + 1); ++X) own[X] = (int32_t)p;
    for (int64_t l = 0; l < T / nf; ++l) {
        int64_t owners = 1;
        for (int64_t i = 1; i < nf; ++i) owners += (own[l * nf + i] != own[l * nf + i - 1]);
        total += nf * (owners - 1);
    }
    free(own);
    return total;
}

/* Amounts of an order (M layouts x M axis ids): per_transition[s] for
 * s = 0..M-2, final_to_natural (last layout back to natural order, done but
 * not counted), split_line[s] for s = 0..M-1. */
int orc_comm_volume(int M, const int64_t *N, int64_t P, const int *order, int64_t *per_transition,
                    int64_t *final_to_natural, int64_t *split_line) {
    if (M < 1 || M > ORC_MAXDIM) return -1;
    int64_t T = 1;
    for (int r = 0; r < M; ++r) T *= N[r];
    int32_t *a = (int32_t *)malloc((size_t)T * sizeof(int32_t));
    int32_t *b = (int32_t *)malloc((size_t)T * sizeof(int32_t));
    int natural[ORC_MAXDIM];
    for (int i = 0; i < M; ++i) natural[i] = i;
    int rc = 0;
    if (!a || !b) {
        rc = -4;
        goto done;
    }
    if ((rc = orc_owner_array(M, N, P, order, a))) goto done;
    for (int s = 0; s + 1 < M; ++s) {
        if ((rc = orc_owner_array(M, N, P, order + (s + 1) * M, b))) goto done;
        per_transition[s] = count_differ(a, b, T);
        int32_t *t = a;
        a = b, b = t;
    }
    if ((rc = orc_owner_array(M, N, P, natural, b))) goto done;
    *final_to_natural = count_differ(a, b, T);
    for (int s = 0; s < M; ++s) split_line[s] = orc_split_line(M, N, P, order + s * M);
done:
    free(a), free(b);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 6. Transpose orders (Sec. 3.2, the C_MD equation; Table 1).               */
/*    The first layout is the natural one; every later layout is any         */
/*    permutation whose last axis was not the last axis of an earlier one.   */
/* ------------------------------------------------------------------------ */

static int64_t factorial(int n) {
    int64_t f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* All permutations of 0..M-1 in lexicographic order, M! rows of M ints. */
static int *all_perms(int M, int64_t *count) {
    int64_t F = factorial(M);
    int *out = (int *)malloc((size_t)(F * M) * sizeof(int));
    if (!out) return NULL;
    int cur[ORC_MAXDIM];
    for (int i = 0; i < M; ++i) cur[i] = i;
    for (int64_t f = 0; f < F; ++f) {
        memcpy(out + f * M, cur, (size_t)M * sizeof(int));
        /* next permutation */
        int i = M - 2;
        while (i >= 0 && cur[i] > cur[i + 1]) --i;
        if (i < 0) break;
        int j = M - 1;
        while (cur[j] < cur[i]) --j;
        int t = cur[i];
        cur[i] = cur[j], cur[j] = t;
        for (int l = i + 1, r = M - 1; l < r; ++l, --r) t = cur[l], cur[l] = cur[r], cur[r] = t;
    }
    *count = F;
    return out;
}

typedef struct {
    int M;
    const int *perms;
    int64_t nperm;
    int seq[ORC_MAXDIM];   /* perm index per layer */
    int64_t n_seen;
    int *out;              /* optional: sequences as M*M ints */
    int64_t cap;
    /* search mode */
    const int64_t *pair;   /* nperm x nperm amounts */
    int64_t best, worst, n_best, n_worst;
    int best_seq[ORC_MAXDIM], worst_seq[ORC_MAXDIM];
    int *best_list;
    int64_t best_list_cap, best_list_n;
} enum_state;

static void emit(enum_state *st) {
    int M = st->M;
    if (st->out && st->n_seen < st->cap)
        for (int s = 0; s < M; ++s)
            memcpy(st->out + (st->n_seen * M + s) * M, st->perms + (int64_t)st->seq[s] * M,
                   (size_t)M * sizeof(int));
    if (st->pair) {
        int64_t tot = 0;
        for (int s = 0; s + 1 < M; ++s) tot += st->pair[(int64_t)st->seq[s] * st->nperm + st->seq[s + 1]];
        if (st->n_seen == 0 || tot < st->best) {
            st->best = tot, st->n_best = 0, st->best_list_n = 0;
            memcpy(st->best_seq, st->seq, sizeof(st->seq));
        }
        if (tot == st->best) {
            if (st->best_list && st->best_list_n < st->best_list_cap) {
                for (int s = 0; s < M; ++s)
                    memcpy(st->best_list + (st->best_list_n * M + s) * M,
                           st->perms + (int64_t)st->seq[s] * M, (size_t)M * sizeof(int));
                st->best_list_n++;
            }
            st->n_best++;
        }
        if (st->n_seen == 0 || tot > st->worst) {
            st->worst = tot, st->n_worst = 0;
            memcpy(st->worst_seq, st->seq, sizeof(st->seq));
        }
        if (tot == st->worst) st->n_worst++;
    }
    st->n_seen++;
}

static void enum_rec(enum_state *st, int layer, unsigned used_last) {
    int M = st->M;
    if (layer == M) {
        emit(st);
        return;
    }
    for (int64_t f = 0; f < st->nperm; ++f) {
        int last = st->perms[f * M + M - 1];
        if (used_last & (1u << last)) continue;
        st->seq[layer] = (int)f;
        enum_rec(st, layer + 1, used_last | (1u << last));
    }
}

/* Number of transpose orders, by enumeration. */
int64_t orc_count_orders(int M) {
    if (M < 1 || M > 6) return -1;
    enum_state st;
    memset(&st, 0, sizeof(st));
    st.M = M;
    int *perms = all_perms(M, &st.nperm);
    if (!perms) return -4;
    st.perms = perms;
    st.seq[0] = 0; /* the natural layout is the lexicographically first permutation */
    enum_rec(&st, 1, 1u << (M - 1));
    free(perms);
    return st.n_seen;
}

/* Writes up to cap orders (M*M ints each) in lexicographic order; returns the count. */
int64_t orc_enumerate_orders(int M, int *out, int64_t cap) {
    if (M < 1 || M > 6) return -1;
    enum_state st;
    memset(&st, 0, sizeof(st));
    st.M = M;
    int *perms = all_perms(M, &st.nperm);
    if (!perms) return -4;
    st.perms = perms;
    st.out = out;
    st.cap = cap;
    st.seq[0] = 0;
    enum_rec(&st, 1, 1u << (M - 1));
    free(perms);
    return st.n_seen;
}

/* Exhaustive search over every order, with the amount of every pair of
 * layouts taken from brute-force owner arrays.  Outputs the best and worst
 * totals (sum of per-transition amounts), how many orders reach each, the
 * lexicographically first best and worst orders, and up to best_cap best
 * orders in lexicographic order. */
int orc_order_search(int M, const int64_t *N, int64_t P, int64_t *best, int64_t *worst,
                     int64_t *n_best, int64_t *n_worst, int *best_order, int *worst_order,
                     int *best_list, int64_t best_cap, int64_t *best_list_n) {
    if (M < 2 || M > 6) return -1;
    int64_t T = 1;
    for (int r = 0; r < M; ++r) T *= N[r];
    enum_state st;
    memset(&st, 0, sizeof(st));
    st.M = M;
    int *perms = all_perms(M, &st.nperm);
    int64_t F = st.nperm;
    int32_t *own = (int32_t *)malloc((size_t)(F * T) * sizeof(int32_t));
    int64_t *pair = (int64_t *)malloc((size_t)(F * F) * sizeof(int64_t));
    int rc = 0;
    if (!perms || !own || !pair) {
        rc = -4;
        goto done;
    }
    for (int64_t f = 0; f < F; ++f)
        if ((rc = orc_owner_array(M, N, P, perms + f * M, own + f * T))) goto done;
    for (int64_t f = 0; f < F; ++f)
        for (int64_t g = 0; g < F; ++g) pair[f * F + g] = count_differ(own + f * T, own + g * T, T);
    st.perms = perms;
    st.pair = pair;
    st.best_list = best_list;
    st.best_list_cap = best_cap;
    st.seq[0] = 0;
    enum_rec(&st, 1, 1u << (M - 1));
    *best = st.best, *worst = st.worst, *n_best = st.n_best, *n_worst = st.n_worst;
    if (best_list_n) *best_list_n = st.best_list_n;
    for (int s = 0; s < M; ++s) {
        memcpy(best_order + s * M, perms + (int64_t)st.best_seq[s] * M, (size_t)M * sizeof(int));
        memcpy(worst_order + s * M, perms + (int64_t)st.worst_seq[s] * M, (size_t)M * sizeof(int));
    }
done:
    free(perms), free(own), free(pair);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 7. The parallel M-D FFT of Fig. 4 with explicit per-rank chunks.          */
/*    Step s transforms the lines along the last axis of layout s inside     */
/*    each rank's chunk; a line cut between ranks is gathered, transformed  */
/*    and handed back (counted in split[s]).  The transpose then sends every */
/*    point to the rank that owns it in the next layout (counted in          */
/*    moved[s] when the rank changes).  After step M the data go back to the */
/*    natural order (moved[M-1]).                                            */
/* ------------------------------------------------------------------------ */

static int64_t find_owner(const int64_t *bnd, int64_t P, int64_t X) {
    int64_t lo = 0, hi = P - 1; /* largest p with bnd[p] <= X */
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (bnd[mid] <= X) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

int orc_fft_fig4(const double *in, double *out, int M, const int64_t *N, int64_t P, const int *order,
                 int sign, int64_t *moved, int64_t *split) {
    if (M < 1 || M > ORC_MAXDIM || P < 1 || (sign != -1 && sign != 1)) return -1;
    int natural[ORC_MAXDIM];
    for (int i = 0; i < M; ++i) natural[i] = i;
    if (!layout_ok(M, order)) return -2;
    for (int i = 0; i < M; ++i)
        if (order[i] != i) return -2;
    for (int s = 1; s < M; ++s) {
        if (!layout_ok(M, order + s * M)) return -2;
        for (int q = 0; q < s; ++q)
            if (order[s * M + M - 1] == order[q * M + M - 1]) return -2;
    }
    int64_t T = 1;
    for (int r = 0; r < M; ++r) T *= N[r];
    if (orc_regime(M, N, P) < 0) return -3;

    int64_t *bnd = (int64_t *)malloc((size_t)(P + 1) * sizeof(int64_t));
    int64_t *nbnd = (int64_t *)malloc((size_t)(P + 1) * sizeof(int64_t));
    cx **buf = (cx **)calloc((size_t)P, sizeof(cx *));
    cx **nbuf = (cx **)calloc((size_t)P, sizeof(cx *));
    int rc = 0;
    if (!bnd || !nbnd || !buf || !nbuf) {
        rc = -4;
        goto done;
    }
    /* initial distribution: chunks of the natural layout */
    for (int64_t p = 0; p <= P; ++p) bnd[p] = orc_fmd(M, N, P, p);
    for (int64_t p = 0; p < P; ++p) {
        buf[p] = (cx *)malloc((size_t)(bnd[p + 1] - bnd[p]) * sizeof(cx));
        if (!buf[p]) {
            rc = -4;
            goto done;
        }
        memcpy(buf[p], (const cx *)in + bnd[p], (size_t)(bnd[p + 1] - bnd[p]) * sizeof(cx));
    }
    for (int s = 0; s < M; ++s) {
        const int *L = order + s * M;
        const int *Lnext = (s + 1 < M) ? order + (s + 1) * M : natural;
        int64_t Nl[ORC_MAXDIM], Nn[ORC_MAXDIM], cl[ORC_MAXDIM], c[ORC_MAXDIM], cn[ORC_MAXDIM];
        for (int i = 0; i < M; ++i) Nl[i] = N[L[i]], Nn[i] = N[Lnext[i]];
        int64_t nf = Nl[M - 1];

        /* Step s+1: 1-D transforms along the last axis of L. */
        cx *line = (cx *)malloc((size_t)nf * sizeof(cx));
        cx *res = (cx *)malloc((size_t)nf * sizeof(cx));
        cx *tmp = (cx *)malloc((size_t)nf * sizeof(cx));
        cx *roots = make_roots(nf, sign);
        if (!line || !res || !tmp || !roots) {
            free(line), free(res), free(tmp), free(roots);
            rc = -4;
            goto done;
        }
        split[s] = 0;
        for (int64_t l = 0; l < T / nf; ++l) {
            int64_t first = l * nf;
            int64_t owners = 0, prev = -1;
            for (int64_t i = 0; i < nf; ++i) { /* gather the line from whoever holds it */
                int64_t p = find_owner(bnd, P, first + i);
                if (p != prev) owners++, prev = p;
                line[i] = buf[p][first + i - bnd[p]];
            }
            split[s] += nf * (owners - 1);
            fft_rec(line, 1, res, nf, roots, nf, tmp);
            for (int64_t i = 0; i < nf; ++i) {
                int64_t p = find_owner(bnd, P, first + i);
                buf[p][first + i - bnd[p]] = res[i];
            }
        }
        free(line), free(res), free(tmp), free(roots);

        /* Transpose: adaptive decomposition of the next layout. */
        for (int64_t p = 0; p <= P; ++p) nbnd[p] = orc_fmd(M, Nn, P, p);
        for (int64_t q = 0; q < P; ++q) {
            nbuf[q] = (cx *)malloc((size_t)(nbnd[q + 1] - nbnd[q]) * sizeof(cx));
            if (!nbuf[q]) {
                rc = -4;
                goto done;
            }
        }
        moved[s] = 0;
        for (int64_t p = 0; p < P; ++p) {
            for (int64_t X = bnd[p]; X < bnd[p + 1]; ++X) {
                orc_coords(M, Nl, X, cl);
                for (int i = 0; i < M; ++i) c[L[i]] = cl[i];
                for (int i = 0; i < M; ++i) cn[i] = c[Lnext[i]];
                int64_t Xn = orc_linear(M, Nn, cn);
                int64_t q = find_owner(nbnd, P, Xn);
                nbuf[q][Xn - nbnd[q]] = buf[p][X - bnd[p]];
                moved[s] += (q != p);
            }
        }
        for (int64_t p = 0; p < P; ++p) {
            free(buf[p]);
            buf[p] = nbuf[p];
            nbuf[p] = NULL;
        }
        memcpy(bnd, nbnd, (size_t)(P + 1) * sizeof(int64_t));
    }
    /* natural order: chunk p of the natural layout holds [bnd[p], bnd[p+1]) */
    for (int64_t p = 0; p < P; ++p)
        memcpy((cx *)out + bnd[p], buf[p], (size_t)(bnd[p + 1] - bnd[p]) * sizeof(cx));
done:
    if (buf)
        for (int64_t p = 0; p < P; ++p) free(buf[p]);
    if (nbuf)
        for (int64_t p = 0; p < P; ++p) free(nbuf[p]);
    free(buf), free(nbuf), free(bnd), free(nbnd);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 8. Amounts of the comparison methods for an N^M grid (Sec. 4).            */
/* ------------------------------------------------------------------------ */

/* 1-D (slab) method: N^3 - N^3 / Np. */
double orc_amount_slab(double N, double P) { return N * N * N - N * N * N / P; }

/* 2-D (pencil) method: 2 N^3 - 2 Np (N^2 / Np)^(3/2). */
double orc_amount_pencil(double N, double P) { return 2.0 * N * N * N - 2.0 * P * pow(N * N / P, 1.5); }

/* M-D (volumetric) method for M = 3, 4, 5: M N^M (N / (N^M / Np)^(1/M) - 1). */
double orc_amount_volumetric(int M, double N, double P) {
    double T = pow(N, (double)M);
    return (double)M * T * (N / pow(T / P, 1.0 / (double)M) - 1.0);
}

/* ------------------------------------------------------------------------ */
/* 9. The comparison methods of Sec. 4 as explicit owners of every point.    */
/*    The 1-D method gives each process whole planes (one axis cut), the     */
/*    2-D method whole lines (two axes cut), the M-D methods blocks (every   */
/*    axis cut).  A step transforms along one axis.  With fewer than M cut   */
/*    axes the transformed axis is never cut: when the next step's axis is   */
/*    cut, its cut moves to the axis just transformed (the transposes of the */
/*    1-D and 2-D methods).  With M cut axes nothing moves and every line is */
/*    shared by the owners of its blocks, each of which gathers the whole    */
/*    line (the model behind A_3D: T (q - 1) points per step).               */
/*    Readings of what Sec. 4 leaves open:                                    */
/*    - the cut axes of the first step are the k slowest axes a, b, ...      */
/*      (the first step transforms the fastest axis);                         */
/*    - Np is split over the k cuts as evenly as possible: its prime factors,*/
/*      largest first, each go to the cut with the smallest product so far  */
/*      (the first such cut on ties); pid = sum_j digit_j prod_{i>j} q_i;    */
/*    - a cut of n points into q blocks gives block j the points             */
/*      [floor(j n / q), floor((j + 1) n / q)), the floor rule of f_MD's 1-D */
/*      case; q <= n, so no block is empty;                                   */
/*    - the output stays in the last step's decomposition.                    */
/* ------------------------------------------------------------------------ */

static void even_split(int64_t P, int k, int64_t *q) {
    int64_t f[64];
    int nf = 0;
    int64_t n = P;
    for (int64_t d = 2; d * d <= n; ++d)
        while (n % d == 0) f[nf++] = d, n /= d;
    if (n > 1) f[nf++] = n;
    for (int j = 0; j < k; ++j) q[j] = 1;
    for (int i = nf - 1; i >= 0; --i) {
        int jm = 0;
        for (int j = 1; j < k; ++j)
            if (q[j] < q[jm]) jm = j;
        q[jm] *= f[i];
    }
}

/* kind: 1 = 1-D (slab), 2 = 2-D (pencil), 3 = M-D (volumetric) method.
 * fft_axes[s]: the axis transformed in step s (a permutation of 0..M-1).
 * Writes per_transition[s] (s < M-1): points whose owner differs between
 * steps s and s+1; split[s]: sum over the lines of step s of
 * N_axis (owners on the line - 1); q_axis[s*M + axis]: processes along that
 * axis in step s (1: not cut).  Every count is by looking at every point.
 * Returns 0, -1 on bad arguments, -2 if a cut has more blocks than points,
 * -3 on allocation failure. */
int orc_block_volume(int M, const int64_t *N, int64_t P, int kind, const int *fft_axes, int64_t *per_transition,
                     int64_t *split, int64_t *q_axis) {
    if (M < 1 || M > ORC_MAXDIM || kind < 1 || kind > 3 || P < 1) return -1;
    int used[ORC_MAXDIM] = {0};
    for (int s = 0; s < M; ++s) {
        if (fft_axes[s] < 0 || fft_axes[s] >= M || used[fft_axes[s]]) return -1;
        used[fft_axes[s]] = 1;
    }
    const int k = kind == 3 ? M : kind;
    if (k > M) return -1;
    int64_t q[ORC_MAXDIM];
    even_split(P, k, q);
    int cut[ORC_MAXDIM][ORC_MAXDIM]; /* [step][j]: the axis of cut j */
    for (int j = 0; j < k; ++j) cut[0][j] = j;
    for (int s = 0; s < M; ++s) {
        if (s > 0)
            for (int j = 0; j < k; ++j) {
                cut[s][j] = cut[s - 1][j];
                if (k < M && cut[s][j] == fft_axes[s]) cut[s][j] = fft_axes[s - 1];
            }
        for (int a = 0; a < M; ++a) q_axis[s * M + a] = 1;
        for (int j = 0; j < k; ++j) {
            if (k < M && cut[s][j] == fft_axes[s]) return -1;
            if (q[j] > N[cut[s][j]]) return -2;
            q_axis[s * M + cut[s][j]] = q[j];
        }
    }
    int64_t T = 1;
    for (int i = 0; i < M; ++i) T *= N[i];
    int64_t *own = (int64_t *)malloc((size_t)T * sizeof(int64_t) * 2);
    int64_t *seen = (int64_t *)malloc((size_t)P * sizeof(int64_t));
    if (!own || !seen) {
        free(own), free(seen);
        return -3;
    }
    int64_t c[ORC_MAXDIM];
    for (int s = 0; s < M; ++s) {
        int64_t *cur = own + (s % 2) * T, *prev = own + ((s + 1) % 2) * T;
        for (int64_t X = 0; X < T; ++X) {
            orc_coords(M, N, X, c);
            int64_t pid = 0;
            for (int j = 0; j < k; ++j) {
                const int64_t n = N[cut[s][j]], x = c[cut[s][j]];
                int64_t b = 0; /* the block of x: the largest b with floor(b n / q) <= x */
                while (b + 1 < q[j] && ((b + 1) * n) / q[j] <= x) ++b;
                pid = pid * q[j] + b;
            }
            cur[X] = pid;
        }
        if (s > 0) {
            int64_t m = 0;
            for (int64_t X = 0; X < T; ++X) m += cur[X] != prev[X];
            per_transition[s - 1] = m;
        }
        /* owners on every line along the step's axis */
        const int f = fft_axes[s];
        int64_t stride = 1;
        for (int i = M - 1; i > f; --i) stride *= N[i];
        for (int64_t p = 0; p < P; ++p) seen[p] = -1;
        split[s] = 0;
        for (int64_t X = 0; X < T; ++X) {
            orc_coords(M, N, X, c);
            if (c[f] != 0) continue; /* X is the first point of its line */
            int64_t owners = 0;
            for (int64_t t = 0; t < N[f]; ++t) {
                const int64_t pid = cur[X + t * stride];
                if (seen[pid] != X) seen[pid] = X, ++owners;
            }
            split[s] += N[f] * (owners - 1);
        }
    }
    free(own), free(seen);
    return 0;
}
