/*
 * mdfft.h -- C ABI of libmdfft: multi-dimensional complex FFTs on one GPU
 * (sm_103a), computed the way of Duy and Ozaki's row-wise adaptive
 * decomposition with transpose-order awareness (arXiv:1302.6189).
 *
 * The problem statement follows Fig. 4 of the paper: input X(N_1..N_M), a
 * number of processes Np and a transpose order; output Xbar(N_1..N_M), the
 * unnormalised M-D DFT of Sec. 2 (forward sign exp(-2 pi i / N)).  On one
 * GPU the Np "processes" are virtual partitions of the row-wise flattened
 * array: they decide the communication amounts reported by
 * mdfft_comm_volume() and counted on the device by mdfft_exec_counted(),
 * not the result, which is the same for every Np and every order.
 *
 * Conventions for every entry point:
 *  - Arrays are dense row-major complex arrays in device memory; complex64 is
 *    (float re, float im), complex128 is (double re, double im).  The natural
 *    layout has axis a slowest and the last axis fastest.
 *  - An order is M layouts x M axis ids (0 = a, 1 = b, ...), each layout
 *    listed from the slowest to the fastest axis.  Layout 0 must be the
 *    natural 0, 1, ..., M-1, and the last entries of the M layouts must be a
 *    permutation of 0..M-1 (each step transforms a new axis; Sec. 3.2, the
 *    C_MD count).  Step s transforms the last axis of layout s and writes the
 *    result in layout s+1 (the "transpose" of Fig. 4); the last step writes
 *    the natural layout (or keeps layout M, see MDFFT_PLAN_OUT_LAST_LAYOUT).
 *  - Every call returns an mdfft_status; nothing throws across the ABI.  On
 *    failure mdfft_last_error() returns a message for the calling thread.
 *  - Execution is asynchronous on the caller's CUDA stream.  Device memory
 *    passed in stays owned by the caller; the plan owns its own device
 *    memory (twiddles, workspace) and frees it in mdfft_destroy().
 *  - A plan may be used from one host thread at a time.  Its executions
 *    share the plan's workspace, so executions of one plan on different
 *    streams must be ordered by the caller (events); on one stream they are.
 */
#ifndef MDFFT_H
#define MDFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MDFFT_MAX_DIMS 8

/* Same type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st *mdfft_stream_t;

typedef struct mdfft_plan_s *mdfft_plan_t;

typedef enum {
    MDFFT_OK = 0,
    MDFFT_E_ARG = -1,         /* bad pointer, size or flag */
    MDFFT_E_ORDER = -2,       /* order violates the layout rules above */
    MDFFT_E_RANGE = -3,       /* Np < 1 or Np > N_1 ... N_M (f_MD undefined) */
    MDFFT_E_NOMEM = -4,       /* host or device allocation failed */
    MDFFT_E_CUDA = -5,        /* a CUDA runtime call failed */
    MDFFT_E_TIMEOUT = -6,     /* a bounded device wait gave up */
    MDFFT_E_UNSUPPORTED = -7  /* size, dtype or M not built into this library */
} mdfft_status;

typedef enum {
    MDFFT_C64 = 0,         /* complex64, FP32 arithmetic */
    MDFFT_C128 = 1,        /* complex128, FP64 arithmetic */
    MDFFT_C64_TC_FP16 = 2, /* complex64 in/out; radix-16 stages as tcgen05 GEMMs, split hi/lo FP16, FP32
                              accumulators in TMEM (persistent kernel: arrays 16-byte aligned) */
    MDFFT_C64_TC_BF16 = 3  /* as above with BF16 hi/lo operands */
} mdfft_dtype;

/* mdfft_plan flags */
#define MDFFT_PLAN_HOST_ONLY 0x1u /* planner only: no device memory; exec refused */
#define MDFFT_PLAN_INPLACE 0x2u   /* allow in_dev == out_dev (one more workspace) */
#define MDFFT_PLAN_PERSISTENT 0x4u /* complex64: use the persistent bulk-copy pipelined pass kernel
                                      wherever one is built (even lengths <= 512); arrays must then be
                                      16-byte aligned */
/*
 * Ownership model of the plan's counted amounts (mdfft_comm_volume,
 * mdfft_exec_counted).  Default: the row-wise f_MD chunks of Sec. 3.  At most
 * one of the following selects a comparison method of Sec. 4 instead, run
 * through the same passes and order (step s transforms the last axis of
 * layout s): the 1-D method (whole planes: one axis cut), the 2-D method
 * (whole lines: two axes cut, M >= 3) or the volumetric M-D method (blocks:
 * every axis cut, each line gathered by each of its owners).  With fewer
 * than M cut axes, the cut of the axis about to be transformed moves to the
 * axis just transformed; the first step cuts the slowest axes; P is split
 * over the cuts as evenly as possible (prime factors, largest first, each to
 * the cut with the smallest product); a cut of n points into q blocks needs
 * q <= n (else E_RANGE).  The output stays in the last step's decomposition.
 */
/*
 * Output layout.  MDFFT_PLAN_OUT_NATURAL (the default): the spectrum in
 * natural row-major order (k_1 .. k_M), the last pass's store being the final
 * transpose of Fig. 4.  MDFFT_PLAN_OUT_LAST_LAYOUT: the spectrum stays in the
 * plan's last layout L_M (row-major with the axes in L_M's order, e.g. dims
 * (N_b, N_c, N_a) for a last layout "bca"); the last pass then stores whole
 * lines without transposing, and final_to_natural is 0.  Applies to both
 * directions (the input is always natural).
 */
#define MDFFT_PLAN_OUT_NATURAL 0x0u
#define MDFFT_PLAN_OUT_LAST_LAYOUT 0x80u
#define MDFFT_PLAN_DECOMP_SLAB 0x10u
#define MDFFT_PLAN_DECOMP_PENCIL 0x20u
#define MDFFT_PLAN_DECOMP_VOLUMETRIC 0x40u
/* Lets mdfft_plan_autotune also choose among radix splits of a line length
 * (radix_plan_alt, e.g. 8x8x4 for 256): the spectrum then changes in its
 * rounding only.  Without it autotuning never changes a result bit. */
#define MDFFT_PLAN_TUNE_RADIX 0x100u

/*
 * mdfft_plan -- build a plan for the M-D FFT of dims N[0..M) with Np = P
 * virtual processes and a transpose order.
 *   out    receives the plan (owned by the caller, free with mdfft_destroy).
 *   M      number of dimensions, 2..MDFFT_MAX_DIMS.
 *   N      the M dims, natural order; each dim must be a supported line
 *          length (products of 2, 3, 5 up to 1024 that the library was built
 *          for) unless MDFFT_PLAN_HOST_ONLY is set (then any dim >= 1).
 *   P      number of virtual processes, 1 <= P <= N_1 ... N_M (f_MD, Sec. 3.2).
 *   order  M*M axis ids as described above, or NULL for the order with the
 *          smallest total communication amount (mdfft_order_search: M <= 5,
 *          and M = 6 where that search is affordable) or else the
 *          balanced-split heuristic's order (mdfft_order_heuristic).
 *   dt     an mdfft_dtype.
 *   flags  MDFFT_PLAN_* bits.
 * Twiddles are made on the device in FP64 (sincospi) and rounded to the
 * pass precision.  Errors: E_ARG, E_ORDER, E_RANGE, E_UNSUPPORTED, E_NOMEM,
 * E_CUDA.
 */
mdfft_status mdfft_plan(mdfft_plan_t *out, int M, const int64_t N[], int64_t P, const int *order,
                        mdfft_dtype dt, unsigned flags);

/*
 * mdfft_plan_batched -- as mdfft_plan for `batch` independent transforms of
 * the same dims per execution (batch >= 1; mdfft_plan is batch = 1).  The
 * arrays of mdfft_exec / mdfft_exec_counted / mdfft_exec_host then hold
 * batch * N_1 ... N_M elements, transform v at element offset v * T, and the
 * plan's workspace is that size too.  Each pass is one launch over the tiles
 * of every transform of the batch (the batch is the outermost tile axis), so
 * the partly filled last wave of CTAs is paid once per pass, not once per
 * transform.  Counted executions add the amounts of all transforms; the
 * amounts of mdfft_comm_volume are per transform.  batch * T must not exceed
 * 2^40 (E_ARG).
 */
mdfft_status mdfft_plan_batched(mdfft_plan_t *out, int M, const int64_t N[], int64_t P, const int *order,
                                mdfft_dtype dt, unsigned flags, int64_t batch);

/*
 * mdfft_exec -- run the plan: M fused passes, pass s doing the 1-D FFTs along
 * the last axis of layout s (Fig. 4, steps 1..M) and storing straight into
 * layout s+1 (the transposes of Fig. 4; the last one gives natural order).
 *   in_dev, out_dev  device arrays of N_1 ... N_M elements of the plan's
 *                    complex type, 16-byte aligned; in_dev is not modified
 *                    unless in_dev == out_dev (needs MDFFT_PLAN_INPLACE);
 *                    partial overlap is E_ARG.
 *   dir        -1 forward (exp(-2 pi i jk/N), as the paper), +1 inverse
 *              (exp(+2 pi i jk/N)).
 *   normalize  0: no scaling (the paper drops the factor); 1: scale by 1/T
 *              (only allowed with dir = +1, giving the exact inverse).
 *   stream     CUDA stream to launch on.
 */
mdfft_status mdfft_exec(mdfft_plan_t plan, const void *in_dev, void *out_dev, int dir, int normalize,
                        mdfft_stream_t stream);

/*
 * mdfft_exec_graph -- as mdfft_exec, replayed from a CUDA graph.  The first
 * call for a given (in_dev, out_dev, dir, normalize) captures the plan's M
 * pass launches into a graph (on a private stream) and instantiates it; every
 * call then runs the graph with one cudaGraphLaunch on `stream`, which saves
 * the per-kernel launch cost of small transforms.  A plan keeps up to 8
 * graphs (the least recently used is replaced); mdfft_plan_autotune drops
 * them.  Same arguments, checks and results as mdfft_exec; pass timing
 * (mdfft_pass_timing) does not record graph executions.
 */
mdfft_status mdfft_exec_graph(mdfft_plan_t plan, const void *in_dev, void *out_dev, int dir, int normalize,
                              mdfft_stream_t stream);

/*
 * mdfft_selftest_wait -- runs, alone in one thread, the bounded mbarrier wait
 * the persistent pipelined kernels use for their bulk copies: arrive = 0
 * arms the barrier for 16 bytes that no copy brings, so the wait must give up
 * after limit_us microseconds (1 .. 10^7) and the call returns
 * MDFFT_E_TIMEOUT with the device still usable; arrive = 1 completes the phase
 * with a plain arrival and returns MDFFT_OK at once.  *waited_us (may be NULL)
 * receives the host-measured duration.  Synchronous; allocates 4 bytes of
 * device memory for the status.  (Failure detection without a fault.)
 */
mdfft_status mdfft_selftest_wait(int arrive, int64_t limit_us, int64_t *waited_us);

/*
 * mdfft_exec_counted -- as mdfft_exec, and every pass also counts on the
 * device the points its store moves to another virtual process, and the
 * points exchanged for lines cut between processes.
 *   counts_dev  device array of 2*M int64 entries, zeroed by this call:
 *               [s], s < M-1: points whose owner changes from layout s to
 *               s+1; [M-1]: last layout to natural order; [M+s]: split-line
 *               amount of step s.  Equal to mdfft_comm_volume's numbers.
 */
mdfft_status mdfft_exec_counted(mdfft_plan_t plan, const void *in_dev, void *out_dev, int dir,
                                int normalize, mdfft_stream_t stream, int64_t *counts_dev);

/* Communication amounts of a plan's order, in data points (Sec. 3, Sec. 4). */
typedef struct {
    int64_t per_transition[MDFFT_MAX_DIMS]; /* [s], s < M-1: points whose owner changes from layout s to s+1 */
    int64_t total;                          /* sum of per_transition: what the order search minimises */
    int64_t final_to_natural;               /* last layout back to natural order (done, not counted; 0 for
                                               the comparison methods, whose output stays where it is) */
    int64_t split_line[MDFFT_MAX_DIMS];     /* [s]: sum over lines of layout s cut between k owners of N_axis (k-1) */
    int64_t paper_total;                    /* total + sum(split_line): comparable with the Sec. 4 closed forms */
    int regime[MDFFT_MAX_DIMS];             /* [s]: leading dims of layout s that chunks are cut on (f_MD case);
                                               axes cut per step for the comparison methods */
    double amount_slab;                     /* Sec. 4 closed forms for the same T and Np: T - T/Np */
    double amount_pencil;                   /* 2N^3 - 2Np (N^2/Np)^(3/2); NaN unless M = 3 and N_1 = N_2 = N_3 */
    double amount_volumetric;               /* M N^M (N / (N^M/Np)^(1/M) - 1); NaN unless all dims equal */
} mdfft_comm;

/*
 * mdfft_comm_volume -- the plan's amounts, computed on the host by
 * intersecting chunk boxes (every chunk of a row-major range is a union of
 * at most 2M-1 axis-aligned boxes; a comparison method's block is one box).
 * The ownership model is the plan's (MDFFT_PLAN_DECOMP_*).  Works on
 * MDFFT_PLAN_HOST_ONLY plans.
 */
mdfft_status mdfft_comm_volume(mdfft_plan_t plan, mdfft_comm *out);

/*
 * mdfft_chunk -- (row-wise plans) the index map of Sec. 3.2 for process pid in layout `step`
 * (0..M-1; M means the natural output layout): x^s = f_MD(pid),
 * x^e = f_MD(pid+1) - 1 over the dims permuted into that layout, and their
 * coordinates in the layout's axis order (start_coord/end_coord: M entries
 * each, may be NULL).  E_ARG if step or pid is out of range.
 */
mdfft_status mdfft_chunk(mdfft_plan_t plan, int step, int64_t pid, int64_t *xs, int64_t *xe,
                         int64_t start_coord[], int64_t end_coord[]);

/*
 * mdfft_exchange_counts -- the all-to-all-v of transition `step` (layout step
 * to step+1; step = M-1: the last layout back to natural order) when the P
 * virtual processes are laid onto G devices in contiguous blocks (device g
 * holds processes floor(gP/G) .. floor((g+1)P/G)-1, i.e. one contiguous
 * row-major range of every layout).  counts (G*G int64): [g*G + h] = points
 * device g holds before the transition and device h after it; the
 * off-diagonal sum is the data that crosses devices (at most the plan's
 * per-transition amount).  Host only; 1 <= G <= P; row-wise plans only.
 */
mdfft_status mdfft_exchange_counts(mdfft_plan_t plan, int step, int G, int64_t *counts);

/*
 * mdfft_block_grid -- for a plan made with an MDFFT_PLAN_DECOMP_* flag: the
 * blocks every natural axis is cut into in step `step` (0..M-1), q_axis[M]
 * (1: not cut).  E_ARG for row-wise plans or a step out of range.
 */
mdfft_status mdfft_block_grid(mdfft_plan_t plan, int step, int64_t *q_axis);

/* The plan's order (M*M ints), e.g. the one the planner picked for order = NULL. */
mdfft_status mdfft_plan_order(mdfft_plan_t plan, int *order_out);

/*
 * mdfft_order_search -- the order with the smallest (want_worst = 0) or
 * largest (want_worst = 1) total amount over all (M-1)!^M orders (Sec. 3.2,
 * Table 1), by dynamic programming over (step, layout, transformed axes).
 * Layouts that cut the same leading axes in the same order (their regime's
 * first k axes) own every point alike, so one pairwise amount serves each
 * pair of such classes: counted over owner arrays on grids of up to 2^16
 * points, by box intersection above.  Ties go to the lexicographically
 * smallest sequence of layouts.  order_out: M*M ints; total: the amount.
 * M <= 6 (E_UNSUPPORTED above); E_UNSUPPORTED too when the amounts would
 * cost more than about 4e10 operations (large 6-D grids at high P: use
 * mdfft_order_heuristic).
 */
mdfft_status mdfft_order_search(int M, const int64_t N[], int64_t P, int want_worst, int *order_out,
                                int64_t *total);

/*
 * Per-pass device timing.  mdfft_pass_timing(plan, 1) clears the record and
 * makes later executions record a CUDA event on their stream before each
 * pass and after the last one (events only: no host synchronisation), for up
 * to MDFFT_TIMING_SLOTS executions (older ones are overwritten); 0 stops.
 * mdfft_pass_times waits for the recorded executions and writes, for each of
 * the M passes (cap entries at most), the mean duration in milliseconds over
 * them; *n_execs (may be NULL) receives how many executions were averaged.
 */
#define MDFFT_TIMING_SLOTS 512
mdfft_status mdfft_pass_timing(mdfft_plan_t plan, int enable);
mdfft_status mdfft_pass_times(mdfft_plan_t plan, float *ms_out, int cap, int *n_execs);

/*
 * mdfft_exec_host -- end-to-end call on host memory: copies in_host (T
 * elements) into dev_in, runs mdfft_exec(dev_in -> dev_out) and copies dev_out
 * back into out_host, all asynchronously on `stream` (use pinned host memory
 * for overlap; pageable memory works but the copies then block the host).
 * dev_in and dev_out are caller-owned device arrays of T elements (they may
 * be the same array only for MDFFT_PLAN_INPLACE plans).  The host buffers
 * must stay valid until the stream reaches the end of the call.  For a
 * batched plan (all sizes times the batch) the work is pipelined per
 * transform on three streams of the plan (copy in, passes, copy out), forked
 * from and joined back into `stream`, so the two copy directions and the
 * passes of neighbouring transforms overlap; results are identical.
 */
mdfft_status mdfft_exec_host(mdfft_plan_t plan, const void *in_host, void *out_host, void *dev_in, void *dev_out,
                             int dir, int normalize, mdfft_stream_t stream);

/* Launch shape of pass s: line length, tile (lines along the tile axes g and
 * h), threads per CTA, CTAs, bytes of shared memory, the radix plan of the
 * 1-D FFTs and the tile order.  Host information only. */
typedef struct {
    int64_t line_length;
    int tile_g, tile_h, threads, smem_bytes;
    int64_t ctas;      /* tiles */
    int fft_axis, store_axis;  /* store_axis: the tile axis g */
    int64_t grid;      /* CTAs launched (= ctas unless persistent) */
    int persistent;    /* 0: one CTA per tile; 1 to 3: persistent kernel with that many landing buffers
                          (ring slots for variants 17-22 of mdfft_plan_tuning) */
    int stages;        /* radix stages of the line length's plan */
    int radix[12];     /* their radices, first stage first (e.g. 16, 16 for 256) */
    int tile_order;    /* 0: g is the output layout's fastest axis (runs of tile_g elements stored);
                          1: input-chunk order (g, h the input layout's second and third fastest axes,
                          tiles in the input's row-major line order: a tile of whole f_MD chunks is one
                          chunk, CTA t owning chunk t) */
} mdfft_pass_info;
mdfft_status mdfft_pass_describe(mdfft_plan_t plan, int s, mdfft_pass_info *out);

/*
 * mdfft_plan_autotune -- for every pass, times the kernel variants built for
 * its line length (the default launch shape and, for complex64 lengths 32,
 * 48, 64, 96, 128, 160, 192, 256, 512, fixed 256- and 512-thread CTAs) with
 * several tile shapes (lines along the output's fastest axis x lines along
 * the next axis), `reps` launches each, and keeps the fastest.  For even
 * complex64 lengths up to 512 the candidates include a persistent kernel
 * that streams tiles through shared memory with bulk (TMA) copies, and for
 * lengths 16, 24, 32, 48, 64, 96, 128 and 256 one that streams them through
 * a ring of two or three shared-memory slots filled by 16-byte asynchronous
 * copies, at a capped number of CTAs per SM, and for even lengths up to 64
 * a kernel with one thread per line that keeps the line in registers through
 * every radix stage; a plan using any of them needs 16-byte aligned arrays
 * in mdfft_exec (E_ARG otherwise).
 * Tensor-core plans (lengths 128, 256, 512) also try 128-thread CTAs (half
 * the lines per tile, more CTAs per SM) and, for 256 and 512, CTAs of two
 * independent 128-thread groups, and non-persistent kernels the
 * input-chunk tile order (mdfft_pass_info.tile_order).  Plans made with
 * MDFFT_PLAN_TUNE_RADIX (complex64) also try the alternative radix plan of
 * the length (its twiddle table is made again for the chosen plan).  Kernel
 * variant, tiling and tile order never change results; a different radix
 * plan changes the rounding only.  in_dev (T elements, only read) and out_dev (T elements,
 * overwritten with scratch) are the caller's; the call synchronises `stream`.
 * ms_before / ms_after (M entries each, may be NULL) receive the mean pass
 * times of the default and of the chosen configuration.
 */
/*
 * mdfft_plan_tuning / mdfft_plan_set_tuning -- a plan's launch choices as 4
 * int32 per pass (kernel variant: 0 default, 1 fixed 256-thread CTAs, 2
 * fixed 512-thread CTAs, 3 / 4 persistent pipelined with 1 / 2 landing
 * buffers, 5 tensor-core kernel with 128-thread CTAs, 6 / 7 fixed 192 /
 * 384-thread CTAs (lengths 24, 48), 8 the alternative radix plan (lengths 32,
 * 48, 64, 96, 128, 160, 192, 256, 512: e.g. 8x8x4 for 256, 8x8x8 for 512),
 * 9 the default shape capped at the registers of 6 CTAs per SM (24 .. 64),
 * 10 / 11 the tensor-core kernel whose 128-thread groups each walk their
 * own tiles (lengths 256 and 512; tiles of 8 or 4 lines), with landing
 * buffers / loading the first stage from HBM, 12 / 13 a persistent complex64
 * kernel that loads the next tile's first-stage inputs into registers while
 * the current tile runs (lengths 24, 32, 48, 64; registers for 2 / 4 CTAs
 * per SM), 14 / 15 the same with the alternative radix plan (64), 16 the
 * 256-point kernel that exchanges values between its two radix-16 stages
 * with warp shuffles instead of shared memory, 17 / 18 / 19 / 20 the
 * persistent ring-of-slots kernel with 2 / 3 / 2 / 2 slots at most 3 / 2 / 4
 * / 2 CTAs per SM (lengths 16, 24, 32, 48, 64, 96, 128, 256), 21 / 22 the
 * same as 17 / 18 with the alternative radix plan (64), 23 one thread per
 * line with every radix stage in registers (lengths 8, 12, 16, 20, 24, 30,
 * 32, 40, 48, 60, 64; 16-byte aligned arrays; 128-line CTAs), 24 the same
 * with 64-line CTAs (48, 60, 64), 25 the same with the alternative radix
 * plan (32, 64), 26 / 27 two threads per line, the stages in registers and
 * one exchange of values between them (32, 64; default / alternative radix
 * plan);
 * lines per tile along g; lines per tile along h; tile order 0 or 1, see
 * mdfft_pass_info), e.g. after
 * mdfft_plan_autotune, to store and give back to a plan of the same dims, P,
 * order, dtype, batch and flags.  set_tuning checks every pass (variant built
 * for its length and dtype, tile within the kernel's lines and the pass's
 * extents) before changing any; it drops captured graphs.  Results do not
 * depend on the tuning.  cap / n: 4 M.  Host-only plans: E_ARG.
 */
mdfft_status mdfft_plan_tuning(mdfft_plan_t plan, int32_t *out, int cap);
mdfft_status mdfft_plan_set_tuning(mdfft_plan_t plan, const int32_t *in, int n);

mdfft_status mdfft_plan_autotune(mdfft_plan_t plan, const void *in_dev, void *out_dev, int reps, mdfft_stream_t stream,
                                 float *ms_before, float *ms_after);

/*
 * mdfft_pattern_probe -- runs `reps` times, on `stream`, a kernel that moves
 * the data of pass s exactly like the plan's default pass kernel (the pass's
 * tiles as built or autotuned when they fit the default CTA, else the
 * default tiling; same loads, the same transposed stores into the next
 * layout) but does no butterflies, and returns its mean duration in ms.  Its bandwidth is the
 * bound the redistribution's access pattern puts on the pass.  complex64
 * plans and line lengths 24, 32, 48, 64, 96, 128, 160, 192, 256, 512 only
 * (E_UNSUPPORTED otherwise).  in_dev is read, out_dev overwritten (T
 * elements each); synchronises the stream.
 */
mdfft_status mdfft_pattern_probe(mdfft_plan_t plan, int s, const void *in_dev, void *out_dev, int reps,
                                 mdfft_stream_t stream, float *ms);

/*
 * mdfft_movement_probe -- the same data movement (out_dev receives what
 * mdfft_pattern_probe writes) by a persistent kernel that streams the tiles
 * through `slots` (2 or 3) shared-memory slots filled by 16-byte asynchronous
 * copies, at most `per_sm` (1-8) CTAs per SM (tiles chosen as in
 * mdfft_pattern_probe): the structure of the ring-of-slots pass kernel
 * without its butterflies, so S - 1 tiles' loads stay in flight per CTA.  Its bandwidth bounds a pass kernel that hides the
 * load latency that far.  complex64 plans, line lengths 16, 24, 32, 48, 64,
 * 96, 128, 256, in_dev and out_dev 16-byte aligned (E_ARG / E_UNSUPPORTED
 * otherwise); mean duration of `reps` launches in *ms; synchronises the stream.
 */
mdfft_status mdfft_movement_probe(mdfft_plan_t plan, int s, int slots, int per_sm, const void *in_dev, void *out_dev,
                                  int reps, mdfft_stream_t stream, float *ms);

/*
 * mdfft_fp64_rate_probe -- measures the device's FP64 multiply-add rate, the
 * denominator of the complex128 path's ALU roofline (that path is bound by
 * the FP64 pipe, not by HBM).  A kernel of `ctas` CTAs x 256 threads runs, in
 * every thread, 8 independent chains of `iters` fused multiply-adds (no
 * memory traffic inside the loop), timed with CUDA events on `stream`
 * (synchronised); *tflops = 2 x (multiply-adds executed) / seconds / 1e12.
 *   out_dev   caller-owned device array of ctas x 256 doubles; each thread
 *             writes the sum of its chains there, so no chain is optimised away.
 *   ctas      1 .. 2^20; iters 1 .. 2^24.
 */
mdfft_status mdfft_fp64_rate_probe(double *out_dev, int ctas, int64_t iters, mdfft_stream_t stream,
                                   double *tflops);

/* Waits for the device and reports whether a pass kernel of this plan gave up
 * a bounded wait since the last check (MDFFT_E_TIMEOUT; the affected output
 * is incomplete).  The kernels that wait on the device are the persistent
 * pipelined kernels that mdfft_plan_autotune may select and the tensor-core
 * kernels of MDFFT_C64_TC_FP16 / _BF16 plans (bulk copies, MMA completion). */
mdfft_status mdfft_plan_check(mdfft_plan_t plan);

/* Device workspace the plan owns, in bytes (0 for host-only plans). */
mdfft_status mdfft_workspace_size(mdfft_plan_t plan, size_t *bytes);

/* Number of kernel launches one mdfft_exec makes (M). */
mdfft_status mdfft_launches_per_exec(mdfft_plan_t plan, int *launches);

/* Is line length n built into this library for dtype dt?  1 yes, 0 no. */
int mdfft_supported_length(int64_t n, mdfft_dtype dt);

mdfft_status mdfft_destroy(mdfft_plan_t plan);

/*
 * Serving: many M-D FFTs of different shapes, continuously batched.
 * (Not in the paper; the engine runs the paper's passes of mdfft_exec.)
 *
 * A server owns a plan per shape (planner's best order for P virtual
 * processes, complex64), a device arena for the workspaces of the requests
 * in flight, and a CUDA graph per table slot.  mdfft_server_step() admits
 * queued requests first come first served while the HBM budget (each request
 * is charged input + output + workspace = 3 T 8 bytes) and the slot count
 * allow, then launches -- as one graph launch of one persistent kernel -- the
 * next pass of every request in flight, whatever its shape.  A request that
 * arrives while others are on the GPU joins at the next step; it leaves after
 * its last pass.  Requests advance one pass per step, so a step has no
 * dependencies inside it and nothing waits on the device.  At low load --
 * no request queued and at most `direct` requests with passes left
 * (mdfft_server_set_direct, default 4) -- a step instead launches every
 * remaining pass of those requests, oldest first, as plain pass launches
 * (those of mdfft_exec): a lone request then runs its passes back to back
 * instead of one per step.  Line lengths
 * 16, 24, 32, 48, 64, 96, 128, 160, 192, 256 run inside the persistent
 * kernel; passes of 16 to 64 points whose arrays are 16-byte aligned go
 * instead to a second persistent kernel of the same graph, launched after
 * it, that runs one thread per line with every radix stage in registers
 * (mdfft_server_set_line_kernel); other supported lengths run as separate
 * launches in the same step.  Results are the same as mdfft_exec's for the
 * same shape (the same radix plans and butterflies in the same order).  All work goes to `stream`; the caller's buffers must stay valid
 * until the request is done.  Errors: E_ARG, E_RANGE (request above the
 * whole budget), E_UNSUPPORTED, E_NOMEM, E_CUDA.
 */
typedef struct mdfft_server_s *mdfft_server_t;

typedef struct {
    int64_t submitted, admitted, completed;
    int64_t steps, graph_launches, kernel_launches;
    int64_t inflight, queued;
    size_t bytes_in_use, budget_bytes;
    int grid_ctas; /* CTAs of the persistent kernel */
    int64_t cancelled;
    int64_t direct_requests; /* requests whose remaining passes ran as plain launches (low load) */
} mdfft_server_stats;

/* budget_bytes: HBM admission budget; max_inflight: 1..512 requests in
 * flight; P: virtual processes of every request's plan (min(P, T)). */
mdfft_status mdfft_server_create(mdfft_server_t *out, size_t budget_bytes, int max_inflight, int64_t P,
                                 mdfft_stream_t stream);
/* Queues one transform of dims N[0..M) from in_dev to out_dev (device
 * complex64 arrays, not overlapping).  *request_id identifies it. */
mdfft_status mdfft_server_submit(mdfft_server_t s, int M, const int64_t N[], const void *in_dev, void *out_dev,
                                 int dir, int normalize, int64_t *request_id);
/* One scheduling step (see above); *launched = 1 if work was launched. */
mdfft_status mdfft_server_step(mdfft_server_t s, int *launched);
/* Up to max_steps steps in a row, stopping at the first that launches
 * nothing; *steps (may be NULL) receives how many launched.  Requests
 * admitted by the first step can run all their passes within one call. */
mdfft_status mdfft_server_run(mdfft_server_t s, int max_steps, int *steps);
/* *done = 1 once the request's result is in out_dev; *done_ms (may be NULL)
 * is then its completion time on the server clock, in ms since the last
 * mdfft_server_reset_clock (or creation), taken from CUDA events. */
mdfft_status mdfft_server_poll(mdfft_server_t s, int64_t request_id, int *done, double *done_ms);
/* Forget a finished (or cancelled) request. */
mdfft_status mdfft_server_release(mdfft_server_t s, int64_t request_id);
/* Cancels a request: a queued one is dropped before it reaches the GPU; an
 * admitted one gets no further passes and its budget and workspace come back
 * once its latest step has run (its out_dev then holds partial results).  A
 * request whose last pass is already on the GPU completes normally.  A
 * cancelled request polls as done with done_ms = -1.  E_ARG for unknown,
 * finished or already cancelled requests. */
mdfft_status mdfft_server_cancel(mdfft_server_t s, int64_t request_id);
/* Steps until every submitted request is done (blocks the host). */
mdfft_status mdfft_server_drain(mdfft_server_t s);
/* Sets the server clock's zero to now (records an event on the stream and waits for it). */
mdfft_status mdfft_server_reset_clock(mdfft_server_t s);
/* Re-captures the graphs with a persistent grid of `ctas` CTAs (autotuning). */
mdfft_status mdfft_server_set_grid(mdfft_server_t s, int ctas);
/* Steps in flight on the GPU at most (1..8, default 2): a batched step is
 * launched only while fewer are outstanding, so requests arriving meanwhile
 * share the next step instead of each adding nearly empty ones (low-load
 * direct steps are held back only while batched steps are in flight). */
mdfft_status mdfft_server_set_depth(mdfft_server_t s, int depth);
/* At most this many consecutive tiles (1..64, default 4) are dealt to a CTA
 * of the persistent kernel at a time; each step deals chunks of its tile
 * count / grid, between 1 and this maximum, so that small steps still use
 * every CTA.  Larger chunks mean fewer item lookups, smaller ones evener
 * load.  Results do not depend on it. */
mdfft_status mdfft_server_set_chunk(mdfft_server_t s, int chunk);
/* Low-load threshold (0..64, default 4; 0 never): a step with no request
 * queued and at most this many requests with passes left launches all their
 * remaining passes directly, oldest request first.  Results do not depend on
 * it. */
mdfft_status mdfft_server_set_direct(mdfft_server_t s, int max_requests);
/* 1 (default): passes of 16 to 64 points with 16-byte aligned arrays run in
 * the line kernel of the step; 0: in the grouped persistent kernel like the
 * other lengths.  Takes effect at the next step; results do not depend on
 * it.  E_ARG unless enable is 0 or 1. */
mdfft_status mdfft_server_set_line_kernel(mdfft_server_t s, int enable);
mdfft_status mdfft_server_get_stats(mdfft_server_t s, mdfft_server_stats *out);
mdfft_status mdfft_server_destroy(mdfft_server_t s);

/*
 * mdfft_exec_noalloc -- the transform of mdfft_plan + mdfft_exec, for callers
 * that cannot let a library allocate GPU memory: applications whose device
 * memory is owned by their own allocator or memory pool, and loops where the
 * device-wide synchronisation that cudaMalloc and cudaFree may cause is not
 * acceptable.  The paper has no counterpart to this entry point; it is a
 * property of this library's interface only.
 *
 * It allocates nothing: no cudaMalloc, cudaFree or any other device allocator
 * (torch's included), and no host heap memory on success.  Its scratch -- the
 * twiddle tables and the array the passes ping-pong through -- is one static
 * device array of MDFFT_NOALLOC_SCRATCH_BYTES that every GPU which loads the
 * library holds until the process exits.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) and caches it; make that
 * first call on each device before any stream capture.  The cached address
 * does not survive cudaDeviceReset: after resetting a device, do not call
 * this entry point on it again in the same process.
 *   M, N, dt, dir, normalize  as for mdfft_plan / mdfft_exec.
 *   order     M*M axis ids as for mdfft_plan; required (NULL is E_ARG) --
 *             get the best order from mdfft_order_search beforehand.
 *   in, out   caller-owned device arrays of N_1 ... N_M elements; they must not
 *             overlap (no in-place); in is not modified.
 * Limits: N_1 ... N_M * element size <= MDFFT_NOALLOC_MAX_ARRAY_BYTES, else
 * E_UNSUPPORTED with a message.  The virtual process count of mdfft_plan is
 * not an argument: it changes no result.
 * Every call shares the one scratch array and leaves its contents behind;
 * nothing in it needs to start at zero (each call writes every scratch byte
 * it reads before reading it).  Calls that can overlap on the GPU -- on
 * different streams, or from different host threads, on one device -- race on
 * the scratch and give wrong results: serialise them.
 */
#define MDFFT_NOALLOC_SCRATCH_BYTES (64ull << 20)
#define MDFFT_NOALLOC_MAX_ARRAY_BYTES (MDFFT_NOALLOC_SCRATCH_BYTES - (256ull << 10))
mdfft_status mdfft_exec_noalloc(int M, const int64_t N[], const int *order, mdfft_dtype dt, const void *in_dev,
                                void *out_dev, int dir, int normalize, mdfft_stream_t stream);

/*
 * Distributed data plane (Sec. 1's setting; the "Transpose" steps of Fig. 4)
 * for the P virtual processes placed on G devices: device g holds processes
 * floor(gP/G) .. floor((g+1)P/G) - 1, i.e. one contiguous row-major range of
 * every layout.  A transform on G devices runs, for step s = 0 .. M-1 on
 * every device g:
 *   mdfft_dist_lines(s)   the 1-D DFTs along layout s's last axis over the
 *                         device's range (lines whole, no transpose);
 *   mdfft_dist_pack(s)    the range's points grouped by destination device
 *                         h = 0 .. G-1 (its owner in layout s+1, natural
 *                         order after the last step) into a send buffer;
 *   the caller's all-to-all-v: device g sends counts[g*G + h] points to h
 *                         (mdfft_exchange_counts(plan, s, G, counts)), h's
 *                         receive buffer holds the groups from g = 0 .. G-1
 *                         back to back;
 *   mdfft_dist_unpack(s)  the receive buffer into the device's range of
 *                         layout s+1.
 * Group (g -> h) lists its points in an order both sides derive from the plan
 * (the intersections of the planner's boxes of the two ranges, each in layout
 * s+1's row-major order), so only values travel.  The library moves no data
 * between devices and needs no peer access: remote data reaches local memory
 * through the caller's transport (NCCL's grouped send/recv through
 * torch.distributed, or host copies) before the unpack.  Plans must be
 * row-wise (no MDFFT_PLAN_DECOMP_*), of batch 1, with natural output order.
 * Local arrays are device memory of the range's length (x1 - x0 of
 * mdfft_dist_local_range); a send or receive buffer holds sum of the row or
 * column of counts.  The first pack or unpack of a (step, G, device)
 * allocates its copy list on the device (kept by the plan).  Everything is
 * asynchronous on `stream`.  Errors: E_ARG; E_UNSUPPORTED from
 * mdfft_dist_lines when a device boundary splits a line of that step (the
 * M-D regime with too many devices).
 */
/* [*x0, *x1): device g's range of layout `step` (0 .. M; M: natural order). */
mdfft_status mdfft_dist_local_range(mdfft_plan_t plan, int step, int G, int g, int64_t *x0, int64_t *x1);
/* Step `step`'s line DFTs of device g (dir, normalize as for mdfft_exec: the
 * inverse conjugates step 0's input and step M-1's output, normalize scales
 * step M-1's output by 1/T); in_local == out_local is allowed. */
mdfft_status mdfft_dist_lines(mdfft_plan_t plan, int step, int G, int g, const void *in_local, void *out_local,
                              int dir, int normalize, mdfft_stream_t stream);
/* Device g's range of layout `step` -> send buffer, grouped by destination. */
mdfft_status mdfft_dist_pack(mdfft_plan_t plan, int step, int G, int g, const void *local, void *sendbuf,
                             mdfft_stream_t stream);
/* Receive buffer (groups from every source device, in device order) ->
 * device h's range of layout step+1. */
mdfft_status mdfft_dist_unpack(mdfft_plan_t plan, int step, int G, int h, const void *recvbuf, void *local,
                               mdfft_stream_t stream);

/* Message of the last failure on the calling thread ("" if none). */
const char *mdfft_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MDFFT_H */
