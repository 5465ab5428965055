/*
 * dsanls.h -- C ABI of the GB300 sketched-ANLS library (libdsanls.so).
 *
 * The library computes nonnegative matrix factorisations M ~ U V^T
 * (M m x n, U m x k, V n x k, all >= 0; Section 2.1, eq. problem) with the
 * sketched alternating nonnegative least squares method of Section 3
 * (SANLS; the single-node body of DSANLS, Alg. 2).  One outer iteration t:
 *
 *   U-half: draw S^t (n x d); A = M S^t; B = V^T S^t; G = B B^T; R = A B^T;
 *           U <- solver(U, G, R, t)           (Section 3.2, eq. sketched_u)
 *   V-half: draw S'^t (m x d'); the same with M^T and the new U
 *                                             (eq. sketched_v, Alg. 1 line 4)
 *
 * solver = projected gradient (eq. gradient_descent) or proximal coordinate
 * descent (Alg. 3, eq. entry_sol); sketches: Gaussian N(0,1/d), column
 * subsampling without replacement, or the identity (Section 3.4).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an int status (DSANLS_OK = 0 or a negative code
 *    below); no C++ exception crosses the ABI.  Handle calls store a message
 *    retrievable with dsanls_last_error().
 *  - Matrices are row-major binary32 unless stated otherwise.
 *  - Input arrays are copied; the caller keeps ownership of everything it
 *    passes.  Output buffers are caller-owned.
 *  - "on_device" = 1 means the pointer is CUDA device memory of the current
 *    device, 0 means host memory (pageable or pinned).
 *  - A handle is bound to the CUDA device current at dsanls_create and is
 *    not thread-safe: use one handle per host thread.
 *  - Work is queued on the handle's stream (dsanls_options.stream; NULL
 *    selects a non-blocking stream created and owned by the handle).  dsanls_step returns once the work is
 *    queued; an asynchronous failure (a CUDA error, a NaN/Inf produced by an
 *    update) surfaces at the next synchronising call (dsanls_rel_error,
 *    dsanls_get_factors, dsanls_sync).
 */
#ifndef DSANLS_H
#define DSANLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define DSANLS_OK 0
#define DSANLS_EINVAL (-1)    /* bad argument (size, pointer, kind, option)      */
#define DSANLS_ENOMEM (-2)    /* device or host allocation failed               */
#define DSANLS_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed     */
#define DSANLS_ESTATE (-4)    /* call out of order, e.g. step before set_dense   */
#define DSANLS_ENUMERIC (-5)  /* an update produced NaN or Inf                   */
#define DSANLS_ETIMEOUT (-6)  /* a bounded device wait gave up                   */

/* ---- sketch kinds (Section 3.4) ------------------------------------- */
#define DSANLS_SKETCH_GAUSSIAN 0   /* i.i.d. N(0, 1/d) entries                       */
#define DSANLS_SKETCH_SUBSAMPLE 1  /* d columns sqrt(n/d) e_i, drawn w/o replacement */
#define DSANLS_SKETCH_IDENTITY 2   /* S = I (needs d = n and d_v = m)                */
#define DSANLS_SKETCH_RADEMACHER 3 /* i.i.d. +-1/sqrt(d) entries: the sign is the top
                                      bit of the entry's Philox word (one of Section
                                      3.4's other random matrices; E[S S^T] = I).
                                      Accepted wherever GAUSSIAN is (all orders and
                                      precisions; not by the batched form)         */
#define DSANLS_SKETCH_COUNT 4      /* count sketch: one entry +-1 per row of S, in the
                                      bucket ((w >> 1) * d) >> 31 with sign -1 for odd
                                      w, w the row's Philox word (column 0, stream
                                      0x30 | side); E[S S^T] = I, no scaling.  Runs
                                      through the dense-sketch paths like GAUSSIAN
                                      (S materialised; not by the batched form)   */
#define DSANLS_SKETCH_SRHT 5       /* subsampled randomized Hadamard transform
                                      S = sqrt(p/d) D H R (Section 3.4's third named
                                      choice): p = the dimension rounded up to a
                                      power of two, H the normalised p x p Sylvester
                                      Walsh-Hadamard matrix, D row signs (top bit of
                                      the row's word, column 0, stream 0x40 | side),
                                      R d of the p columns drawn without replacement
                                      (the subsampling draw with side 0x40 | side),
                                      ascending.  Entry (i, j) = D_i (-1)^popcount(
                                      i & J_j) / sqrt(d); needs d <= p.  Runs through
                                      the dense-sketch paths like GAUSSIAN (S
                                      materialised; not by the batched form)       */

/* ---- subproblem solvers (Section 3.5) -------------------------------- */
#define DSANLS_SOLVER_PGD 0   /* one projected gradient step, eq. gradient_descent */
#define DSANLS_SOLVER_RCD 1   /* proximal coordinate descent, Alg. 3               */
/* The row update's U G is binary32-accurate in every precision: for one PGD
 * step with 32 < k <= 128 it runs on tensor cores from a three-way bf16 split
 * of U and G (six products, fp32 accumulation; dropped terms of order 2^-24
 * of the product), otherwise on CUDA cores in binary32. */

/* ---- arithmetic of the sketched products A = M S and R = A B^T -------- */
#define DSANLS_PREC_FP32 0    /* binary32 operands and accumulation (CUDA cores)  */
#define DSANLS_PREC_BF16 1    /* bf16 operands, fp32 accumulation (tcgen05)       */
#define DSANLS_PREC_FP8 2     /* fp8 E4M3 M (one scale per 128-row block) and S
                                 (entries N(0,1), 1/sqrt(d) applied to the fp32
                                 accumulator); B = Y^T S and R = A B^T in bf16   */

/* ---- order of the Gaussian right-hand side R = M S B^T ----------------- */
#define DSANLS_ORDER_PAPER 0  /* R = (M S) B^T: A = M S first (eq. def_A_B), then
                                 A B^T (eq. gradient_descent); 2 rows K d flops   */
#define DSANLS_ORDER_REASSOCIATED 1
                              /* R = M (S B^T): P = S B^T (K x k) first, then
                                 M P; 2 K d k + 2 rows K k flops.  Equal in exact
                                 arithmetic (associativity), rounded differently;
                                 dense sketches (Gaussian, Rademacher) with FP32
                                 (dense or sparse M), BF16 (dense M: S, B and P
                                 rounded to bf16) or FP8 (dense M: B and P^T
                                 from bf16 operands, then M in E4M3 per 128-row
                                 block and P^T in E4M3 per row for R = M P)      */

/* ---- Philox field streams (counter word 3, low byte) ------------------ */
#define DSANLS_STREAM_SKETCH_U 0
#define DSANLS_STREAM_SKETCH_V 1
#define DSANLS_STREAM_INIT_U 2
#define DSANLS_STREAM_INIT_V 3

typedef struct dsanls_options {
    int32_t solver;        /* DSANLS_SOLVER_*; default PGD                           */
    int32_t precision;     /* DSANLS_PREC_*; default FP32                            */
    int32_t d_v;           /* sketch size d' of the V-half; 0 = same as d            */
    int32_t power_iters;   /* power iterations for lambda_max(G); default 32         */
    double alpha;          /* mu_t = alpha + beta * t (eq. reg_sub); default 1       */
    double beta;           /* default 1                                              */
    int64_t t;             /* iteration index of the next outer iteration; default 0 */
    int32_t bound_clamp;   /* 1: clamp entries at sqrt(2 ||M||_F) (eq. extra_con)    */
    int32_t use_graph;     /* 1: replay each outer iteration as a CUDA graph         */
    int32_t order;         /* DSANLS_ORDER_*; default PAPER                          */
    int32_t inner_iters;   /* PGD: projected-gradient steps per half-step on the
                              proximal row objective 1/2 x^T (G + mu_t I) x -
                              (r + mu_t u)^T x (eq. reg_sub), from x = u; 1 (the
                              default) is the single step of eq. gradient_descent.
                              1..256; must be 1 with RCD and in the batched form */
    void *stream;          /* cudaStream_t for all work; NULL = the handle's own     */
    int32_t regen_sketch;  /* BF16, paper order, Gaussian sketch: 1 draws S inside the
                              tensor-core GEMMs (warps of the GEMM compute each S^T
                              tile from the Philox field) instead of a sketch pre-pass
                              read by TMA; bitwise the same results.  Default 0: the
                              pre-pass, measured faster (the draw costs ~45 ALU ops per
                              entry and is repeated by every row tile)               */
} dsanls_options;

typedef struct dsanls_ctx *dsanls_t;

/* Fill *opt with the defaults listed above. */
int dsanls_default_options(dsanls_options *opt);

/* Create a handle for an m x n problem of rank k with sketch size d for the
 * U-half (and, unless set_options overrides d_v, for the V-half).
 * seed keys the Philox field (S^t, S'^t, default U^0, V^0; Section 3.3's
 * shared seed).  Requires m, n >= 1, 1 <= k <= 128, d >= 1; for SUBSAMPLE
 * d <= n; for IDENTITY d == n.  Factors start as the default
 * Uniform[0,1) draws of streams 2 and 3.  EINVAL, ENOMEM, ECUDA. */
int dsanls_create(int64_t m, int64_t n, int32_t k, int32_t d, int32_t sketch_kind,
                  uint64_t seed, dsanls_t *out);

int dsanls_get_options(dsanls_t h, dsanls_options *opt);
/* Validates and applies options; d_v follows the same rules as d for the
 * V-half (against m).  BF16 needs dense data and a Gaussian or identity
 * sketch (identity: R = M V from bf16 operands, the unsketched subproblem),
 * FP8 dense data and a Gaussian sketch; BF16 needs m, n, d, d_v multiples of
 * 8, FP8 m and n multiples of 16.
 * ORDER_REASSOCIATED needs a Gaussian or Rademacher sketch (EINVAL
 * otherwise). */
int dsanls_set_options(dsanls_t h, const dsanls_options *opt);

/* Dense M: m rows of n binary32 values, row stride ld >= n (elements).  The
 * library keeps M and M^T in device memory (plus bf16 copies when the BF16
 * precision is selected).  Synchronises the handle's stream. */
int dsanls_set_dense(dsanls_t h, const float *M, int64_t ld, int32_t on_device);

/* Sparse M in CSR: rowptr[m+1] (int64, rowptr[0] = 0, nondecreasing,
 * rowptr[m] = nnz), col[nnz] (int32 in [0,n), strictly increasing within a
 * row), val[nnz].  The transposed CSR (CSR of M^T, n rows) may be passed in
 * t_rowptr/t_col/t_val; if t_rowptr is NULL the library builds it on the host
 * (host inputs only).  Synchronises the handle's stream. */
int dsanls_set_csr(dsanls_t h, const int64_t *rowptr, const int32_t *col, const float *val,
                   int64_t nnz, const int64_t *t_rowptr, const int32_t *t_col,
                   const float *t_val, int32_t on_device);

/* Replace U (m x k) and V (n x k), both row-major; either may be NULL to keep
 * the current one.  Values are used as given (no projection). */
int dsanls_set_factors(dsanls_t h, const float *U, const float *V, int32_t on_device);

/* Run outer_iters outer iterations (Alg. 1/Alg. 2 loop body: U-half then
 * V-half), advancing t by outer_iters.  Asynchronous on the stream. */
int dsanls_step(dsanls_t h, int32_t outer_iters);

/* Run only one half at the current t without advancing t: side 0 updates U
 * (eq. sketched_u), side 1 updates V (eq. sketched_v) using the current U. */
int dsanls_half_step(dsanls_t h, int32_t side);

/* ||M - U V^T||_F / ||M||_F of the current factors (Section 5.1), FP64
 * accumulation.  Synchronises; reports pending asynchronous errors. */
int dsanls_rel_error(dsanls_t h, double *out);

/* Copy U (m x k) and V (n x k) out; either may be NULL.  Synchronises. */
int dsanls_get_factors(dsanls_t h, float *U, float *V, int32_t on_device);

/* G (k x k, FP64, row-major) and eta of the last half-step of the given
 * side, for inspection; either output may be NULL.  Synchronises. */
int dsanls_get_gram(dsanls_t h, int32_t side, double *G, double *eta);

/* Wait for all queued work; reports pending asynchronous errors. */
int dsanls_sync(dsanls_t h);

/* ---- profiling ---------------------------------------------------------
 * Phases of one half-step, timed by dsanls_profile_half_step. */
#define DSANLS_PHASE_SKETCH 0     /* draw S^t: Philox field or Feistel indices          */
#define DSANLS_PHASE_B 1          /* B = Y^T S (eq. def_A_B)                            */
#define DSANLS_PHASE_PRODUCT 2    /* A = X S (dense: the O(mnd) GEMM; sparse: SpMM)     */
#define DSANLS_PHASE_RHS 3        /* R = A B^T (zero when fused into PRODUCT)           */
#define DSANLS_PHASE_GRAM 4       /* G = B B^T in FP64                                  */
#define DSANLS_PHASE_STEP_SIZE 5  /* lambda_max(G), mu_t, eta_t                         */
#define DSANLS_PHASE_UPDATE 6     /* fused NNLS row update                              */
#define DSANLS_NPHASES 7

/* Run the half-step of `side` reps times (it updates the factor like
 * dsanls_half_step) with CUDA events on the handle's stream at every phase
 * boundary; ms[0..DSANLS_NPHASES) receives the mean milliseconds per phase.
 * Synchronises. */
int dsanls_profile_half_step(dsanls_t h, int32_t side, int32_t reps, double *ms);

/* Cumulative number of kernel launches issued by the library in this
 * process (a replayed CUDA graph counts each of its kernels).  No GPU work. */
int dsanls_kernel_launches(uint64_t *out);

/* ---- test switches (no counterpart in the paper) ------------------------
 * For tests of the failure paths without faulting the GPU.  Both are
 * process-wide and off by default.
 *
 * dsanls_debug_fail_alloc_after(n): n >= 0 lets the next n device
 * allocations of handles (dsanls_create, set_*, step workspaces) succeed and
 * makes the one after fail as if the device were out of memory (the call
 * returns DSANLS_ENOMEM and releases what it had allocated); n < 0 turns the
 * switch off.  Never fails itself.
 *
 * dsanls_debug_tc_wait(wait_ns, starve), on the current device: wait_ns > 0
 * replaces the 2 s limit of the bounded waits of the tensor-core kernels
 * (0 restores it); starve = 1 (needs wait_ns > 0) makes the TMA producer of
 * the tensor-core GEMM issue no copy, so its consumers' waits run out with
 * nothing in flight: the kernel frees its tensor memory, returns, and the
 * next synchronising call of the handle reports DSANLS_ETIMEOUT.  EINVAL for
 * starve outside {0, 1} or starve without a limit; ECUDA if the device
 * symbols cannot be written.  Synchronous. */
int dsanls_debug_fail_alloc_after(int64_t n);
int dsanls_debug_tc_wait(uint64_t wait_ns, int32_t starve);
/* Index checks of the debug build: a library compiled with -DDSANLS_BOUNDS
 * (paper_2009_02845_gb300.build.build(bounds=True) -> libdsanls_bounds.so)
 * checks every index it takes from the data -- the columns of a CSR, the row
 * keys and scatter destinations of the sub-CSR build -- against its array,
 * skips an access that would leave it and counts it.  out[0] = failed checks
 * since the last reset, out[1] = site code of the first (101-105: sub-CSR
 * gather, scatter and right-hand side; 201-202: CSR product), out[2] = its
 * index; reset = 1 clears them.  Returns 1 in the checking build, 0 in the
 * normal one (out all 0), EINVAL for a NULL out.  Synchronous. */
int dsanls_debug_bounds_report(int32_t reset, int64_t *out);

/* Message of the last failed call on handle h; with h == NULL, of the last
 * failed dsanls_create or stateless primitive on the calling thread ("" if
 * none).  The string stays valid until the next call that fails. */
const char *dsanls_last_error(dsanls_t h);
void dsanls_destroy(dsanls_t h);

/* ---- stateless primitives of the hot path (device pointers) ----------
 * Each runs on `stream` (cudaStream_t, NULL = default) and returns after
 * queuing; EINVAL on bad sizes or NULL pointers, ECUDA on launch failure. */

/* Raw Philox4x32-10 words of the field: out[i*cols + j] = word (i & 3) of
 * Philox(counter = (i >> 2, j, t mod 2^32, stream_id | (t >> 32) << 8),
 *        key = (seed mod 2^32, seed >> 32))   (Salmon et al. 2011). */
int dsanls_philox_field(uint64_t seed, uint32_t stream_id, uint64_t t, int64_t rows,
                        int64_t cols, uint32_t *out, void *stream);

/* Gaussian sketch entries S[i][j] = z(i, j) * scale for i < rows, j < cols,
 * z standard normal by Box-Muller on the field words (pairs (w0,w1) give rows
 * 4q, 4q+1, (w2,w3) rows 4q+2, 4q+3) -- the N(0, 1/d) matrix of Section 3.4
 * with scale = 1/sqrt(d).  transposed = 0 writes S row-major (rows x cols),
 * 1 writes S^T row-major (cols x rows). */
int dsanls_gaussian_field(uint64_t seed, uint32_t stream_id, uint64_t t, int64_t rows,
                          int64_t cols, float scale, int32_t transposed, float *out,
                          void *stream);

/* Rademacher sketch entries S[i][j] = (top bit of w(i, j) set ? -scale :
 * +scale), w the entry's field word (same counter layout as above); the
 * +-1/sqrt(d) matrix of DSANLS_SKETCH_RADEMACHER with scale = 1/sqrt(d).
 * transposed as above. */
int dsanls_rademacher_field(uint64_t seed, uint32_t stream_id, uint64_t t, int64_t rows,
                            int64_t cols, float scale, int32_t transposed, float *out,
                            void *stream);

/* Count sketch S (rows x cols) of DSANLS_SKETCH_COUNT for side (0 or 1,
 * stream 0x30 | side) and iteration t: S[i][h(i)] = s(i), zero elsewhere.
 * transposed as above. */
int dsanls_count_field(uint64_t seed, uint32_t side, uint64_t t, int64_t rows, int64_t cols,
                       int32_t transposed, float *out, void *stream);

/* SRHT S (rows x cols) of DSANLS_SKETCH_SRHT for side (0 or 1) and iteration
 * t, times scale (1/sqrt(cols) gives the sketch itself, 1 the unit draws):
 * S[i][j] = D_i (-1)^popcount(i & J_j) scale.  Needs 1 <= cols <= p (rows
 * rounded up to a power of two) and rows <= 2^30; out is a device buffer of
 * rows x cols floats (cols x rows if transposed).  Allocates and frees its
 * own scratch (J and a p-bit bitmap) and synchronises the stream; EINVAL on
 * bad sizes, ENOMEM / ECUDA from the allocation or the launches. */
int dsanls_srht_field(uint64_t seed, uint32_t side, uint64_t t, int64_t rows, int64_t cols,
                      float scale, int32_t transposed, float *out, void *stream);

/* Uniform [0,1) field X[i][j] = (w >> 8) * 2^-24, row-major rows x cols. */
int dsanls_uniform_field(uint64_t seed, uint32_t stream_id, uint64_t t, int64_t rows,
                         int64_t cols, float *out, void *stream);

/* The d column indices of a subsampling sketch (Section 3.4: columns drawn
 * uniformly without replacement), ascending: {pi(0), ..., pi(d-1)} for the
 * 4-round Feistel permutation pi of {0..n-1} keyed by (seed, t, side) with
 * cycle walking.  1 <= d <= n. */
int dsanls_subsample_indices(uint64_t seed, uint32_t side, uint64_t t, int64_t n, int32_t d,
                             int32_t *J, void *stream);

/* ---- batched form: many independent dense problems ---------------------
 * A batch advances `count` independent problems M_i (m_i x n_i) ~ U_i V_i^T
 * together, each with its own rank k_i (1..32), sketch sizes d_i, d'_i and
 * Philox seed_i (Gaussian sketches; binary32 arithmetic).  Every phase of a
 * half-step is one persistent kernel that takes (instance, tile) work items
 * from a device queue; with use_graph each outer iteration is one CUDA graph
 * launch.  The first dsanls_batch_step times a few persistent launch
 * geometries on the real batch (factors and t are restored afterwards) and
 * keeps the fastest, cached per batch shape list and dtype in the process
 * and, when DSANLS_TUNE_CACHE names a file, across processes.  Default
 * factors are the Uniform[0,1) draws of streams 2 and 3 keyed by seed_i.
 * Instance i follows exactly the single-problem method of dsanls_create. */
typedef struct dsanls_batch_ctx *dsanls_batch_t;

/* Arrays of length count: m, n (1..2^24), k (1..32), d and d_v (1..2^20), seeds.
 * EINVAL, ENOMEM, ECUDA (message in dsanls_last_error(NULL)). */
int dsanls_batch_create(int32_t count, const int64_t *m, const int64_t *n, const int32_t *k,
                        const int32_t *d, const int32_t *d_v, const uint64_t *seeds,
                        dsanls_batch_t *out);
/* solver, alpha, beta, power_iters, t, use_graph, order, precision and stream
 * are used; precision FP32 or BF16 (M_i, S_i, Y_i, B_i and A_i or P_i rounded
 * to bf16 where they enter a product, fp32 accumulation, G_i in FP64 from the
 * unrounded B_i), inner_iters 1, bound_clamp 0, d_v ignored (given per
 * instance). */
int dsanls_batch_set_options(dsanls_batch_t b, const dsanls_options *opt);
/* Dense M_i (m_i x n_i, row stride ld); copied, with its transpose. Synchronises. */
int dsanls_batch_set_dense(dsanls_batch_t b, int32_t i, const float *M, int64_t ld, int32_t on_device);
int dsanls_batch_set_factors(dsanls_batch_t b, int32_t i, const float *U, const float *V, int32_t on_device);
/* outer_iters iterations of every instance; ESTATE until every M_i is set. */
int dsanls_batch_step(dsanls_batch_t b, int32_t outer_iters);
int dsanls_batch_get_factors(dsanls_batch_t b, int32_t i, float *U, float *V, int32_t on_device);
/* out[i] = ||M_i - U_i V_i^T||_F / ||M_i||_F for every instance (host array of count). */
int dsanls_batch_rel_error(dsanls_batch_t b, double *out);
/* Run both half-steps once (advancing the factors, not t) with CUDA events
 * around the five phases; ms[side*5 + p] = milliseconds of phase p (0 sketch,
 * 1 B = Y^T S, 2 R = (X S) B^T, 3 Gram and step size, 4 update).  Synchronises. */
int dsanls_batch_profile(dsanls_batch_t b, double *ms);
/* Persistent CTAs chosen by the autotuner (0 before the first step). */
int dsanls_batch_tuned_blocks(dsanls_batch_t b, int32_t *persistent_ctas);
/* BF16 paper order: R_i = (X_i S_i) B_i^T runs on tcgen05 tensor cores (one
 * persistent launch over (instance, row tiles) items, A_i kept on chip).  Each
 * half-step (side 0: U, side 1: V) has its own tile, chosen by the autotuner
 * from the time of that half-step's product: *chunk = sketch columns per chunk
 * (64, 128, 192 or 256; it sets the tile's shared memory and tensor-memory
 * columns and so its CTAs per SM), *ctas = persistent CTAs, *row_tiles = 128-row
 * tiles per work item (1, or 2 sharing every copy of the sketch chunk),
 * *pipeline = how the kernel is organised (0: every thread issues 16-byte
 * cp.async copies into the operand ring; 1: one thread feeds the ring by TMA
 * tile copies and another issues the products; 2: as 1 with two row tiles per
 * item, the ring kept full across chunks and items while warps 2-5 round each
 * D1 chunk to bf16 in tensor memory, the second product reads it there and its
 * chunk partials are summed in registers, so a chunk may be 256 wide); all
 * 0 before the first step or in the other forms.  row_tiles and pipeline may be
 * NULL; side must be 0 or 1. */
int dsanls_batch_tuned_tile(dsanls_batch_t b, int32_t side, int32_t *chunk, int32_t *ctas, int32_t *row_tiles,
                            int32_t *pipeline);
/* Pin the tile of the tensor-core product of one half-step (side 0 or 1) or of
 * both (side -1) instead of letting the autotuner time the candidates: pipeline
 * 0 or 1 with (chunk, stages, row_tiles) one of (64,4,1) (128,3,1) (128,4,1)
 * (256,4,1) (64,2,1) (64,4,2) (128,3,2) (128,4,2) (192,3,2) (64,2,2), or pipeline
 * 2 with (256,3,2) (192,3,2) (128,4,2) (64,5,2); (0,0,0,any) returns that side to the
 * autotuner.  Takes effect at the next step (the iteration graph is rebuilt);
 * other configurations return EINVAL and change nothing. */
int dsanls_batch_set_tile(dsanls_batch_t b, int32_t side, int32_t chunk, int32_t stages, int32_t row_tiles,
                          int32_t pipeline);
const char *dsanls_batch_last_error(dsanls_batch_t b);
void dsanls_batch_destroy(dsanls_batch_t b);

/* ---- learned warm start (k <= 32) ---------------------------------------
 * Learned form of a half-step: for each row, the proximal row problem
 *   f(x) = 1/2 x^T (G + mu_t I) x - (r + mu_t u)^T x,  x >= 0   (eq. reg_sub)
 * is started from a small MLP's prediction, corrected by pg_iters projected
 * gradient steps (step eta_t), and the plain projected-gradient step of
 * eq. gradient_descent is kept instead whenever its objective is lower.
 * Network: h1 = GELU(W1g vec(Gn) + W1b bn + b1), h2 = GELU(W2 h1 + b2),
 * y = ReLU(W3 h2 + b3) on the normalised inputs Gn = (G + mu I)/s,
 * s = tr(G + mu I)/k, bn = b/beta, beta = ||b||/sqrt(k); x0 = y beta/s.
 * Parameters (fp32 masters, used rounded to bf16; fp32 accumulation), in
 * order: W1g (h x k*k), W1b (h x k), b1 (h), W2 (h x h), b2 (h), W3 (k x h), b3 (k). */
typedef struct dsanls_mlp_ctx *dsanls_mlp_t;

/* k in [1, 32], hidden in [1, 256]; buffers for up to max_rows rows in
 * max_groups subproblems per call; weights U(-sqrt(3/fan_in), +) from Philox
 * stream 0x20 keyed by seed, biases 0. */
int dsanls_mlp_create(int32_t k, int32_t hidden, int64_t max_rows, int32_t max_groups, uint64_t seed,
                      dsanls_mlp_t *out);
int dsanls_mlp_param_count(dsanls_mlp_t m, int64_t *count);
int dsanls_mlp_get_params(dsanls_mlp_t m, float *theta);        /* host array of param_count */
int dsanls_mlp_set_params(dsanls_mlp_t m, const float *theta);  /* host array of param_count */
/* Device arrays: G (ngroups x k x k), mu (ngroups), group_off (ngroups + 1,
 * rows of group g are group_off[g] .. group_off[g+1]-1), b (rows x k, b = r + mu u).
 * x_out (rows x k) = the network's warm start in the original scale. */
int dsanls_mlp_predict(dsanls_mlp_t m, const float *G, const float *mu, const int64_t *group_off, int32_t ngroups,
                       const float *b, int64_t rows, float *x_out, void *stream);
/* Loss 1/2 mean ||y - y*||^2 against the normalised exact minimisers
 * y* = xstar s / beta, its gradient (host array, nullable) and, if lr > 0,
 * one Adam step (beta1 0.9, beta2 0.999, eps 1e-8).  Synchronises. */
int dsanls_mlp_train_step(dsanls_mlp_t m, const float *G, const float *mu, const int64_t *group_off,
                          int32_t ngroups, const float *b, const float *xstar, int64_t rows, float lr,
                          double *loss, float *grad, void *stream);
void dsanls_mlp_destroy(dsanls_mlp_t m);
/* Use network m (NULL: the plain solver) in the handle's half-steps; m must
 * outlive its use; needs k <= 32 and m's max_rows >= max(m, n). */
int dsanls_set_mlp(dsanls_t h, dsanls_mlp_t m, int32_t pg_iters);
/* Rows (cumulative) for which the learned point was kept.  Synchronises. */
int dsanls_mlp_kept(dsanls_t h, int64_t *kept);
/* Training triples of the current state, without updating it: runs the
 * sketched products of `side` at the current t and returns G (k x k, device
 * fp32), mu_t (device, 1), b = r + mu u (rows x k, device) and x* (rows x k,
 * device), the proximal minimiser by `iters` FISTA steps (Beck and Teboulle
 * 2009).  k <= 32.  Synchronises. */
int dsanls_harvest(dsanls_t h, int32_t side, int32_t iters, float *G, float *mu, float *b, float *xstar);

/* ---- allocation-free Gram ---------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot let a library allocate device memory -- a host framework that
 * owns all device memory through its own pool and forbids cudaMalloc/cudaFree
 * in plugins, or a latency-critical loop that cannot afford the implicit
 * device synchronisation of cudaFree.
 *
 * G (k x k, FP64, row-major, device) = B B^T for B (k x d, binary32,
 * row-major, device), the same kernels and arithmetic as the Gram of a
 * half-step.  It allocates nothing: its only scratch is a fixed 2 MiB
 * file-scope device array inside libdsanls.so (FP64 partial Grams of up to
 * floor(262144 / k^2) CTAs), which every GPU that loads the library holds
 * until the process exits.  The fixed size costs parallelism: the partial
 * Gram runs on at most floor(262144 / k^2) CTAs -- 16 at k = 128, 26 at
 * k = 100, 64 at k = 64 -- where the handle's Gram uses up to 304 (2 per SM),
 * so at large k and d it is several times slower; from k <= 29 on it gets
 * the full grid.  The first call on a device resolves that array's device
 * address (cudaGetSymbolAddress, with the device current); make that first
 * call before any stream capture -- a first call while `stream` is being
 * captured returns EINVAL and queues nothing.  All calls on a device share the
 * array: calls whose executions overlap on the GPU race and give wrong
 * results -- serialise them (one stream, or events).  Every partial a call
 * reads is written by the same call, so stale contents from an earlier call
 * never leak into G.  Queued on `stream` (cudaStream_t, NULL = default
 * stream); returns once queued.  EINVAL for NULL pointers, k outside
 * [1, 128] or d outside [1, 2^31 - 1] (message in dsanls_last_error(NULL));
 * ECUDA on a launch failure. */
int dsanls_gram_noalloc(const float *B, int32_t k, int64_t d, double *G, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DSANLS_H */
