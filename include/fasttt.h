/*
 * fasttt.h — C ABI of libfasttt.so, a GB300 (sm_103a) implementation of FastTT,
 * the sparse tensor-train decomposition of Li, Yu and Batselier ("Faster Tensor
 * Train Decomposition for Sparse Data").
 *
 * Conventions (Sec. 2 of the paper, 0-based here):
 *   - a d-way tensor A has mode sizes n_1..n_d; its COO input is an int32 index
 *     array of shape (d, nnz) in structure-of-arrays layout (mode k's indices are
 *     the contiguous row k: idx[k*nnz + e]) and nnz values;
 *   - TT core k (k = 1..d) is a row-major r_{k-1} x n_k x r_k array of doubles,
 *     r_0 = r_d = 1; entry a(i) = G_1[i_1] G_2[i_2] ... G_d[i_d] (Sec. 2.3);
 *   - the k-unfolding has rows (i_1..i_k) and columns (i_{k+1}..i_d), last index
 *     fastest (Sec. 2.2).
 *
 * Pointers named d_* are device pointers (cudaMalloc / torch CUDA memory) on the
 * current device; "host" pointers are ordinary host memory.  Every call runs its
 * work on the caller's CUDA stream (NULL = the legacy default stream) and returns
 * once its results are ready, unless stated otherwise.  No call falls back to
 * the CPU: without a usable CUDA device every entry point returns FASTTT_ECUDA.
 *
 * Errors: every int-returning call returns FASTTT_OK (0) or a negative code
 * below; fasttt_last_error() then gives a message (thread-local, valid until the
 * thread's next call).  No C++ exception crosses this boundary.
 */
#ifndef FASTTT_H
#define FASTTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FASTTT_MAX_D 64

/* return codes */
#define FASTTT_OK 0
#define FASTTT_EINVAL (-1)   /* bad argument: index out of range, NaN/Inf value, d < 2, no nonzero ... */
#define FASTTT_EDUP (-2)     /* the COO input repeats a coordinate */
#define FASTTT_ENOMEM (-3)   /* a device allocation failed */
#define FASTTT_ETIMEOUT (-4) /* an iteration hit its bound (Jacobi sweeps) */
#define FASTTT_ENUMERIC (-5) /* non-finite intermediate in the dense rounding */
#define FASTTT_ERANK (-6)    /* a dense intermediate would exceed the size limits */
#define FASTTT_ECUDA (-7)    /* a CUDA runtime call failed (message has the CUDA error) */

/* value / core dtypes */
#define FASTTT_F64 0
#define FASTTT_F32 1

/* fasttt_opts.precision */
#define FASTTT_PREC_FP64 0   /* every floating-point step in IEEE FP64 */
#define FASTTT_PREC_MIXED 1  /* chosen per bond of the Gram route: the Gram and the
                              * projection as FP32-level tensor-core products (3 exact bf16
                              * slices per operand; split TF32 for small products), the
                              * Gram's distance from the exact one probed, and the bond kept
                              * at that level only when every kept sigma^2 clears the error
                              * floor and the rank decision does not move within it; other
                              * bonds are redone with FP64-level products.  Factors
                              * re-orthonormalised by CholeskyQR with an FP64 Cholesky;
                              * eigenvalues, rank rule, norms and the direct-route SVDs in
                              * FP64.  FP32-level accuracy (~1e-6 relative) on the bonds kept
                              * at that level; the statistics count both kinds of bond. */

/* fasttt_opts.rounding */
#define FASTTT_STATIC 0      /* delta_k of eq. (11), Alg. 6 */
#define FASTTT_DYNAMIC 1     /* the re-spent error budget of Alg. 8 */

/* fasttt_opts.stage */
#define FASTTT_STAGE_FULL 0  /* Alg. 7: exact TT, then TT-rounding */
#define FASTTT_STAGE_EXACT 1 /* Alg. 4 only: the lossless exact sparse TT (no cores) */
#define FASTTT_STAGE_DEPAR 2 /* Alg. 4 and the value Depar of the middle unfolding (Alg. 3), no
                                rounding: the grouping and Depar factors of tensors whose exact
                                ranks are too large to round (intermediates always kept) */

typedef struct fasttt_opts {
  int p;              /* split point 1..d; 0 = choose by Alg. 9 (flop model, eq. (13)) */
  int precision;      /* FASTTT_PREC_FP64 or FASTTT_PREC_MIXED */
  int rounding;       /* FASTTT_STATIC or FASTTT_DYNAMIC */
  int depar_values;   /* 1: value Depar (Alg. 3, exact parallelism) of the middle unfolding; 0: off */
  int stage;          /* FASTTT_STAGE_FULL, FASTTT_STAGE_EXACT or FASTTT_STAGE_DEPAR */
  int keep_intermediates; /* 1: keep group maps, middle COO, Depar factors, singular values */
  int64_t max_rank;   /* > 0: cap every TT rank (fixed-rank variant, Sec. 3.4); 0: none */
  int64_t max_sweeps; /* Jacobi sweep bound of the dense SVDs; 0 = default (40) */
  int sparse_sweep;   /* first SVD sweep (Alg. 6) bonds: FASTTT_SWEEP_AUTO, _SPARSE or _DENSE */
  int gemm_engine;    /* FASTTT_GEMM_TENSOR (default) or FASTTT_GEMM_DFMA */
  int64_t max_spin;   /* polls of every device-side spin-wait (grid barriers, tensor-core
                         pipeline waits) before it gives up and the call fails with
                         FASTTT_ETIMEOUT; 0 = default (2^24 barrier polls, 2^22 pipeline polls) */
} fasttt_opts;

/* Engine of the dense FP64 contractions.  TENSOR: products of at least 2^22
 * multiply-adds (inner dimension 64 or more) run on the tcgen05 tensor cores from exact bf16 slices of the
 * FP64 operands (8 slices of 7 bits: every slice product exact, the level sums
 * exact in FP32 over windows of 384 and then in 64-bit integers; FP64-level
 * results, Ozaki-Ogita-Oishi-Rump splitting), smaller ones on FP64 DFMA.  DFMA:
 * every FP64 product on FP64 DFMA.  In mixed precision, TENSOR runs the large
 * products from 3 slices of 8 bits (FP32-level).  A tensor-core kernel whose
 * bounded wait gives up makes the call fail with FASTTT_ETIMEOUT. */
#define FASTTT_GEMM_TENSOR 0
#define FASTTT_GEMM_DFMA 1

/* How a bond k of the first SVD sweep sees G_k = W_{k-1} x_1 P_k (P_k the right
 * quasi-permutation core of Alg. 4).  DENSE: G_k is materialised (r_{k-1} x n_k x
 * r~_k) and its k-unfolding goes through the dense SVD.  SPARSE: G_k stays
 * implicit (W_{k-1} and the group maps); the Gram Z Z^T of Z = unfold_2(G_k)
 * ((r_{k-1} n_k)^2) and the projection U^T Z are formed from the nonzero blocks
 * only, which is what makes r~_k in the millions feasible.  AUTO: SPARSE when the
 * dense core would exceed 2 GiB and r_{k-1} n_k <= 16384, else DENSE.  SPARSE
 * requested where r_{k-1} n_k > 16384 falls back to DENSE. */
#define FASTTT_SWEEP_AUTO 0
#define FASTTT_SWEEP_SPARSE 1
#define FASTTT_SWEEP_DENSE 2

/* Fills *opts with the defaults: p = 0, FP64, static rounding, value Depar on,
 * full stage, no intermediates, no rank cap, default sweep bound, AUTO sweep. */
void fasttt_default_opts(fasttt_opts* opts);

typedef struct fasttt_stats {
  int d, p;
  int64_t nnz_in;            /* entries passed in */
  int64_t nnz;               /* entries kept (explicit zeros dropped) */
  int64_t dropped;           /* explicit zeros dropped */
  int64_t R;                 /* nonzero p-fibers (eq. (4)) at the chosen p */
  int64_t Rs[FASTTT_MAX_D];  /* R for every p = 1..d when Alg. 9 ran (index p-1), else 0 */
  int64_t rt[FASTTT_MAX_D + 1];    /* r~_k after Alg. 4 (k = 0..d) */
  int64_t ranks[FASTTT_MAX_D + 1]; /* r_k of the output (k = 0..d) */
  int64_t beta_r, beta_c;    /* row / column classes of the middle unfolding (value Depar) */
  int64_t jacobi_sweeps;     /* total Jacobi sweeps over all dense SVDs */
  int64_t launches;          /* CUDA kernels this call launched */
  int64_t jacobi_block_sweeps; /* Jacobi sweeps run on the shared-memory block schedule */
  int64_t coop_launch_error;   /* last error code of a refused cooperative launch (0: none) */
  double norm2;              /* ||A||_F^2 */
  double err2;               /* sum over truncations of the discarded sigma^2 (||E_k||_F^2) */
  double deltas[FASTTT_MAX_D + 1]; /* delta_k used at bond k (0 where unused) */
  double ms_ingest, ms_group, ms_depar, ms_round, ms_total; /* CUDA-event stage times */
  /* CUDA-event time and algorithmic work of the heavy kernel classes: FP64 GEMM
   * (2MNK flops), Jacobi sweeps (dot products + applied rotations, flops) and
   * radix-sort passes (key/value bytes moved) */
  double ms_gemm, flop_gemm, ms_jacobi, flop_jacobi, ms_sort, bytes_sort;
  double ms_jacobi32, flop_jacobi32; /* FP32 Jacobi sweeps (large eigenproblems) */
  double ms_gemm_tc, flop_gemm_tc;   /* split-TF32 tensor-core GEMMs (mixed precision) */
  int64_t sparse_bonds;      /* first-sweep bonds run block-sparse (FASTTT_SWEEP_SPARSE path) */
  double ms_tridiag, flop_tridiag; /* Householder tridiagonalisation of Gram matrices (2 n^3 flops) */
  double ms_tdeig;           /* bisection + inverse iteration on the tridiagonal matrices */
  int64_t eig_tridiag;       /* Gram eigenproblems solved by the FP64 tridiagonal route */
  int64_t eig_fallbacks;     /* Gram eigenproblems handed to the iterative (Jacobi) eigensolver */
  double ms_gemm_oz, flop_gemm_oz; /* tcgen05 GEMMs on exact bf16 slices (2MNK flops of the FP64 product) */
  double ms_tridiag32, flop_tridiag32; /* FP32 tridiagonalisation of the fast eigensolver's start (2 n^3 flops) */
  double ms_tsqr, flop_tsqr;  /* Householder TSQR of tall-skinny SVDs and its Q application (4 m n^2 flops each) */
  int64_t eig_fast;           /* Gram eigenproblems solved by the fast route (FP32 start + refinement) */
  int64_t qr_cholqr2;         /* QR steps of Alg. 6's right-to-left sweep done by CholeskyQR2 */
  int64_t qr_svd;             /* QR steps that fell back to an untruncated SVD (CholeskyQR2 broke down) */
  int64_t mixed_fp32_bonds;   /* mixed precision: Gram-route SVDs whose FP32-level result was kept */
  int64_t mixed_fp64_bonds;   /* mixed precision: Gram-route SVDs redone with FP64-level products */
  int64_t wait_timeouts;      /* device spin-waits of this call that gave up (see max_spin) */
} fasttt_stats;

typedef struct fasttt_tt fasttt_tt; /* opaque result handle */

/*
 * fasttt_decompose — Alg. 7 (FastTT): Alg. 4 with Alg. 5 (exact grouping of the
 * sparse unfoldings into quasi-permutation cores, Sec. 3.1-3.2), value Depar of
 * the middle unfolding (Alg. 3 with exact parallelism), then Alg. 6 (or Alg. 8)
 * TT-rounding to relative accuracy eps (Sec. 3.3-3.5).
 *
 *  d, dims      order d (2..FASTTT_MAX_D) and host array of the d mode sizes (>= 1);
 *  nnz, d_idx   number of COO entries and their (d, nnz) int32 indices, 0-based;
 *  d_vals       nnz values, FASTTT_F64 or FASTTT_F32 (upcast exactly to FP64);
 *  eps          relative accuracy (>= 0); eps = 0 keeps the numerical ranks
 *               (sigma_i > max(M,N) 2^-52 sigma_1, M x N the unfolding's size);
 *  opts         NULL for the defaults;
 *  stream       cudaStream_t (NULL = default stream);
 *  out          receives a handle owned by the caller (free with fasttt_tt_free);
 *  stats        optional (may be NULL), filled on success and, as far as known,
 *               on failure.
 * Inputs are borrowed and only read; they must stay valid until the call returns.
 * Errors: EINVAL (bad sizes, index out of range, NaN/Inf, all-zero tensor),
 * EDUP (repeated coordinate), ENOMEM, ERANK, ETIMEOUT, ENUMERIC, ECUDA.
 */
int fasttt_decompose(int d, const int64_t* dims, int64_t nnz, const int32_t* d_idx,
                     const void* d_vals, int val_dtype, double eps, const fasttt_opts* opts,
                     void* stream, fasttt_tt** out, fasttt_stats* stats);

/* Releases a handle and all device memory it owns (NULL is a no-op). */
void fasttt_tt_free(fasttt_tt* tt);

/* Copies the handle's statistics into *stats. */
int fasttt_tt_stats(const fasttt_tt* tt, fasttt_stats* stats);

/* Copies the d+1 TT ranks r_0..r_d into the host array ranks. */
int fasttt_tt_ranks(const fasttt_tt* tt, int64_t* ranks);

/* Borrowed device pointer to core k (1..d), r_{k-1} x n_k x r_k FP64 row-major;
 * valid until fasttt_tt_free. */
int fasttt_tt_core(const fasttt_tt* tt, int k, const double** d_core);

/*
 * fasttt_tt_round — Alg. 2 (TT-rounding of a TT given by its cores, Section 2.4):
 * right-to-left orthogonalisation (core k's 1-unfolding factored by an
 * untruncated SVD standing in for the QR factorisation, the orthonormal factor
 * staying in core k and the rest multiplied into core k-1), then
 * ||A||_F = ||G_1||_F, delta = eps ||A||_F / sqrt(d-1) and left-to-right
 * delta-truncated SVDs of the 2-unfoldings, S V^T multiplied into the next core.
 *
 *  d, dims, ranks  order (1..FASTTT_MAX_D), host arrays of the d mode sizes and the
 *                  d+1 ranks (r_0 = r_d = 1);
 *  d_cores         host array of d device pointers, core k r_{k-1} x n_k x r_k FP64
 *                  row-major (borrowed, only read; a handle's cores may be passed);
 *  eps             relative accuracy (>= 0; 0 keeps the numerical ranks of the
 *                  unfoldings, as fasttt_decompose);
 *  opts            NULL for the defaults; read: precision, max_rank, max_sweeps,
 *                  gemm_engine, keep_intermediates (singular values per bond);
 *                  rounding must be FASTTT_STATIC;
 *  out, stats      as fasttt_decompose (stats: ranks, norm2 = ||A||^2, err2 = the
 *                  discarded sigma^2 summed over the bonds, deltas, stage times).
 * Errors: EINVAL (bad sizes or ranks, null pointers, dynamic rounding), ENOMEM,
 * ERANK, ETIMEOUT, ENUMERIC, ECUDA.
 */
int fasttt_tt_round(int d, const int64_t* dims, const int64_t* ranks, const double* const* d_cores,
                    double eps, const fasttt_opts* opts, void* stream, fasttt_tt** out,
                    fasttt_stats* stats);

/*
 * fasttt_tt_add — the TT of A + beta B (Lemma 2, eq. (6)) from the cores of two TTs
 * with the same mode sizes: core 1 = [A_1, beta B_1], core d = [A_d; B_d], the cores
 * in between block diagonal (d = 1: A_1 + beta B_1); ranks r_k^A + r_k^B.  Arguments
 * as fasttt_tt_round (cores borrowed and only read); out receives a new handle whose
 * stats hold d and the ranks only.  Round the sum with fasttt_tt_round.
 * Errors: EINVAL, ENOMEM, ERANK, ECUDA.
 */
int fasttt_tt_add(int d, const int64_t* dims, const int64_t* ranks_a, const double* const* d_cores_a,
                  const int64_t* ranks_b, const double* const* d_cores_b, double beta, void* stream,
                  fasttt_tt** out);

/* Arrays a handle can hand out with fasttt_tt_count / fasttt_tt_copy.  k is the
 * core index (1..d) or the bond index where noted; ignored otherwise. */
#define FASTTT_ARR_CORE 0        /* f64, core k (r_{k-1} n_k r_k) */
#define FASTTT_ARR_LEFT_PARENT 1 /* i32, core k < p: alpha_{k-1} of every alpha_k (r~_k) */
#define FASTTT_ARR_LEFT_INDEX 2  /* i32, core k < p: i_k of every alpha_k (r~_k) */
#define FASTTT_ARR_RIGHT_INDEX 3 /* i32, core k > p: i_k of every alpha_{k-1} (r~_{k-1}) */
#define FASTTT_ARR_RIGHT_CHILD 4 /* i32, core k > p: alpha_k of every alpha_{k-1} (r~_{k-1}) */
#define FASTTT_ARR_MID_ROW 5     /* i64, middle unfolding X entries sorted by (row, col) */
#define FASTTT_ARR_MID_COL 6     /* i64 */
#define FASTTT_ARR_MID_VAL 7     /* f64 */
#define FASTTT_ARR_ROW_ID 8      /* i64, nonzero rows of X ascending */
#define FASTTT_ARR_ROW_CLASS 9   /* i32, value-Depar class of each nonzero row */
#define FASTTT_ARR_ROW_PREF 10   /* f64, prefactor (first nonzero) of each nonzero row */
#define FASTTT_ARR_COL_ID 11     /* i64, nonzero columns of X ascending */
#define FASTTT_ARR_COL_CLASS 12  /* i32 */
#define FASTTT_ARR_COL_PREF 13   /* f64 */
#define FASTTT_ARR_DP_ROW 14     /* i32, entries of D' (beta_r x beta_c) sorted by (row, col) */
#define FASTTT_ARR_DP_COL 15     /* i32 */
#define FASTTT_ARR_DP_VAL 16     /* f64 */
#define FASTTT_ARR_LAM_S 17      /* f64, Lambda_S (beta_r) */
#define FASTTT_ARR_LAM_T 18      /* f64, Lambda_T (beta_c) */
#define FASTTT_ARR_SIGMA 19      /* f64, singular values computed at bond k, descending */

/* Number of elements of array `what` (>= 0), or a negative error code
 * (EINVAL when the array does not exist, e.g. intermediates were not kept). */
int64_t fasttt_tt_count(const fasttt_tt* tt, int what, int k);

/* Copies `count` elements of array `what` into dst (host or device memory;
 * count must equal fasttt_tt_count). */
int fasttt_tt_copy(const fasttt_tt* tt, int what, int k, void* dst, int64_t count);

/*
 * tt_eval_at — entry evaluation (Sec. 2.3): out[e] = G_1[i_1^e] ... G_d[i_d^e]
 * for m index tuples.
 *  d, dims, ranks   host arrays: d mode sizes, d+1 ranks (r_0 = r_d = 1);
 *  d_cores          host array of d device pointers, core k row-major r_{k-1} x n_k x r_k;
 *  dtype            FASTTT_F64 or FASTTT_F32 (cores and output alike);
 *  m, d_idx         (d, m) int32 indices, structure-of-arrays, 0-based;
 *  d_out            m outputs.
 * Ranks up to 8192 are supported (ERANK beyond).  Indices are range-checked on the
 * device; a bad index makes the call return EINVAL (outputs then unspecified).
 */
int tt_eval_at(int d, const int64_t* dims, const int64_t* ranks, const void* const* d_cores,
               int dtype, int64_t m, const int32_t* d_idx, void* d_out, void* stream);

/*
 * tt_eval_backward — adjoint of tt_eval_at: for L = sum_e g_e a(i^e),
 *   dL/dG_k[i] = sum_{e: i_k^e = i} g_e L_{k-1}(e)^T R_{k+1}(e),
 * L/R the left/right partial products of the chain.  d_grad_cores is a host
 * array of d device pointers shaped like the cores; gradients are ADDED to them
 * (zero them first for a plain gradient).  recompute = 1 recomputes the right
 * partial products per mode instead of storing all of them
 * (O(m * max r) scratch instead of O(m * sum r)).
 */
int tt_eval_backward(int d, const int64_t* dims, const int64_t* ranks,
                     const void* const* d_cores, int dtype, int64_t m, const int32_t* d_idx,
                     const void* d_grad_out, void* const* d_grad_cores, int recompute,
                     void* stream);

/*
 * tt_eval_backward_noalloc — for callers that cannot call cudaMalloc (or any
 * allocator) on the device: for example a host framework that owns all device
 * memory through its own pool, or an embedded runtime with a fixed memory budget.
 * The paper has no counterpart; this is a library-level service.
 * Same arguments and result as tt_eval_backward with recompute = 0 (gradients
 * ADDED into d_grad_cores, which the caller allocates at the cores' shapes and
 * dtype).  Its scratch is a file-scope device array of
 * FASTTT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits; the call allocates nothing.  Every call looks up that
 * array's device address with the caller's device current.  The call reads the
 * kernel's error flag back, so it synchronises the stream before returning.  All
 * calls share the one array, so calls that overlap on the GPU (other streams,
 * other threads) race: serialise them.  The scratch holds, per resident warp, the
 * left partial products (r_0 + ... + r_{d-1} values of the cores' dtype) after a
 * 256-byte error word; the grid is limited to the warps that fit, and a call is
 * rejected with FASTTT_ERANK only when not even one thread block's warps fit.
 * Within this library's limits (d <= 64, ranks <= 8192, so
 * r_0 + ... + r_{d-1} <= 516,097) one block always fits, so large rank sums only
 * lower the number of warps at work.  Other errors as tt_eval_backward.
 */
#define FASTTT_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int tt_eval_backward_noalloc(int d, const int64_t* dims, const int64_t* ranks,
                             const void* const* d_cores, int dtype, int64_t m, const int32_t* d_idx,
                             const void* d_grad_out, void* const* d_grad_cores, void* stream);

/*
 * tt_fit_gd — fixed-rank fitting of a TT to given entries (the tensor-completion
 * use of fixed-rank TT approximations, Sec. 3.4) by plain gradient descent with
 * the adjoint of the entry formula (Sec. 2.3).  Each step evaluates the residual
 * r_e = a(i^e) - v_e, takes the gradient of L = 1/2 sum_e r_e^2 (the adjoint with
 * upstream weights r_e) and moves every core from the same point:
 * G_k <- G_k - lr dL/dG_k (product and difference rounded separately).
 *  d, dims, ranks, dtype  as tt_eval_at; the ranks stay fixed;
 *  d_cores                host array of d device pointers, UPDATED IN PLACE;
 *  m, d_idx, d_vals       the m entries: (d, m) int32 indices (0-based, SoA) and
 *                         their values in the cores' dtype;
 *  steps, lr              number of steps (>= 0) and the step length;
 *  h_losses               host array of steps + 1 doubles: L before every step
 *                         and after the last (FP64 sums of the squared residuals).
 * Scratch (residuals, one gradient per core, the adjoint's partials) is allocated
 * on the device for the call.  Synchronous with respect to the host.
 * Errors: EINVAL (bad sizes, null pointers, negative steps, non-finite lr, an index
 * out of range), ERANK, ENOMEM, ECUDA.
 */
int tt_fit_gd(int d, const int64_t* dims, const int64_t* ranks, void* const* d_cores, int dtype,
              int64_t m, const int32_t* d_idx, const void* d_vals, int64_t steps, double lr,
              double* h_losses, void* stream);

/* Message of the calling thread's last error ("" if none). */
const char* fasttt_last_error(void);

/* Library version string. */
const char* fasttt_version(void);

/* Host-only test hooks (no device work; callable without a GPU).
 * fasttt_debug_select_p: the split index p of Alg. 9 that fasttt_decompose takes for
 * mode sizes dims (d of them) and the nonzero p-fiber counts Rs[p-1] (eq. (4)): the
 * argmin over p of eq. (13) with the bounds of eq. (10) (r capped at max_rank when
 * > 0), exact in 128-bit integers (saturating at 2^128 - 1), ties to the smallest p.
 * Returns p in 1..d, or EINVAL (d outside 2..FASTTT_MAX_D, a size or R outside
 * 1..2^31-1, max_rank < 0).
 * fasttt_debug_rank_rule: the rank r_k the rounding takes at bond `bond` (1..d-1)
 * from the n singular values h_sigma (descending, host): eps_zero = 0: the smallest
 * r >= 1 whose tail sqrt(sum_{i>r} sigma_i^2) (summed from the smallest up) is <= delta;
 * eps_zero = 1: the count of sigma_i > max(M,N) 2^-52 sigma_1 with M x N the size of
 * the bond's unfolding of the d-way tensor (at least 1); then min(r, max_rank) when
 * max_rank > 0.  Returns r, or EINVAL. */
int fasttt_debug_select_p(int d, const int64_t* dims, const int64_t* Rs, int64_t max_rank);
int64_t fasttt_debug_rank_rule(const double* h_sigma, int64_t n, double delta, int eps_zero, int d,
                               const int64_t* dims, int bond, int64_t max_rank);

/* Test hook for the host-side failure paths: the n-th device allocation from now
 * (n >= 1) fails with ENOMEM; n = 0 disables it.  Affects the calling process. */
void fasttt_debug_fail_alloc_after(int64_t n);

/* Test hook for the dense eigensolver of the rounding SVDs (the paper has no
 * counterpart; it exposes the Gram eigendecomposition of S7-S10 so that it can
 * be checked on matrices with chosen spectra).  d_G: symmetric n x n FP64,
 * row-major, device, read only.  d_V: n x n device output, eigenvector j in
 * d_V[j*n .. j*n + n).  h_lam: n host doubles, eigenvalue j (unordered).
 * method 0: FP64 Householder tridiagonalisation + bisection + inverse
 * iteration only (FASTTT_ENUMERIC when that route declines); 1: FP32 Jacobi
 * start + Ogita-Aishima refinement + FP64 Jacobi polish only; 2: 3, else 0,
 * else 1 (what the library uses); 3: the fast route only (FP32 tridiagonal
 * start, Ogita-Aishima refinement with FP64-level tensor-core products,
 * Rayleigh-Ritz on runs of close eigenvalues; FASTTT_ENUMERIC when it
 * declines).  stream: cudaStream_t or NULL; returns after synchronising it. */
int fasttt_debug_sym_eig(const double* d_G, int64_t n, double* d_V, double* h_lam, int method, void* stream);

/* Test hook for the GEMM engines (the paper has no counterpart): C = A B with
 * A (M x K), B (K x N), C (M x N) row-major FP64 device arrays.  engine 0: FP64
 * DFMA; 1: tcgen05 on 7 exact bf16 slices (FP64-level); 2: tcgen05 on 3 slices
 * (FP32-level); 3: split-TF32 mma.sync (FP32-level).  FASTTT_ENUMERIC when the
 * tensor-core kernel declined or gave up.  Synchronises the stream. */
int fasttt_debug_gemm(int64_t M, int64_t N, int64_t K, const double* d_A, const double* d_B, double* d_C, int engine,
                      void* stream);

/* Test hook for CholeskyQR2 (the QR factorisation of Alg. 6's right-to-left
 * sweep, and the re-orthonormalisation of the mixed precision; the paper names
 * a QR factorisation only).  d_Z: M x N FP64 row-major device array, M <= N,
 * overwritten by Q (orthonormal rows); d_R: M x M device array (caller-allocated)
 * receives the upper triangular R with Z = R^T Q.  precision FASTTT_PREC_MIXED:
 * the Grams and the solve updates are FP32-level products (the Cholesky
 * factorisations stay FP64).  FASTTT_ENUMERIC when a Cholesky factorisation
 * breaks down or the second Gram is further than 0.5 from I (Z too ill
 * conditioned for the Gram's precision); FASTTT_EINVAL for bad arguments.
 * Synchronises the stream. */
int fasttt_debug_cholqr(int64_t M, int64_t N, double* d_Z, double* d_R, int precision, void* stream);

/* Test hook for the dense SVD of the rounding sweeps (the paper has no
 * counterpart; it exposes the SVD behind S7-S10 so that it can be checked on
 * matrices with chosen singular values).  d_Z: M x N FP64, row-major, device,
 * read only.  All min(M, N) singular values are kept: h_sigma receives them
 * (host, descending), d_U (M x r row-major) and d_Vt (r x N row-major, device,
 * caller-allocated, r = min(M, N)) the factors with Z = U diag(sigma) Vt.
 * precision: FASTTT_PREC_FP64 or FASTTT_PREC_MIXED.  The route is the library's
 * (one-sided Jacobi, through TSQR for tall-skinny shapes, or the Gram route).
 * FASTTT_EINVAL for bad arguments.  Synchronises the stream. */
int fasttt_debug_svd(int64_t M, int64_t N, const double* d_Z, double* h_sigma, double* d_U, double* d_Vt,
                     int precision, void* stream);

/* Test hook for the symmetric (Gram) products of the rounding stage: C = A A^T
 * (M x M, row-major) for a row-major M x K device matrix A, through the same
 * engines as fasttt_debug_gemm (0..3) on their symmetric path: only the tiles
 * on or above the diagonal are computed and mirrored, and the tensor-core
 * engines split A once for both operands.  Caller-owned device buffers;
 * FASTTT_EINVAL for bad arguments, FASTTT_ENUMERIC when a tensor-core kernel
 * declined or gave up.  Synchronises the stream. */
int fasttt_debug_gram(int64_t M, int64_t K, const double* d_A, double* d_C, int engine, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FASTTT_H */
