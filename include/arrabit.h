/*
 * arrabit.h - C ABI of a GB300 (sm_103a) implementation of the subspace-update +
 * augmented Rayleigh-Ritz hot path of ARRABIT (Wen & Zhang, "Block algorithms with
 * augmented Rayleigh-Ritz projections for large-scale eigenpair computation",
 * arXiv 1507.06078).
 *
 * Problem statement (Section 1; Section 2 "our task is to compute k largest
 * eigenpairs"): given a sparse symmetric A in R^{n x n}, an integer k and a tolerance,
 * return (Lambda_k, Q_k) with A Q_k = Q_k Lambda_k and Q_k^T Q_k = I for the k
 * algebraically largest, or (by running on sigma I - A) smallest, eigenvalues.
 *
 * Conventions for every call:
 *  - Return value: an arb_status.  Nothing aborts, traps or exits; a failing CUDA call
 *    returns ARB_CUDA_ERROR and arb_last_error() describes it.
 *  - Dense blocks ("multivectors") on the device are ROW-MAJOR n x ncols float64 with a
 *    leading dimension ld >= ncols counted in elements (row i starts at ptr + i*ld).
 *  - Device pointers must point into memory of the context's device; "host" pointers
 *    are ordinary (preferably pinned) host memory.
 *  - The caller owns every buffer it passes; the library owns its workspaces (allocated
 *    per context on first use and kept until arb_ctx_destroy).
 *  - All device work runs on the context's stream.  Calls that return host values
 *    synchronise that stream; the others are asynchronous with respect to the host.
 *  - One context per host thread at a time; contexts are not thread-safe.
 */
#ifndef ARRABIT_H
#define ARRABIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct arb_ctx_s* arb_ctx;
typedef struct arb_mat_s* arb_mat;

typedef enum {
  ARB_OK = 0,
  ARB_NOT_CONVERGED = 1,  /* outputs hold the best pairs found; info->maxres says how good */
  ARB_INVALID_ARG = -1,
  ARB_OUT_OF_MEMORY = -2,
  ARB_NOT_SYMMETRIC = -3,
  ARB_BREAKDOWN = -4,     /* the iterate lost all numerical rank */
  ARB_CUDA_ERROR = -5,
  ARB_TIMEOUT = -6,
  ARB_REJECTED = -7
} arb_status;

typedef enum { ARB_LARGEST = 0, ARB_SMALLEST = 1 } arb_which;
/* ARB_FP64: every step in FP64.  ARB_MIXED: an FP32 phase (FP32 blocks, filter and Gram
 * runs), then FP64 refinement.  ARB_MIXED_DF: as ARB_MIXED, but the refinement's filter
 * (Algorithm 8's multi-power steps) runs in double-float arithmetic (hi + lo FP32 pairs,
 * about 44 significant bits) on the FP32 pipe; its Rayleigh-Ritz steps stay in FP64.  The
 * paper runs one precision throughout; the FP32 and double-float variants are this
 * library's. */
typedef enum { ARB_FP64 = 0, ARB_MIXED = 1, ARB_MIXED_DF = 2 } arb_precision;
/* Section 5: Chebyshev interpolant of max(0,t)^(10d) (the paper's choice) or the
 * classic Chebyshev polynomial T_d (eq. cheby-poly, the paper's comparison filter). */
typedef enum { ARB_FILTER_CHEBINTERP = 0, ARB_FILTER_CHEBYSHEV = 1 } arb_filter_kind;

/* Why the outer loop of Algorithm 8 ended (Section 5, "Outer loop stop rule"). */
typedef enum {
  ARB_STOP_CONVERGED = 0, /* maxres <= tol (eq. out-stop) */
  ARB_STOP_NEAR_TOL = 1,  /* case (iii): maxres < (1 + 9h/k) tol */
  ARB_STOP_STALLED = 2,   /* case (ii): no maxres decrease for 3 outer iterations */
  ARB_STOP_MAXIT = 3,     /* case (i) */
  ARB_STOP_ALL_LOCKED = 4
} arb_stop_reason;

/* Solver parameters (Section 5 and Algorithm 8).  Names follow the paper except that the
 * block width k+q is called p here and the paper's augmentation count p is called q. */
typedef struct {
  int32_t p;            /* block width = k + guard vectors (Section 5 "Guard vectors"); 0: k + round(0.1 k) */
  int32_t q;            /* augmentation blocks in [X, AX, ..., A^q X] (Alg. 5; default 1) */
  int32_t degree;       /* polynomial degree d (Section 5; default 3) */
  int32_t maxit;        /* outer iterations (default 30) */
  int32_t maxit1;       /* inner stop-rule checks per outer iteration (default 10) */
  int32_t maxit2;       /* filter applications between checks (default 5) */
  int32_t inner_fixed;  /* > 0: exactly this many filters per outer iteration, no rcond rule */
  int32_t filter;       /* arb_filter_kind */
  int32_t precision;    /* arb_precision: ARB_FP64, or ARB_MIXED (FP32 phase, then FP64 refinement) */
  int32_t b_update;     /* when the filter interval end b = mu_{k+q} is refreshed:
                           0 = at continuation steps only (Algorithm 8, the default);
                           1 = after every ARR projection (Section 5's estimation paragraph) */
  double tol1;          /* first continuation tolerance; 0: max(1e-6, tol) if tol <= 1e-8 else tol */
  double shift_sigma;   /* sigma of sigma I - A for ARB_SMALLEST; NaN: Gershgorin upper bound of A */
  double tol_switch;    /* ARB_MIXED: relative residual at which the FP32 phase hands over to
                           FP64 (never below 32 u32 ||A||, the FP32 floor); 0: 1e-5.  The FP32
                           phase also ends when an outer iteration fails to halve maxres.  The
                           FP64 phase starts from the FP32 Ritz block with b = mu_{k+q}. */
  uint64_t seed;        /* stream for padding columns (Philox4x32-10 + Box-Muller) */
  int32_t inner;        /* arb_inner_solver: ARB_INNER_MPM (default) or ARB_INNER_GN (Algorithm 8's branches) */
  int32_t adapt;        /* bit 0 (ARB_ADAPT_Q): raise q by one after an ARR when eq. block holds, up to
                           q_max; bit 1 (ARB_ADAPT_DEGREE): set the degree after every ARR by eqs. hat-d
                           and degree, up to d_max; q and degree are then the initial values */
  int32_t q_max;        /* cap of the adaptive q (0: 3, Section 5), also capped so that (q+1) p < n */
  int32_t d_max;        /* cap of the adaptive degree (0: 15, Section 5) */
} arb_options;

/* Inner solver of Algorithm 8: the multi-power method (Section 3) or Gauss-Newton
 * (Algorithm 4, Section 2.5). */
typedef enum { ARB_INNER_MPM = 0, ARB_INNER_GN = 1 } arb_inner_solver;
enum { ARB_ADAPT_Q = 1, ARB_ADAPT_DEGREE = 2 };

typedef struct {
  double maxres;        /* max_{i<=k} res_i, eq. resi */
  double a, b0, b_final;/* filter interval ends: a, the first and the last b (Section 5) */
  double sigma;         /* shift used for ARB_SMALLEST (0 for ARB_LARGEST) */
  double t_total, t_filter, t_arr; /* seconds spent in the call / inner loops / ARR steps */
  int64_t spmm_cols;    /* SpMV-equivalents: sum of block widths over all products with A */
  int32_t outer_iters;
  int32_t n_filters;    /* filter applications, all outer iterations */
  int32_t n_locked;     /* size of the locked set at exit */
  int32_t stop_reason;  /* arb_stop_reason */
  int32_t last_rank;    /* dimension of the last Rayleigh-Ritz subspace */
  int32_t outer_iters_fp32; /* ARB_MIXED: outer iterations of the FP32 phase */
  int32_t max_locked;   /* largest locked set of any outer iteration (eq. defl) */
  int32_t final_q;      /* augmentation blocks of the last ARR (differs from opts->q with ARB_ADAPT_Q) */
  int32_t final_d;      /* polynomial degree at exit (differs from opts->degree with ARB_ADAPT_DEGREE) */
  int32_t reserved0;
} arb_info;

/* ---------------------------------------------------------------- context, matrices */

/* Create a context on CUDA device `device`.  `cuda_stream` is the cudaStream_t all of the
 * context's device work runs on; NULL means the legacy default stream. */
arb_status arb_ctx_create(arb_ctx* out, int device, void* cuda_stream);
arb_status arb_ctx_destroy(arb_ctx ctx);

/* Dense arithmetic of a context: with enable != 0, its FP64 Gram products and tall-skinny
 * products (arb_gram, arb_orth, arb_rcond_gram, arb_rayleigh_ritz, arb_arr and the same
 * steps inside arb_solve) take FP64 operands, split them into hi + lo FP32 pairs and
 * multiply-add in double-float arithmetic on the FP32 pipe (compensated Dot2 sums, about
 * 2^-44 relative per term), returning FP64; the Jacobi eigensolver (arb_syevj and the
 * same step inside those calls) then runs orders above 32 in double-float arithmetic too
 * and stops at off(H) <= 1e-13 ||H||_F.  Off by default (plain FP64).  ARB_MIXED_DF
 * solves switch it on for their refinement phase and restore the setting afterwards.  The
 * paper computes in FP64 throughout; this mode is the library's.  Errors:
 * ARB_INVALID_ARG for a NULL context. */
arb_status arb_ctx_set_dense_df(arb_ctx ctx, int enable);
/* Description of the last error seen by this context (static storage, never NULL). */
const char* arb_last_error(arb_ctx ctx);
const char* arb_status_string(arb_status s);
/* Number of kernels this context has launched since it was created. */
int64_t arb_kernel_launches(arb_ctx ctx);

/* Defaults of Section 5 for k wanted pairs: p = k + round(0.1 k), q = 1, d = 3,
 * maxit = 30, maxit1 = 10, maxit2 = 5. */
void arb_options_default(arb_options* opts, int32_t k);

/* Copy a symmetric matrix in CSR form into library-owned device memory.
 * rowptr: int32[n+1] (rowptr[0] = 0, nondecreasing, rowptr[n] = nnz); col: int32[nnz]
 * with 0 <= col < n; val: float64[nnz].  ptr_on_device != 0 means the three arrays are
 * device pointers, else host pointers.  Symmetry is the caller's promise (it is not
 * checked); rowptr/col ranges are checked for host inputs -> ARB_INVALID_ARG. */
arb_status arb_matrix_create_csr(arb_ctx ctx, int64_t n, int64_t nnz, const int32_t* rowptr,
                                 const int32_t* col, const double* val, int ptr_on_device,
                                 arb_mat* out);
/* The same with FP32 values (val: float32[nnz], host or device as ptr_on_device): they are
 * widened to FP64 on the device and also kept as the FP32 copy the mixed paths use. */
arb_status arb_matrix_create_csr_f32(arb_ctx ctx, int64_t n, int64_t nnz, const int32_t* rowptr,
                                     const int32_t* col, const float* val, int ptr_on_device,
                                     arb_mat* out);
/* Host-side symmetry check of CSR arrays (host pointers): ARB_OK when every stored a_ij
 * (duplicates summed) matches a_ji to rel_tol * max|a|, ARB_NOT_SYMMETRIC otherwise,
 * ARB_INVALID_ARG for malformed arrays.  The method assumes symmetry (Section 1); the
 * matrix-creation calls take it as the caller's promise, this checks it. */
arb_status arb_csr_check_symmetric(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                                   const double* val, double rel_tol);
arb_status arb_matrix_destroy(arb_mat mat);

/* SELL-C-sigma layout (Kreutzer, Hager, Wellein, Fehske & Bishop, SIAM J. Sci. Comput. 2014)
 * of a CSR pattern, computed on the host (no device, no context).
 * Rows are sorted by decreasing nonzero count within each window of sigma consecutive rows
 * (ties: lower row first).  The sorted rows are cut into chunks of C, and each chunk is
 * stored column-major with the width of its longest row: slot cptr[c] + j*C + r holds
 * nonzero j of the chunk's row r.
 * Inputs: rowptr int32[n+1] (rowptr[0] = 0, nondecreasing); C >= 1; sigma >= 1.
 * Outputs (caller-owned host arrays):
 *  - perm int32[n]: the original row at each sorted position;
 *  - len int32[n]: its nonzero count;
 *  - cptr int64[ceil(n/C) + 1]: the first slot of each chunk;
 *  - *slots: the slot count, cptr's last entry;
 *  - src int64[slots], if non-NULL: the CSR index stored in each slot, -1 for padding.
 * Errors: ARB_INVALID_ARG for bad arguments, a bad rowptr, or src_capacity < *slots.  In
 * the last case *slots is still set, so a first call with src = NULL sizes src. */
arb_status arb_sell_layout(int64_t n, const int32_t* rowptr, int32_t C, int32_t sigma,
                           int32_t* perm, int32_t* len, int64_t* cptr, int64_t* src,
                           int64_t src_capacity, int64_t* slots);
/* Give a matrix a SELL-C-sigma copy (the layout above, built from its CSR arrays).  From
 * then on every SpMM of the filter, augmentation, Rayleigh-Ritz and residual steps reads it.
 * This covers FP64, FP32 and double-float values, all made now.
 * Rows are processed in sorted order and written to their original block rows. Each row's
 * nonzeros are summed in CSR order, so results equal the CSR path's. The one exception is
 * the column reductions, which sum rows in another order.
 * C = 0 drops the copy (CSR again). 1 <= C <= 1024 and sigma >= 1 otherwise; C = 32 with
 * sigma a multiple of it is the usual choice.
 * Not to be called while other calls use the matrix.  The CSR arrays are kept.
 * Errors: ARB_INVALID_ARG, ARB_CUDA_ERROR (the matrix is then back on CSR). */
arb_status arb_matrix_set_sell(arb_ctx ctx, arb_mat mat, int32_t C, int32_t sigma);
/* The matrix's SELL parameters and slot count (0, 0, 0: CSR only). */
arb_status arb_matrix_sell_info(arb_mat mat, int32_t* C, int32_t* sigma, int64_t* slots);
/* Gershgorin interval [lo, hi] of A (host outputs); stands in for the paper's eigs
 * estimate of lambda_n (Section 5, "Estimation of lambda_n and lambda_{k+q}"). */
arb_status arb_matrix_gershgorin(arb_ctx ctx, arb_mat mat, double* lo, double* hi);

/* ---------------------------------------------------------------- the whole method */

/* ARRABIT with the multi-power inner solver (Algorithm 8) for the k largest or smallest
 * eigenpairs of A.
 *  x0:     n x p row-major float64 start block (ld = p), host or device per x0_on_device;
 *          NULL draws it from opts->seed with the library's Philox generator.
 *  evals:  host float64[k]: eigenvalues of A, descending for ARB_LARGEST, ascending for
 *          ARB_SMALLEST (Rayleigh quotients x_i^T A x_i).
 *  evecs:  n x k COLUMN-major float64 with leading dimension ldq >= n, host or device per
 *          evecs_on_device; may be NULL.  Each column has unit norm and its largest-
 *          magnitude entry positive.
 *  info:   may be NULL.
 * Requires 0 < k <= p and (q+1) p < n.  Returns ARB_OK when the outer stop rule (or its
 * near-tolerance case) is met, ARB_NOT_CONVERGED otherwise (outputs still filled). */
arb_status arb_solve(arb_ctx ctx, arb_mat mat, int32_t k, arb_which which, double tol,
                     const arb_options* opts, const double* x0, int x0_on_device,
                     double* evals, double* evecs, int64_t ldq, int evecs_on_device,
                     arb_info* info);

/* The i.i.d. Gaussian start block of Algorithm 8 ("initialize an i.i.d. Gaussian random
 * matrix X"): X (device, n x ncols row-major, ldx) gets element (i, j) = sample i*ncols + j
 * of the stream `seed` - Philox4x32-10 (Salmon et al., SC'11) on counter (e/2, 0, 0, 0)
 * with key (seed), two 53-bit uniforms, Box-Muller (cos for even e, sin for odd e).
 * arb_solve draws its start block this way when x0 is NULL. */
arb_status arb_gaussian_block(arb_ctx ctx, int64_t n, int32_t ncols, uint64_t seed, double* X,
                              int64_t ldx);

/* ---------------------------------------------------------------- hot-path steps
 * All pointers below are DEVICE pointers.  B denotes op_scale * A + op_shift * I. */

/* Y = psi_d(S) X diag(xscale), S = (2/(b-a)) (B - aI) - I: the filter of Algorithm 7 (the
 * map of eq. rhod with Alg. 8's call poly(A - aI, X, 0, b - a, Gamma_d)), evaluated in
 * the Chebyshev basis by Clenshaw's recurrence, d fused SpMM passes.
 * coef: HOST float64[degree+1], Chebyshev coefficients c_0..c_d of psi_d.
 * X, Y: n x ncols (ldx, ldy); Y must not overlap X.  xscale: float64[ncols] or NULL (1).
 * colss: float64[ncols] or NULL; receives the column sums of squares of Y (the MPM
 * normalisation of Section 3 needs 1/sqrt of these). */
arb_status arb_filter(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, double a,
                      double b, int32_t degree, const double* coef, const double* X,
                      int64_t ldx, int32_t ncols, const double* xscale, double* Y, int64_t ldy,
                      double* colss);

/* The same filter with FP32 blocks and FP32 arithmetic (the mixed-precision path's
 * filter; column sums of squares still accumulate in FP64).  X, Y: n x ncols FP32,
 * row-major; A's values are rounded to FP32 once and kept with the matrix. */
arb_status arb_filter_f32(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, double a,
                          double b, int32_t degree, const double* coef, const float* X,
                          int64_t ldx, int32_t ncols, const double* xscale, float* Y,
                          int64_t ldy, double* colss);

/* The same filter in double-float arithmetic (the ARB_MIXED_DF refinement's filter).  X and
 * Y are FP64 n x ncols row-major (device); X is rounded to hi + lo FP32 pairs, the d
 * Clenshaw passes run on those pairs (sums by two-sum, products by the FMA-exact product;
 * about 2^-44 relative error per operation) and the result is returned as hi + lo in FP64.
 * colss (device float64[ncols] or NULL) gets the FP64 column sums of squares of Y.  A's
 * double-float values are made once and kept with the matrix.  Errors: as arb_filter. */
arb_status arb_filter_df(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, double a,
                         double b, int32_t degree, const double* coef, const double* X,
                         int64_t ldx, int32_t ncols, const double* xscale, double* Y, int64_t ldy,
                         double* colss);

/* One instance of a batched filter (arb_filter_batched): the same arguments as arb_filter
 * / arb_filter_f32, X and Y FP32 when fp32 != 0, else FP64. */
typedef struct {
  arb_mat mat;
  double op_scale, op_shift, a, b;
  int32_t degree;
  int32_t fp32;
  const double* coef;    /* HOST, degree+1 Chebyshev coefficients */
  const void* X;         /* device, n x ncols, row-major */
  int64_t ldx;
  int32_t ncols;
  int32_t reserved0;
  const double* xscale;  /* device float64[ncols] or NULL */
  void* Y;               /* device, n x ncols; must not overlap X */
  int64_t ldy;
  double* colss;         /* device float64[ncols] or NULL: column sums of squares of Y */
} arb_filter_job;

/* Filter many instances (different matrices, widths, degrees, precisions) in persistent
 * cooperative launches, one per element type and vector width present (FP32 with 16-byte
 * rows, FP32 otherwise, FP64 likewise): all d_max passes of all instances of a class, a
 * grid-wide barrier between passes, tiles of rows handed to warps by per-pass ticket
 * counters.  Y equals the per-instance arb_filter / arb_filter_f32 result bit for bit (the
 * same operations in the same order per element); colss equals the column sums of squares
 * of Y to ~1e-14 relative (FP32 jobs sum in double-float pairs, FP64 jobs in FP64; the
 * order differs from the single-instance filter's).  X and Y are n rows of ldx / ldy
 * elements; rows of a 16-byte class may be read up to their leading dimension. */
arb_status arb_filter_batched(arb_ctx ctx, int32_t njobs, const arb_filter_job* jobs);

/* Host-side coefficients c_0..c_d (float64[degree+1]) of the degree-d Chebyshev
 * interpolant of max(0,t)^(10 d) at t_j = -cos(j pi/d) (Section 5, eq. chebfun-f), or of
 * T_d for ARB_FILTER_CHEBYSHEV. */
arb_status arb_filter_coefficients(int32_t filter, int32_t degree, double* coef);

/* Y = B X (one block product with A; Alg. 5 augmentation and Alg. 1's U^T A U). */
arb_status arb_spmm(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift,
                    const double* X, int64_t ldx, int32_t ncols, double* Y, int64_t ldy);

/* C = X^T Y (na x nb, row-major, ldc): the tall-skinny Gram product used by the inner
 * stop rule (eq. inn-stop, X^T X), orth(Z) and H = U^T A U.  Deterministic. */
arb_status arb_gram(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t na,
                    const double* Y, int64_t ldy, int32_t nb, double* C, int64_t ldc);

/* C = X^T Y for FP32 blocks X (n x na), Y (n x nb), result FP64 (the mixed path's FP32
 * Gram products).  Runs on the tensor cores when both blocks have leading dimensions that
 * are multiples of 4 and 16-byte aligned bases: every product as hi*hi + hi*lo + lo*hi of
 * TF32 parts (tcgen05.mma kind::tf32), FP32 sums over runs of 256 rows added in
 * double-float, about 1e-8 relative to ||x_i|| ||y_j|| per entry; otherwise on CUDA cores
 * (FP32 over 64-row runs, FP64 across runs).  Deterministic.  Errors: ARB_INVALID_ARG,
 * ARB_CUDA_ERROR (also if a tensor-core pipeline wait timed out). */
arb_status arb_gram_f32(arb_ctx ctx, int64_t n, const float* X, int64_t ldx, int32_t na,
                        const float* Y, int64_t ldy, int32_t nb, double* C, int64_t ldc);

/* arb_gram for callers that cannot let a library allocate device memory: applications
 * whose device memory is owned by their own pool allocator (which may hold all free memory
 * and must see every allocation), and latency-bound loops that must not meet the implicit
 * device synchronisation of cudaMalloc / cudaFree.  The same product C = X^T Y, but its
 * split-K partial sums live in a static device array of 1,048,576 doubles (8 MiB) that
 * the library holds on every device it is loaded on until the process exits, so the call
 * allocates nothing.  The paper has no counterpart; this is an interface variant only.
 *  - Limit: na * nb <= 1048576, else ARB_INVALID_ARG (nothing is launched).  Larger
 *    shapes go through arb_gram.  The row split shrinks so the partial sums fit.
 *  - The first call on a device looks up the array's device address (with that device
 *    current) and caches it for the process; make that first call before any stream
 *    capture.  cudaDeviceReset discards the array with the device's context, so do not
 *    call this after resetting a device it was used on.
 *  - Every call shares the one array: calls whose kernels overlap on the GPU (different
 *    streams, or two contexts on one device) race on it and must be serialised by the
 *    caller.  Each call overwrites every partial sum it reads, so no clearing is needed.
 *  - Results equal arb_gram's up to the order of the split sums. */
arb_status arb_gram_noalloc(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t na,
                            const double* Y, int64_t ldy, int32_t nb, double* C, int64_t ldc);

/* Out = alpha In W + beta Out for FP32 blocks In (n x na) and Out (n x nb), row-major with
 * leading dimensions ldi, ldo, and an FP64 matrix W (na x nb, row-major, ldw), all device
 * pointers: the mixed path's tall-skinny products - the Ritz rotation X = U V (Alg. 1 step
 * 4), the SVQB map and the block projections.  With na >= 8, leading dimensions that are
 * multiples of 4 and 16-byte aligned bases it runs on the tensor cores: W is rounded to
 * FP32, every product formed as hi*hi + hi*lo + lo*hi of TF32 parts (tcgen05.mma
 * kind::tf32) and summed in FP32 in tensor memory, about 1e-6 relative to
 * sum_k |In_ik| |W_kj| per entry; otherwise on CUDA cores in FP32.  beta = 0 does not read
 * Out.  In and Out must not overlap.  Errors: ARB_INVALID_ARG; ARB_CUDA_ERROR (also if a
 * tensor-core pipeline wait timed out). */
arb_status arb_gemm_tall_f32(arb_ctx ctx, int64_t n, const float* In, int64_t ldi, int32_t na,
                             const double* W, int64_t ldw, int32_t nb, double alpha, double beta,
                             float* Out, int64_t ldo);

/* Eigen-decomposition H = V diag(w) V^T of a symmetric m x m matrix (row-major, ldh) by
 * parallel cyclic Jacobi on the device (Alg. 1 step 3, reading H = V Sigma V^T).
 * w: float64[m] descending; V: m x m row-major (ldv), column j the eigenvector of w[j].
 * H is not modified.  sweeps (host, may be NULL) receives the sweep count.  Sweeps stop at
 * off(H) <= 1e-15 ||H||_F (FP64), or 1e-13 ||H||_F for orders above 32 on a context with
 * double-float dense arithmetic (arb_ctx_set_dense_df). */
arb_status arb_syevj(arb_ctx ctx, int32_t m, const double* H, int64_t ldh, double* w,
                     double* V, int64_t ldv, int32_t* sweeps);

/* Reciprocal 1-norm condition number of the symmetric Gram matrix G = X^T X
 * (eq. inn-stop); host output; 0 when G is not numerically positive definite. */
arb_status arb_rcond_gram(arb_ctx ctx, int64_t n, const double* X, int64_t ldx,
                          int32_t ncols, const double* xscale, double* rc);

/* U = an orthonormal basis of the numerical range of Z (Alg. 1 step 1, "orthonormalize
 * Z"): two passes of eigen-truncated Gram orthonormalisation with unit-column scaling.
 * U: n x m capacity (ldu); *rank (host) receives the number of columns written. */
arb_status arb_orth(arb_ctx ctx, int64_t n, const double* Z, int64_t ldz, int32_t m,
                    double* U, int64_t ldu, int32_t* rank);

/* (Y, w) = RR(B, Z), Algorithm 1.  Y: n x m capacity (ldy), w: float64[m] device,
 * descending; *rank (host) = number of Ritz pairs produced (= rank of Z). */
arb_status arb_rayleigh_ritz(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift,
                             int64_t n, const double* Z, int64_t ldz, int32_t m, double* Y,
                             int64_t ldy, double* w, int32_t* rank);

/* (Y, w) = ARR(B, X, q), Algorithm 5: Rayleigh-Ritz on span[X, BX, ..., B^q X] (built as
 * an orthonormal block Krylov basis), leading `npairs` Ritz pairs kept.
 * X: n x ncols; Y: n x npairs (ldy); w: float64[npairs] device; *rank (host) = subspace
 * dimension.  Fewer than npairs directions -> ARB_BREAKDOWN. */
arb_status arb_arr(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, int64_t n,
                   const double* X, int64_t ldx, int32_t ncols, int32_t q, int32_t npairs,
                   double* Y, int64_t ldy, double* w, int32_t* rank);

/* ---------------------------------------------------------------- serving
 * Continuous batching of eigen-solves on one GPU (a request loop over arb_solve).
 * Requests are admitted in arrival order as soon as one of `max_slots` worker slots is free
 * and the request's HBM footprint (arb_server_footprint) fits in what the admitted
 * requests leave of `hbm_budget_bytes`; admitted solves run concurrently, each slot on
 * its own CUDA stream and context.  A request whose footprint exceeds the whole budget
 * is refused at submission with ARB_REJECTED.  Results are the same as a standalone
 * arb_solve with the same inputs (the kernels are deterministic).  The server is
 * thread-safe for arb_submit / arb_wait; destroy it only after every wait has returned. */
typedef struct arb_server_s* arb_server;
typedef int64_t arb_ticket;

/* Bytes of device workspace a solve of an n x p block with q augmentation blocks takes
 * (precision: arb_precision); -1 on bad arguments. */
int64_t arb_server_footprint(int64_t n, int64_t nnz, int32_t p, int32_t q, int32_t precision);
arb_status arb_server_create(int device, size_t hbm_budget_bytes, int32_t max_slots, arb_server* out);
/* Queue a solve of `mat` (which must live on the server's device and stay alive until
 * the request is waited for).  x0: host n x p start block (copied) or NULL; want_evecs:
 * keep the eigenvectors for arb_wait. */
arb_status arb_submit(arb_server srv, arb_mat mat, int32_t k, arb_which which, double tol,
                      const arb_options* opts, const double* x0, int want_evecs, arb_ticket* ticket);
/* Wait up to timeout_ms (< 0: forever) for a request; ARB_TIMEOUT if it is not done yet
 * (the ticket stays valid).  On completion the outputs are filled as by arb_solve (evecs
 * host, column-major, ldq), latency_s (may be NULL) is submit-to-completion wall time,
 * the ticket is retired, and the solve's own status is returned. */
arb_status arb_wait(arb_server srv, arb_ticket ticket, int32_t timeout_ms, double* evals, double* evecs,
                    int64_t ldq, arb_info* info, double* latency_s);
/* Stop the server: queued requests are dropped, running ones finish, threads join. */
arb_status arb_server_destroy(arb_server srv);

/* Solve nb independent problems (uneven sizes) as one batch: up to max_concurrent solves
 * run at once, each on its own stream, largest first; HBM admission as for the server
 * with a budget of 90% of the device's free memory.  Per-instance arguments as for
 * arb_solve (x0[i] host or NULL; evecs[i] host column-major or NULL; ldq may be NULL for
 * ldq[i] = n_i; opts and info may be NULL).  Returns ARB_OK when every instance converged,
 * else the first failing status (or ARB_NOT_CONVERGED). */
arb_status arb_solve_batched(arb_ctx ctx, int32_t nb, const arb_mat* mats, const int32_t* k,
                             const arb_which* which, const double* tol, const arb_options* opts,
                             const double* const* x0, double* const* evals, double* const* evecs,
                             const int64_t* ldq, arb_info* info, int32_t max_concurrent);

/* ---------------------------------------------------------------- lock-step batching */

/* Autotuner of the fused block SpMM for one matrix, by measurement: every candidate row
 * layout - CSR, or SELL-C-sigma with C = 8 (sigma = 256) or C = 32 (sigma = 1024) - and
 * vector width per lane - 4, 2 or 1 FP32 columns, so a warp covers a column slice of 128,
 * 64 or 32 per row - is timed on one fused filter-like pass over an n x ncols FP32 block
 * (gathers plus the X and Z streams of the Clenshaw recurrence; CUDA events on the
 * context's stream, best of 3), and the fastest is kept with the matrix: its SELL copy is
 * made or dropped (as by arb_matrix_set_sell) and the width caps every later fused SpMM on
 * it, batched or not.  choice (host int32[2], may be NULL) receives {C (0: CSR), width};
 * ms (host, may be NULL) the candidate's time per pass.  Not to be called while other
 * calls use the matrix.  The paper tunes nothing of this kind (its products are MKL
 * calls); the degree is chosen by the paper's own rule (ARB_ADAPT_DEGREE).
 * Errors: ARB_INVALID_ARG, ARB_CUDA_ERROR. */
arb_status arb_matrix_autotune(arb_ctx ctx, arb_mat mat, int32_t ncols, int32_t* choice, double* ms);

typedef struct {
  int64_t rounds;            /* inner-step rounds of the lock-step loop */
  int64_t batched_launches;  /* persistent batched filter launches, direct or from graphs */
  int64_t graph_launches;    /* rounds replayed from a captured CUDA graph */
  int64_t graphs_captured;   /* distinct round shapes captured */
  int64_t single_steps;      /* inner steps run for one instance alone (GN, double-float filter) */
  double t_total;            /* seconds spent in the call */
  double t_batched;          /* host seconds from forming a round's batch to its completion */
  double t_single;           /* host seconds in the rounds' single-instance steps */
  double t_checks;           /* host seconds in the inner stop checks and ARR tails */
  double t_batch_kernel;     /* device seconds of the batched filter launches (CUDA events) */
  double t_prepare;          /* host seconds forming the batches (descriptors, upload) */
  int64_t batched_jobs;      /* instance steps filtered by the batched launches, summed over rounds */
} arb_batch_stats;

enum { ARB_BATCH_GRAPHS = 1, ARB_BATCH_AUTOTUNE = 2 };

/* Solve nb independent problems (Algorithm 8 each, uneven sizes, widths and degrees) in
 * lock step: every instance runs its own outer iterations, stop rules and precision
 * phases, but in each round every instance that is in its inner loop takes one
 * multi-power step, and the filters of all those steps run as one batched filter
 * (arb_filter_batched: one persistent cooperative launch per element type present, all
 * passes of all instances, a grid-wide barrier between passes).  Instances whose step
 * cannot join the batch (the GN inner solver, the double-float refinement filter of
 * ARB_MIXED_DF) take it alone in the same round.
 * flags: ARB_BATCH_GRAPHS captures the device work of a round into a CUDA graph the second
 * time the same launch shape occurs (the same descriptor addresses, job counts per class
 * and maximum degree; everything else is read from the descriptors) and replays it
 * afterwards, with the round's descriptors re-uploaded before each replay;
 * ARB_BATCH_AUTOTUNE runs arb_matrix_autotune on every distinct matrix first (width p of
 * its first problem).  The work runs on a stream of its own, ordered after the context's
 * stream; each instance has workspaces of its own for the duration of the call.
 * Arguments and outputs per instance as for arb_solve (x0[i] host n_i x p_i or NULL;
 * evecs[i] host column-major or NULL; ldq may be NULL for ldq[i] = n_i; opts, info and
 * stats may be NULL).  Returns ARB_OK when every instance converged, else the first
 * failing status (or ARB_NOT_CONVERGED).  The paper solves one problem at a time; the
 * lock-step batch is this library's. */
arb_status arb_solve_lockstep(arb_ctx ctx, int32_t nb, const arb_mat* mats, const int32_t* k, const arb_which* which,
                              const double* tol, const arb_options* opts, const double* const* x0,
                              double* const* evals, double* const* evecs, const int64_t* ldq, arb_info* info,
                              int32_t flags, arb_batch_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* ARRABIT_H */
