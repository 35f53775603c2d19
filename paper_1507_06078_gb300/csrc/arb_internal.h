// Internal declarations shared by the CUDA translation units of the ARRABIT library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "arrabit.h"

namespace arb {

// A double-float value hi + lo (two FP32 numbers, |lo| <= ulp(hi)/2): blocks of the
// double-float refinement filter (df.cu).
struct __align__(8) df2 {
  float hi, lo;
};

// Workspace slots owned by a context.  Each slot is one device allocation that grows on
// demand; contents are not preserved across calls that request a larger size.
enum WsSlot : int {
  WS_GRAM_PART = 0,   // split-K partial sums of Gram products
  WS_SS_PART,         // per-block column sums of squares from the fused SpMM
  WS_COEF,            // per-step per-column filter coefficients
  WS_SMALL0,          // small dense matrices (Gram, eigenvectors, ...)
  WS_SMALL1,
  WS_SMALL2,
  WS_SMALL3,
  WS_VEC0,            // short vectors
  WS_VEC1,
  WS_VEC2,
  WS_INT0,
  WS_JACOBI,          // Jacobi rotation table + reduction scratch
  WS_FILT_W1,         // filter work blocks (step-level entry point)
  WS_FILT_W2,
  WS_TALL0,           // n x w temporaries of orth / RR / ARR entry points
  WS_TALL1,
  WS_TALL2,
  WS_SOLVER_X,        // solver state (iterate, work blocks, bases)
  WS_SOLVER_Y,
  WS_SOLVER_W1,
  WS_SOLVER_W2,
  WS_SOLVER_QC,
  WS_SOLVER_XALL,
  WS_SOLVER_U,
  WS_SOLVER_AU,
  WS_SOLVER_T,
  WS_SOLVER_T2,
  WS_S_V,             // solver: eigenvectors of H, selected columns
  WS_S_VSEL,
  WS_S_VEC,           // solver: short per-column vectors
  WS_F32_X,           // mixed-precision solver: FP32 iterate, work blocks and bases
  WS_F32_W1,
  WS_F32_W2,
  WS_F32_XALL,
  WS_F32_U,
  WS_F32_AU,
  WS_F32_T,
  WS_F32_T2,
  WS_BATCH_WORK,      // batched filter: per-instance work blocks and multiplier tables
  WS_BATCH_DESC,
  WS_TC_ERR,          // tensor-core kernels: error word
  WS_TC_IMG,          // tensor-core tall products: packed split W
  WS_ORTH_NORM,       // orth's recovery of truncated directions: column norms, column list
  WS_ORTH_IDX,
  WS_CHOL,            // Cholesky: diagonal-block inverse, status words, factor, inverse
  WS_CHOL_STATUS,
  WS_CHOL_R,
  WS_CHOL_RINV,
  WS_NUM_SLOTS
};

}  // namespace arb

struct arb_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  int64_t launches = 0;
  std::string last_error = "no error";
  void* ws[arb::WS_NUM_SLOTS] = {};
  size_t ws_bytes[arb::WS_NUM_SLOTS] = {};
  void* host_pinned = nullptr;  // small staging area for read-backs
  size_t host_pinned_bytes = 0;
  int jacobi_max_blocks = 0;    // co-resident blocks for the cooperative Jacobi kernel
  int jacobi_max_blocks_df = 0;  // ... and for its double-float form
  bool stream_ordered = false;  // workspaces from cudaMallocAsync/cudaFreeAsync on `stream`
  // Cooperative (grid-synchronising) launches use at most 1/coop_share of the device's
  // co-resident CTAs, so that the grids of coop_share contexts running concurrently (the
  // server's slots) always fit on the device together and none waits on another's CTAs.
  int coop_share = 1;
  // FP64 Gram and tall-skinny products in double-float arithmetic on the FP32 pipe
  // (arb_ctx_set_dense_df; ARB_MIXED_DF solves set it for their refinement phase)
  bool dense_df = false;
  // device error word of pipelined kernels whose bounded waits gave up (two ints, zeroed);
  // read and cleared at every host synchronisation of d2h_sync
  int32_t* err_dev = nullptr;
  // ordering event of the lock-step driver's contexts (made with them)
  cudaEvent_t ev_join = nullptr;
};

struct arb_mat_s {
  arb_ctx ctx = nullptr;  // creating context (not dereferenced on destroy)
  int device = 0;
  int64_t n = 0, nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;  // FP32 copy of val for the mixed-precision filter (made on demand)
  arb::df2* valdf = nullptr;  // double-float copy of val for the double-float filter (made on demand)
  int32_t max_row_nnz = -1;  // longest row (-1: unknown)
  // SELL-C-sigma copy (arb_matrix_set_sell; sell_C = 0: CSR only).  The SpMM kernels take
  // it when present; the CSR arrays stay for everything else.
  int32_t sell_C = 0, sell_sigma = 0;
  int64_t sell_slots = 0;
  int32_t* sell_perm = nullptr;  // [n] original row at each sorted position
  int32_t* sell_len = nullptr;   // [n] its nonzero count
  int64_t* sell_cptr = nullptr;  // [chunks + 1] first slot of each chunk
  int32_t* sell_col = nullptr;   // [slots] column indices (padding: 0)
  double* sell_val = nullptr;    // [slots] values (padding: 0), and their FP32 / double-float copies
  float* sell_val32 = nullptr;
  arb::df2* sell_valdf = nullptr;
  // group table of the bulk-copy FP32 SpMM (spmm_bulk.cu), made on first use
  int32_t* bulk_tab = nullptr;
  // autotuned SpMM settings (arb_matrix_autotune): widest vector access per lane of the
  // FP32 / FP64 fused SpMM kernels (0: the widest the operands allow), tuned flag
  int32_t tune_vec = 0;
  bool tuned = false;
  bool gersh_valid = false;
  double gersh_lo = 0.0, gersh_hi = 0.0;
  std::mutex mu;  // guards the lazily made val32 / valdf and the Gershgorin cache (shared by server workers)
};

namespace arb {

// ---------------------------------------------------------------- error plumbing
arb_status set_error(arb_ctx ctx, arb_status st, const std::string& msg);
arb_status cuda_error(arb_ctx ctx, cudaError_t e, const char* what, const char* file, int line);

#define ARB_CUDA(ctx, expr)                                                   \
  do {                                                                        \
    cudaError_t e__ = (expr);                                                 \
    if (e__ != cudaSuccess) return ::arb::cuda_error((ctx), e__, #expr, __FILE__, __LINE__); \
  } while (0)

// Check the launch just made and count it.
#define ARB_LAUNCHED(ctx)                                                     \
  do {                                                                        \
    (ctx)->launches++;                                                        \
    cudaError_t e__ = cudaGetLastError();                                     \
    if (e__ != cudaSuccess) return ::arb::cuda_error((ctx), e__, "kernel launch", __FILE__, __LINE__); \
  } while (0)

#define ARB_TRY(expr)                        \
  do {                                       \
    arb_status s__ = (expr);                 \
    if (s__ != ARB_OK) return s__;           \
  } while (0)

// Device workspace of at least `bytes` for `slot`.
arb_status ws_get(arb_ctx ctx, int slot, size_t bytes, void** out);
template <typename T>
inline arb_status ws(arb_ctx ctx, int slot, size_t count, T** out) {
  return ws_get(ctx, slot, count * sizeof(T) + 256, reinterpret_cast<void**>(out));
}
// Release every workspace slot of the context.
arb_status ws_release_all(arb_ctx ctx);
// Device bytes the solver's workspaces take for an n x p block, q augmentation blocks and
// a matrix with nnz entries (FP32 / double-float copies included for the mixed paths).
size_t solve_footprint(int64_t n, int64_t nnz, int32_t p, int32_t q, int32_t precision);
// The whole method on ctx (used by arb_solve and by the server's workers).
arb_status solve_on(arb_ctx ctx, arb_mat mat, int32_t k, arb_which which, double tol, const arb_options* opts,
                    const double* x0, int x0_on_device, double* evals, double* evecs, int64_t ldq,
                    int evecs_on_device, arb_info* info);
// The context's device error word (allocated and zeroed on first use).
arb_status device_error_word(arb_ctx ctx, int32_t** out);
// Pinned host staging of at least `bytes`.
arb_status host_stage(arb_ctx ctx, size_t bytes, void** out);
// Copy `bytes` from device to a host pointer through the stream and wait.
arb_status d2h_sync(arb_ctx ctx, void* host, const void* dev, size_t bytes);

// ---------------------------------------------------------------- kernels (spmm.cu)
// out = sy[c] * (alpha * (A Yin) + beta * Yin) + sx[c] * X + sz[c] * Z, row-major blocks of
// element type T (float64 path or the FP32 filter of the mixed path).
// Optional outputs: `out` (skipped when NULL) and per-column reductions into `colred`
// (FP64 sums over rows of out^2, or of out * Yin when dot_with_yin).
template <typename T>
struct SpmmArgs {
  const arb_mat_s* A = nullptr;
  int32_t ncols = 0;
  const T* Yin = nullptr;
  int64_t ldy = 0;
  double alpha = 1.0, beta = 0.0;
  const double* sy = nullptr;  // NULL: 1
  const T* X = nullptr;
  int64_t ldx = 0;
  const double* sx = nullptr;  // required when X != NULL
  const T* Z = nullptr;
  int64_t ldz = 0;
  const double* sz = nullptr;  // required when Z != NULL
  T* out = nullptr;
  int64_t ldo = 0;
  double* colred = nullptr;    // float64[ncols] result of the column reduction, or NULL
  bool dot_with_yin = false;
};
template <typename T>
arb_status spmm_fused(arb_ctx ctx, const SpmmArgs<T>& a);
// double-float blocks (df.cu): leading dimensions even, 16-byte aligned bases
template <>
arb_status spmm_fused<df2>(arb_ctx ctx, const SpmmArgs<df2>& a);
// The FP32 product by the bulk-copy pipelined kernel (spmm_bulk.cu) when the operands allow
// it (rows of at most 32 nonzeros, CSR, ncols a multiple of 4, 16-byte aligned rows);
// *launched = false leaves the work to the caller.  want_red: per-CTA partial column sums
// into *part (grid x ncols, *grid_out CTAs).
arb_status spmm_bulk_f32(arb_ctx ctx, const arb_mat_s* A, const SpmmArgs<float>& a, const float* val, bool want_red,
                         bool* launched, int* grid_out, double** part);
// FP32 copy of A's values (kept with the matrix).
arb_status ensure_val32(arb_ctx ctx, arb_mat mat);

// ---------------------------------------------------------------- double-float (df.cu)
// Double-float copy of A's values (kept with the matrix).
arb_status ensure_valdf(arb_ctx ctx, arb_mat mat);
// dst (n x ncols, df) = src (FP64), rounded to nearest double-float
arb_status to_df(arb_ctx ctx, int64_t n, const double* src, int64_t lds, int32_t ncols, df2* dst, int64_t ldd);
// dst (FP64) = hi + lo of src
arb_status from_df(arb_ctx ctx, int64_t n, const df2* src, int64_t lds, int32_t ncols, double* dst, int64_t ldd);

// Gershgorin lower/upper bound of A into host doubles.
arb_status gershgorin(arb_ctx ctx, arb_mat mat, double* lo, double* hi);

// Column sums of squares of a block (ncols results, device).
arb_status col_sumsq(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t ncols,
                     double* out);

// ---------------------------------------------------------------- kernels (dense.cu)
// C (na x nb, ldc, FP64) = X^T Y over n rows of element type T; deterministic split-K.
// FP32 inputs are multiplied and summed in FP32 over runs of 64 rows and the run sums are
// added in FP64.  symmetric: X == Y.
template <typename T>
arb_status gram(arb_ctx ctx, int64_t n, const T* X, int64_t ldx, int32_t na, const T* Y, int64_t ldy,
                int32_t nb, double* C, int64_t ldc);
// The FP64 Gram product with caller-provided partial-sum storage (part_capacity doubles,
// at least na * nb); no workspace is requested.  The row split shrinks to fit.
arb_status gram_into(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t na, const double* Y,
                     int64_t ldy, int32_t nb, double* C, int64_t ldc, double* part, size_t part_capacity);
// Out (n x nb) = alpha * In (n x na) * W (na x nb, FP64, ldw) + beta * Out, accumulated in T.
// Out must not alias In.
template <typename T>
arb_status gemm_tall(arb_ctx ctx, int64_t n, const T* In, int64_t ldi, int32_t na, const double* W,
                     int64_t ldw, int32_t nb, double alpha, double beta, T* Out, int64_t ldo);
// dst[:, j] = src[:, idx[j]] for j < ncols (idx on device)
template <typename T>
arb_status col_norms2(arb_ctx ctx, int64_t n, const T* X, int64_t ldx, int32_t m, double* out);
template <typename T>
arb_status gather_cols(arb_ctx ctx, int64_t n, const T* src, int64_t lds, const int32_t* idx,
                       int32_t ncols, T* dst, int64_t ldd);
// dst[:, j] = idx[j] >= 0 ? srcA[:, idx[j]] : srcB[:, -idx[j]-1]
template <typename T>
arb_status gather_cols2(arb_ctx ctx, int64_t n, const T* srcA, int64_t ldA, const T* srcB, int64_t ldB,
                        const int32_t* idx, int32_t ncols, T* dst, int64_t ldd);
// dst = src (n x ncols), converting the element type
template <typename Ti, typename To>
arb_status copy_block(arb_ctx ctx, int64_t n, const Ti* src, int64_t lds, int32_t ncols, To* dst,
                      int64_t ldd);
// res[c] = sqrt(ss[c]) / max(1, |lambda_c|), lambda_c = smallest ? sigma - mu_c : mu_c
arb_status residual_finish(arb_ctx ctx, int32_t p, const double* ss, const double* mu, int smallest,
                           double sigma, double* res);
// Per-column index of the largest |x| (ties: smallest row) -> sign[c] = +-1.
arb_status column_signs(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t ncols,
                        double* sign);
// evecs[c * ldq + i] = sign[c] * X[i * ldx + perm[c]]  (column-major output)
arb_status write_colmajor(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, const int32_t* perm,
                          const double* sign, int32_t k, double* out, int64_t ldq);
arb_status fill(arb_ctx ctx, double* p, int64_t count, double v);
// H <- (H + H^T)/2 for an m x m row-major matrix
arb_status symmetrize(arb_ctx ctx, int32_t m, double* H, int64_t ldh);
// H with its diagonal blocks (starts off[b], sizes rk[b]) computed in full and, off the
// diagonal, only the upper blocks (the lower ones zero): averaged inside diagonal blocks,
// the upper blocks mirrored below
arb_status symmetrize_upper_blocks(arb_ctx ctx, int32_t m, double* H, int64_t ldh, const int32_t* off,
                                  const int32_t* rk, int32_t nblk);
// w <- w - a v - b u and dst <- s src (n-vectors)
arb_status lin3(arb_ctx ctx, int64_t n, double* w, double a, const double* v, double b, const double* u);
arb_status scale_vec(arb_ctx ctx, int64_t n, double* dst, const double* src, double s);
// Lanczos estimates of the extreme eigenvalues of A with residual-based margins
// (*lo <= lambda_min, *hi >= lambda_max up to the Lanczos residual bound), from `steps`
// steps started at the Gaussian column of Philox stream `seed`.
arb_status lanczos_bounds(arb_ctx ctx, arb_mat mat, int32_t steps, uint64_t seed, double* lo, double* hi);
// G <- diag(s) G diag(s)
arb_status scale_sym(arb_ctx ctx, int32_t m, double* G, int64_t ldg, const double* s);
// s[c] = 1/sqrt(ss[c]) (0 when ss[c] == 0)
arb_status inv_sqrt(arb_ctx ctx, int32_t m, const double* ss, double* s);
// Ghat = D G D with D = diag(1/sqrt(G_ii)); d gets the diagonal of D.
arb_status svqb_prep(arb_ctx ctx, int32_t m, const double* G, int64_t ldg, double* Ghat,
                     double* d);
// M[:, j] = d .* W[:, j] / sqrt(theta_j) for theta_j > tau * theta_0 (else 0); *rank_dev.
arb_status svqb_finish(arb_ctx ctx, int32_t m, const double* theta, const double* W,
                       int64_t ldw, const double* d, double tau, double* M, int32_t* rank_dev);
// rc = 1/(||G||_1 ||G^{-1}||_1) from G and its eigen-decomposition, into rc_dev.
arb_status rcond_from_eig(arb_ctx ctx, int32_t m, const double* G, int64_t ldg,
                          const double* theta, const double* W, int64_t ldw, double* rc_dev);
// Largest p of the concatenation [vlock (nl), vnew (nn)] (descending, stable): map[s] and
// val[s]; map < nl -> locked index, else nl + index into vnew.  *count = min(p, nl+nn).
arb_status select_top(arb_ctx ctx, const double* vlock, int32_t nl, const double* vnew,
                      int32_t nn, int32_t p, int32_t* map, double* val);
// Gaussian fill from the Philox4x32-10 stream `seed` (row-major n x ncols, element
// i*ncols + j), same numbering as the input generators.
template <typename T>
arb_status gaussian_fill(arb_ctx ctx, int64_t n, int32_t ncols, uint64_t seed, T* X, int64_t ldx);

// ---------------------------------------------------------------- tensor-core Gram (tc.cu)
// part[s] (na x nb, FP64) = X^T Y over rows [s*rows, (s+1)*rows) of FP32 blocks by
// split-TF32 tcgen05 products; *err_dev set nonzero if an mbarrier wait gave up.
bool gram_tc_supported(int64_t n, int64_t ldx, int64_t ldy, const void* X, const void* Y);
int gram_tc_rows_align();
int gram_tc_tile_m();
int gram_tc_tile_n();
// Out = alpha In W + beta Out on the tensor cores (tc.cu): FP32 In (n x na), Out (n x nb), FP64 W
// (na x nb) packed into img (gemm_tc_image_floats(na, nb) floats, 16-byte aligned) first.
bool gemm_tc_supported(int64_t ldi, int64_t ldo, const void* In, const void* Out);
size_t gemm_tc_image_floats(int32_t na, int32_t nb);
arb_status gemm_tc_launch(arb_ctx ctx, int64_t n, const float* In, int64_t ldi, int32_t na, const double* W,
                          int64_t ldw, int32_t nb, float alpha, float beta, float* Out, int64_t ldo, float* img,
                          int* err_dev);
arb_status gram_tc_launch(arb_ctx ctx, int64_t n, const float* X, int64_t ldx, int32_t na, const float* Y,
                          int64_t ldy, int32_t nb, int symmetric, double* part, int64_t nsplit, int64_t rows,
                          int* err_dev);

// ---------------------------------------------------------------- Cholesky (chol.cu)
// In place: the upper triangle of the symmetric m x m matrix A (row-major, lda) becomes the
// factor R with A = R^T R (FP64, blocked right-looking).  A pivot <= thr (or not finite)
// stops the factorisation: status[0] = 1, status[1] = its index (device words, cleared
// first).  No host synchronisation.
arb_status cholesky_upper(arb_ctx ctx, int32_t m, double* A, int64_t lda, double thr, int32_t* status);
int cholesky_max_order();
// M (m x m, row-major, ld m) = diag(d) R^{-1} (d NULL: R^{-1}) for the upper factor R;
// nothing is written when status[0] != 0.
arb_status triangular_inverse(arb_ctx ctx, int32_t m, const double* R, int64_t lda, const double* d, double* M,
                              const int32_t* status);
// Ginv (m x m, ld m) = G^{-1} of a symmetric positive definite G through its Cholesky factor
// (R, Rinv: m x m work); status[0] != 0 (device) when G is not numerically positive definite.
arb_status spd_inverse(arb_ctx ctx, int32_t m, const double* G, int64_t ldg, double* R, double* Rinv, double* Ginv,
                       int32_t* status);
// M[i][i] += s for i < m
arb_status add_diagonal(arb_ctx ctx, int32_t m, double* M, int64_t ldm, double s);
// rc_dev = 1 / (||G||_1 ||G^{-1}||_1) with G^{-1} from the Cholesky factor of G; 0 when G is
// not numerically positive definite.  R, Rinv, Ginv: m x m work matrices.
arb_status rcond_from_cholesky(arb_ctx ctx, int32_t m, const double* G, int64_t ldg, double* R, double* Rinv,
                               double* Ginv, int32_t* status, double* rc_dev);

// ---------------------------------------------------------------- batched filter (batched.cu)
// A prepared batched filter: descriptors on the device, workspaces.  filter_batched_launch
// issues one kernel per job class present (capturable into a CUDA graph).
struct BatchPlan {
  struct Class {             // jobs of one element type and vector width: 0 FP32 x4, 1 FP32 x1,
    int first = 0;           // 2 FP64 x2, 3 FP64 x1 (in class order on the device)
    int count = 0;
    int grid = 0;
    const int64_t* doff = nullptr;  // pass and table-prologue offsets over the class's jobs
    const int64_t* dcs = nullptr;   // column-sum offsets over the class's columns
    unsigned long long* tickets = nullptr;  // per-pass tile counters
  };
  int32_t njobs = 0;
  int dmax = 0;
  std::vector<arb_filter_job> jobs;
  Class cls[4];
  const void* dj = nullptr;  // device job and pass descriptors
  const void* dp = nullptr;
  double* part = nullptr;    // column-sum partials
};
arb_status filter_batched_prepare(arb_ctx ctx, int32_t njobs, const arb_filter_job* jobs, BatchPlan* plan);
arb_status filter_batched_launch(arb_ctx ctx, const BatchPlan& plan);
arb_status filter_batched(arb_ctx ctx, int32_t njobs, const arb_filter_job* jobs);

// ---------------------------------------------------------------- Jacobi (jacobi.cu)
// w (descending), V (row-major, column j = eigenvector) of symmetric H (not modified).
// Sweeps stop when off(A) <= tol ||H||_F: 1e-15 for FP64 data, 1e-10 where H is formed from
// FP32 blocks and so carries FP32-level errors itself.
// frees a matrix's SELL-C-sigma arrays (sell.cu)
void matrix_free_sell(arb_mat m);
// frees a matrix's bulk-copy group table (spmm_bulk.cu)
void matrix_free_bulk(arb_mat m);
// df: orders above 32 in double-float arithmetic on the FP32 pipe (stops at <= 1e-13).
// jac_df / jac_tol: the Jacobi arithmetic and tolerance for matrices formed from element
// type T: FP32 bases (accurate to ~1e-7) and double-float dense products take the
// double-float kernel; plain FP64 keeps FP64 throughout.
arb_status syevj(arb_ctx ctx, int32_t m, const double* H, int64_t ldh, double* w, double* V,
                 int64_t ldv, int32_t* sweeps, double tol = 1e-15, bool df = false);
template <typename T>
inline bool jac_df(arb_ctx ctx) {
  return sizeof(T) == 4 || ctx->dense_df;
}
template <typename T>
inline double jac_tol(arb_ctx ctx) {
  return sizeof(T) == 4 ? 1e-10 : (ctx->dense_df ? 1e-13 : 1e-15);
}

// ---------------------------------------------------------------- composite steps (steps.cu)
struct FilterPlan {
  double alpha = 1.0, beta = 0.0;  // S = alpha A + beta I
  int32_t degree = 0;
  double coef[64] = {};            // Chebyshev coefficients c_0..c_d
};
// S from B = op_scale A + op_shift I and the interval [a, b] of Algorithm 8's call
// poly(B - aI, X, 0, b - a, Gamma_d).
FilterPlan make_filter_plan(double op_scale, double op_shift, double a, double b, int32_t degree,
                            const double* coef);
// Y = psi_d(S) (X diag(xscale)); W1, W2: n x ncols work blocks (ldw); Y may be NULL, in
// which case the result overwrites one of W1/W2 and *result points at it.  colss: column
// sums of squares of the result (device, may be NULL).
template <typename T>
arb_status filter_apply(arb_ctx ctx, arb_mat mat, const FilterPlan& plan, const T* X, int64_t ldx,
                        int32_t ncols, const double* xscale, T* W1, T* W2, int64_t ldw, T* Y,
                        int64_t ldy, double* colss, T** result);

// Orthonormal basis of range(Z) (two eigen-truncated Gram passes).  U must not alias Z and
// has room for m columns; tmp: n x m work block.  *rank on host.  recover: when the Gram
// passes truncated directions, project Z off the basis and orthonormalise what is left
// above rounding level (up to two rounds), so a block whose singular values span more
// than the Gram passes resolve (~1e-6 of the largest) keeps its small directions.
template <typename T>
arb_status orth(arb_ctx ctx, int64_t n, const T* Z, int64_t ldz, int32_t m, T* U, int64_t ldu, T* tmp,
                int64_t ldt, int32_t* rank, bool recover = false);

// Reciprocal 1-norm condition number of diag(xs) X^T X diag(xs) (host result).
template <typename T>
arb_status rcond_gram(arb_ctx ctx, int64_t n, const T* X, int64_t ldx, int32_t ncols, const double* xs,
                      double* rc);

// X <- X - Q (Q^T X)
template <typename T>
arb_status project_out(arb_ctx ctx, int64_t n, const T* Q, int64_t ldq, int32_t nq, T* X, int64_t ldx,
                       int32_t ncols);

// Block-Krylov Rayleigh-Ritz: U holds an orthonormal basis of span[X, BX, ..., B^q X]
// (projected against Qc), AU = B U, then H = U^T AU is diagonalised.
// Outputs: *m (subspace dimension, host), theta (device, m, descending), V (device m x m,
// row-major with leading dimension m; column j is the eigenvector of theta_j).
template <typename T>
struct ArrWork {
  T* U = nullptr;  int64_t ldu = 0;   // n x mcap
  T* AU = nullptr; int64_t ldau = 0;  // n x mcap
  T* T1 = nullptr; int64_t ldt = 0;   // n x w
  T* T2 = nullptr; int64_t ldt2 = 0;  // n x w
};
template <typename T>
arb_status arr_basis_and_eig(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, int64_t n, T* X,
                             int64_t ldx, int32_t w, const T* Qc, int64_t ldqc, int32_t nl, int32_t q,
                             const ArrWork<T>& wk, int32_t* m_out, double* theta, double* V);

}  // namespace arb
