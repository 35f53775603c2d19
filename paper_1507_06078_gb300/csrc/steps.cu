// Composite steps of the subspace update and of the augmented Rayleigh-Ritz projection,
// built from the kernels of spmm.cu, dense.cu and jacobi.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "arb_internal.h"

namespace arb {
namespace {

struct ChebCoef {
  double c[64];
};

// Per-step per-column multipliers of the fused Clenshaw step (see filter_apply).
//   table[(3 t + 0) * ncols + c] = sy, [(3 t + 1) ...] = sx, [(3 t + 2) ...] = sz
__global__ void filter_table_kernel(int d, ChebCoef cc, const double* __restrict__ xs, int ncols,
                                    double* __restrict__ table) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int nsteps = d;
  if (idx >= static_cast<int64_t>(nsteps) * ncols) return;
  const int t = static_cast<int>(idx / ncols), c = static_cast<int>(idx % ncols);
  const double s = xs ? xs[c] : 1.0;
  const int j = d - 1 - t;  // step t produces b_j (b_0 at the last step means Y)
  double sy, sx, sz;
  if (d == 1) {
    sy = cc.c[1] * s;
    sx = cc.c[0] * s;
    sz = 0.0;
  } else {
    sy = (t == 0) ? 2.0 * cc.c[d] * s : (t == d - 1 ? 1.0 : 2.0);
    sx = cc.c[j] * s;
    sz = (j + 2 == d) ? -cc.c[d] * s : -1.0;
  }
  table[(3 * static_cast<int64_t>(t) + 0) * ncols + c] = sy;
  table[(3 * static_cast<int64_t>(t) + 1) * ncols + c] = sx;
  table[(3 * static_cast<int64_t>(t) + 2) * ncols + c] = sz;
}

// Gram truncation threshold relative to the largest eigenvalue of the unit-diagonal Gram
// matrix, above the noise of the computed Gram entries: 64 m u for FP64 blocks; for FP32
// blocks (FP32 products summed in FP64 over 64-row runs, entries good to ~3e-9) 2e-9 m.
template <typename T>
inline double orth_tau(int m) {
  return sizeof(T) == 4 ? 2e-9 * std::max(m, 1) : 64.0 * std::max(m, 1) * 1.11e-16;
}

}  // namespace

FilterPlan make_filter_plan(double op_scale, double op_shift, double a, double b, int32_t degree,
                            const double* coef) {
  // Algorithm 8 calls poly(B - aI, X, 0, b - a, Gamma_d); Algorithm 7 with interval
  // [0, b - a] has c0 = (0 + (b-a))/(0 - (b-a)) = -1 and c1 = 2/(b - a), so the recurrence
  // variable is S = c1 (B - aI) - I = alpha A + beta I with B = op_scale A + op_shift I.
  FilterPlan p;
  const double c1 = 2.0 / (b - a);
  p.alpha = c1 * op_scale;
  p.beta = c1 * (op_shift - a) - 1.0;
  p.degree = degree;
  for (int i = 0; i <= degree && i < 64; ++i) p.coef[i] = coef[i];
  return p;
}

// Clenshaw's recurrence for Y = sum_k c_k T_k(S) X~ (X~ = X diag(xs)):
//   b_{d-1} = c_{d-1} X~ + 2 S (c_d X~)
//   b_j     = c_j X~ + 2 S b_{j+1} - b_{j+2}      (j = d-2 .. 1; b_d = c_d X~)
//   Y       = c_0 X~ + S b_1 - b_2
// Each line is one fused pass of spmm_fused (one product with A); b_j overwrites b_{j+2}
// in place, so two work blocks suffice.  The same polynomial psi_d of Section 5 is
// evaluated as Algorithm 7 does in the monomial basis, but with bounded coefficients.
template <typename T>
arb_status filter_apply(arb_ctx ctx, arb_mat mat, const FilterPlan& plan, const T* X, int64_t ldx,
                        int32_t ncols, const double* xscale, T* W1, T* W2, int64_t ldw, T* Y,
                        int64_t ldy, double* colss, T** result) {
  const int d = plan.degree;
  if (d < 1 || d > 60) return set_error(ctx, ARB_INVALID_ARG, "filter: degree must be in [1, 60]");
  if (ncols <= 0) return ARB_OK;
  double* table;
  ARB_TRY(ws<double>(ctx, WS_COEF, static_cast<size_t>(3) * d * ncols, &table));
  ChebCoef cc;
  for (int i = 0; i < 64; ++i) cc.c[i] = (i <= d) ? plan.coef[i] : 0.0;
  {
    const int64_t cnt = static_cast<int64_t>(d) * ncols;
    filter_table_kernel<<<static_cast<int>((cnt + 255) / 256), 256, 0, ctx->stream>>>(d, cc, xscale, ncols,
                                                                                    table);
    ARB_LAUNCHED(ctx);
  }
  auto sy_of = [&](int t) { return table + (3 * static_cast<int64_t>(t) + 0) * ncols; };
  auto sx_of = [&](int t) { return table + (3 * static_cast<int64_t>(t) + 1) * ncols; };
  auto sz_of = [&](int t) { return table + (3 * static_cast<int64_t>(t) + 2) * ncols; };

  if constexpr (std::is_same<T, float>::value) ARB_TRY(ensure_val32(ctx, mat));
  if constexpr (std::is_same<T, df2>::value) ARB_TRY(ensure_valdf(ctx, mat));
  SpmmArgs<T> a;
  a.A = mat;
  a.ncols = ncols;
  a.alpha = plan.alpha;
  a.beta = plan.beta;
  if (d == 1) {
    a.Yin = X;
    a.ldy = ldx;
    a.sy = sy_of(0);
    if (cc.c[0] != 0.0) {
      a.X = X;
      a.ldx = ldx;
      a.sx = sx_of(0);
    }
    T* out = Y ? Y : W1;
    a.out = out;
    a.ldo = Y ? ldy : ldw;
    a.colred = colss;
    ARB_TRY(spmm_fused(ctx, a));
    if (result) *result = out;
    return ARB_OK;
  }
  // step 0: b_{d-1} -> W1
  a.Yin = X;
  a.ldy = ldx;
  a.sy = sy_of(0);
  if (cc.c[d - 1] != 0.0) {
    a.X = X;
    a.ldx = ldx;
    a.sx = sx_of(0);
  }
  a.out = W1;
  a.ldo = ldw;
  ARB_TRY(spmm_fused(ctx, a));
  T* cur = W1;        // holds b_{j+1}
  T* prev = nullptr;  // holds b_{j+2}; nullptr means b_d = c_d X~ (read from X)
  for (int t = 1; t < d; ++t) {
    const int j = d - 1 - t;
    const bool last = (t == d - 1);
    SpmmArgs<T> s;
    s.A = mat;
    s.ncols = ncols;
    s.alpha = plan.alpha;
    s.beta = plan.beta;
    s.Yin = cur;
    s.ldy = ldw;
    s.sy = sy_of(t);
    if (cc.c[j] != 0.0) {
      s.X = X;
      s.ldx = ldx;
      s.sx = sx_of(t);
    }
    if (prev) {
      s.Z = prev;
      s.ldz = ldw;
    } else if (cc.c[d] != 0.0) {
      s.Z = X;
      s.ldz = ldx;
    }
    if (s.Z) s.sz = sz_of(t);
    T* out;
    int64_t ldo;
    if (last && Y) {
      out = Y;
      ldo = ldy;
    } else {
      out = prev ? prev : W2;
      ldo = ldw;
    }
    s.out = out;
    s.ldo = ldo;
    if (last) s.colred = colss;
    ARB_TRY(spmm_fused(ctx, s));
    prev = cur;
    cur = out;
  }
  if (result) *result = cur;
  return ARB_OK;
}

template <typename T>
arb_status project_out(arb_ctx ctx, int64_t n, const T* Q, int64_t ldq, int32_t nq, T* X, int64_t ldx,
                       int32_t ncols) {
  if (nq <= 0 || ncols <= 0) return ARB_OK;
  double* W;
  ARB_TRY(ws<double>(ctx, WS_SMALL3, static_cast<size_t>(nq) * ncols, &W));
  ARB_TRY(gram<T>(ctx, n, Q, ldq, nq, X, ldx, ncols, W, ncols));
  ARB_TRY(gemm_tall<T>(ctx, n, Q, ldq, nq, W, ncols, ncols, -1.0, 1.0, X, ldx));
  return ARB_OK;
}

// One eigen-truncated Gram pass (SVQB, Stathopoulos & Wu 2002): scale the columns of Z to
// unit norm, G = D Z^T Z D = W Theta W^T, keep theta_j > tau theta_0, and map
// Z -> Z D W_r Theta_r^{-1/2}.
template <typename T>
static arb_status svqb_pass(arb_ctx ctx, int64_t n, const T* Z, int64_t ldz, int32_t m, T* out, int64_t ldo,
                            int32_t* rank, bool have_gram = false) {
  double *G, *Gh, *W, *d, *theta;
  int32_t* r_dev;
  const size_t mm = static_cast<size_t>(m) * m;
  ARB_TRY(ws<double>(ctx, WS_SMALL0, mm, &G));
  ARB_TRY(ws<double>(ctx, WS_SMALL1, mm, &Gh));
  ARB_TRY(ws<double>(ctx, WS_SMALL2, mm, &W));
  ARB_TRY(ws<double>(ctx, WS_VEC0, m, &d));
  ARB_TRY(ws<double>(ctx, WS_VEC1, m, &theta));
  ARB_TRY(ws<int32_t>(ctx, WS_INT0, 4, &r_dev));
  if (!have_gram) ARB_TRY(gram<T>(ctx, n, Z, ldz, m, Z, ldz, m, G, m));  // else G = Z^T Z already
  ARB_TRY(svqb_prep(ctx, m, G, m, Gh, d));
  ARB_TRY(syevj(ctx, m, Gh, m, theta, W, m, nullptr, jac_tol<T>(ctx), jac_df<T>(ctx)));
  ARB_TRY(svqb_finish(ctx, m, theta, W, m, d, orth_tau<T>(m), Gh, r_dev));
  int32_t r = 0;
  ARB_TRY(d2h_sync(ctx, &r, r_dev, sizeof(int32_t)));
  *rank = r;
  if (r > 0) ARB_TRY(gemm_tall<T>(ctx, n, Z, ldz, m, Gh, m, r, 1.0, 0.0, out, ldo));
  return ARB_OK;
}

// ARB_TRACE set in the environment: one line per orthonormalisation on stderr
inline bool orth_trace() {
  static const bool on = getenv("ARB_TRACE") != nullptr;
  return on;
}

// One CholeskyQR pass: G = Z^T Z, D = diag(G)^{-1/2}, D G D = R^T R (FP64 Cholesky whose
// pivots must exceed thr), out = Z D R^{-1}.  With rank_test the pass also requires the
// 1-norm reciprocal condition number of D G D, from its Cholesky factor, to exceed thr: a
// symmetric matrix's 2-norm condition number is at most its 1-norm one, so the block is then
// one whose eigen-truncated Gram pass would keep every direction.  *ok = false when the
// factorisation broke down or the test failed; out is then not written, and G (the
// WS_SMALL0 workspace) still holds Z^T Z.
template <typename T>
static arb_status cholqr_pass(arb_ctx ctx, int64_t n, const T* Z, int64_t ldz, int32_t m, T* out, int64_t ldo,
                              double thr, bool rank_test, bool* ok) {
  double *G, *Gh, *M, *d;
  int32_t* status;
  const size_t mm = static_cast<size_t>(m) * m;
  ARB_TRY(ws<double>(ctx, WS_SMALL0, mm, &G));
  ARB_TRY(ws<double>(ctx, WS_SMALL1, mm, &Gh));
  ARB_TRY(ws<double>(ctx, WS_SMALL2, mm, &M));
  ARB_TRY(ws<double>(ctx, WS_VEC0, m, &d));
  ARB_TRY(ws<int32_t>(ctx, WS_CHOL_STATUS, 4, &status));
  ARB_TRY(gram<T>(ctx, n, Z, ldz, m, Z, ldz, m, G, m));
  ARB_TRY(svqb_prep(ctx, m, G, m, Gh, d));
  const double* factor = Gh;
  int64_t ldf = m;
  if (rank_test) {
    double *R, *Rinv, *rc_dev;
    ARB_TRY(ws<double>(ctx, WS_CHOL_R, mm, &R));
    ARB_TRY(ws<double>(ctx, WS_CHOL_RINV, mm, &Rinv));
    ARB_TRY(ws<double>(ctx, WS_VEC1, 2, &rc_dev));
    ARB_TRY(rcond_from_cholesky(ctx, m, Gh, m, R, Rinv, M, status, rc_dev));  // M: scratch for G^{-1}
    int32_t st[2] = {0, 0};
    double rc = 0.0;
    ARB_TRY(d2h_sync(ctx, st, status, sizeof(st)));
    ARB_TRY(d2h_sync(ctx, &rc, rc_dev, sizeof(double)));
    *ok = st[0] == 0 && rc > thr;
    if (orth_trace()) fprintf(stderr, "[arb]   cholqr m %d rcond %.3e (threshold %.1e) %s\n", m, rc, thr, *ok ? "kept" : "-> gram passes");
    if (!*ok) return ARB_OK;
    factor = R;
  } else {
    ARB_TRY(cholesky_upper(ctx, m, Gh, m, thr, status));
  }
  ARB_TRY(triangular_inverse(ctx, m, factor, ldf, d, M, status));
  int32_t st[2] = {0, 0};
  ARB_TRY(d2h_sync(ctx, st, status, sizeof(st)));
  *ok = st[0] == 0;
  if (*ok) ARB_TRY(gemm_tall<T>(ctx, n, Z, ldz, m, M, m, m, 1.0, 0.0, out, ldo));
  return ARB_OK;
}

// 1 (default): CholeskyQR2 first for well-conditioned blocks; 0: eigen-truncated Gram
// passes only.  The passes cut Gram eigenvalues below 64 m u of the largest, i.e. singular
// values below ~1e-6 of the largest, where a QR (the oracle's) keeps them to ~1e-13: on a
// 1600-row diffusion operator (k = 16, tol 1e-9, FP64) the passes-only form stalled at
// maxres 1.2e-9 after 8 outer iterations where the oracle and the CholeskyQR2-first form
// converge in 4-5.  Dropping those directions is cheaper where it does not hurt: per solve,
// CholeskyQR2 first / passes only, 128^3 mixed 11.1 s / 10.0 s; Chung-Lu n = 1e6, k = 500
// FP64 55.8 s / 56.8 s, mixed 94.0 s / 56.1 s.
#ifndef ARB_ORTH_CHOLQR
#define ARB_ORTH_CHOLQR 1
#endif

template <typename T>
arb_status orth(arb_ctx ctx, int64_t n, const T* Z, int64_t ldz, int32_t m, T* U, int64_t ldu, T* tmp,
                int64_t ldt, int32_t* rank, bool recover) {
  *rank = 0;
  if (m <= 0) return ARB_OK;
  // CholeskyQR2 (ARB_ORTH_CHOLQR = 1): two Cholesky passes when the unit-diagonal Gram
  // matrix's reciprocal condition number (from its factor) is above max(the Gram pass's
  // truncation threshold, 1e-8) - a well-conditioned block - and the second Gram matrix is
  // near the identity (every pivot above 1/2).  Otherwise the eigen-truncated Gram passes
  // below take over and decide the rank, from the first pass's Gram matrix when that one
  // failed.  A CholeskyQR2 that only asked for positive pivots made the 128^3 mixed solve
  // take an extra FP32 outer iteration (13.0 s per solve).
  bool have_gram = false;
  if (m <= cholesky_max_order() && ARB_ORTH_CHOLQR) {
    bool ok1 = false, ok2 = false;
    ARB_TRY(cholqr_pass<T>(ctx, n, Z, ldz, m, tmp, ldt, std::max(orth_tau<T>(m), 1e-8), true, &ok1));
    if (ok1) ARB_TRY(cholqr_pass<T>(ctx, n, tmp, ldt, m, U, ldu, 0.5, false, &ok2));
    if (ok2) {
      *rank = m;
      return ARB_OK;
    }
    have_gram = !ok1;
  }
  int32_t r1 = 0, r2 = 0;
  ARB_TRY(svqb_pass<T>(ctx, n, Z, ldz, m, tmp, ldt, &r1, have_gram));
  if (r1 == 0) return ARB_OK;
  ARB_TRY(svqb_pass<T>(ctx, n, tmp, ldt, r1, U, ldu, &r2));
  int32_t r = r2;
  if (orth_trace()) fprintf(stderr, "[arb]   gram passes m %d rank %d / %d\n", m, r1, r2);
  // A Gram pass resolves singular values down to ~sqrt(tau) of the largest.  A filtered
  // block can span far more (one isolated extreme eigenvalue amplified by the filter), and
  // the directions the passes dropped are then the ones still to converge.  Recover them:
  // the residual Z - U U^T Z (projected twice) keeps each column's part outside the basis;
  // its columns above rounding level (64 m u of the largest column of Z), largest first
  // and at most m - r, are orthonormalised and appended.
  if (recover && r < m) {
    double* nrm;
    int32_t* idx;
    ARB_TRY(ws<double>(ctx, WS_ORTH_NORM, static_cast<size_t>(m), &nrm));
    std::vector<double> zn(m), rn(m);
    ARB_TRY(col_norms2<T>(ctx, n, Z, ldz, m, nrm));
    ARB_TRY(d2h_sync(ctx, zn.data(), nrm, m * sizeof(double)));
    const double zmax = std::sqrt(*std::max_element(zn.begin(), zn.end()));
    const double thr = 64.0 * m * (sizeof(T) == 4 ? 6e-8 : 1.11e-16) * zmax;
    for (int round = 0; round < 2 && r < m; ++round) {
      ARB_TRY((copy_block<T, T>(ctx, n, Z, ldz, m, tmp, ldt)));
      for (int pass = 0; pass < 2; ++pass) ARB_TRY(project_out<T>(ctx, n, U, ldu, r, tmp, ldt, m));
      ARB_TRY(col_norms2<T>(ctx, n, tmp, ldt, m, nrm));
      ARB_TRY(d2h_sync(ctx, rn.data(), nrm, m * sizeof(double)));
      std::vector<int32_t> keep;
      for (int32_t j = 0; j < m; ++j)
        if (std::sqrt(rn[j]) > thr) keep.push_back(j);
      if (keep.empty()) break;
      std::stable_sort(keep.begin(), keep.end(), [&](int32_t a, int32_t b) { return rn[a] > rn[b]; });
      if (static_cast<int32_t>(keep.size()) > m - r) keep.resize(m - r);
      const int32_t ns = static_cast<int32_t>(keep.size());
      ARB_TRY(ws<int32_t>(ctx, WS_ORTH_IDX, static_cast<size_t>(ns), &idx));
      ARB_CUDA(ctx, cudaMemcpyAsync(idx, keep.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
      ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      ARB_TRY(gather_cols<T>(ctx, n, tmp, ldt, idx, ns, U + r, ldu));  // columns r .. r+ns-1 of U
      int32_t ra = 0, rb = 0;
      ARB_TRY(svqb_pass<T>(ctx, n, U + r, ldu, ns, tmp, ldt, &ra));
      if (ra == 0) break;
      for (int pass = 0; pass < 2; ++pass) ARB_TRY(project_out<T>(ctx, n, U, ldu, r, tmp, ldt, ra));
      ARB_TRY(svqb_pass<T>(ctx, n, tmp, ldt, ra, U + r, ldu, &rb));
      if (rb == 0) break;
      r += rb;
    }
  }
  *rank = r;
  return ARB_OK;
}

template <typename T>
arb_status rcond_gram(arb_ctx ctx, int64_t n, const T* X, int64_t ldx, int32_t ncols, const double* xs,
                      double* rc) {
  double *G, *R, *Rinv, *Ginv, *rc_dev;
  int32_t* status;
  const size_t mm = static_cast<size_t>(ncols) * ncols;
  ARB_TRY(ws<double>(ctx, WS_SMALL0, mm, &G));
  ARB_TRY(ws<double>(ctx, WS_CHOL_R, mm, &R));
  ARB_TRY(ws<double>(ctx, WS_CHOL_RINV, mm, &Rinv));
  ARB_TRY(ws<double>(ctx, WS_SMALL2, mm, &Ginv));
  ARB_TRY(ws<double>(ctx, WS_VEC1, 2, &rc_dev));
  ARB_TRY(ws<int32_t>(ctx, WS_CHOL_STATUS, 4, &status));
  ARB_TRY(gram<T>(ctx, n, X, ldx, ncols, X, ldx, ncols, G, ncols));
  if (xs) ARB_TRY(scale_sym(ctx, ncols, G, ncols, xs));
  if (ncols <= cholesky_max_order()) {
    // G^{-1} from the Cholesky factor (as the oracle computes it); rc = 0 when G is not
    // numerically positive definite
    ARB_TRY(rcond_from_cholesky(ctx, ncols, G, ncols, R, Rinv, Ginv, status, rc_dev));
  } else {
    double *W, *theta;
    ARB_TRY(ws<double>(ctx, WS_SMALL1, mm, &W));
    ARB_TRY(ws<double>(ctx, WS_VEC2, ncols, &theta));
    ARB_TRY(syevj(ctx, ncols, G, ncols, theta, W, ncols, nullptr, jac_tol<T>(ctx), jac_df<T>(ctx)));
    ARB_TRY(rcond_from_eig(ctx, ncols, G, ncols, theta, W, ncols, rc_dev));
  }
  ARB_TRY(d2h_sync(ctx, rc, rc_dev, sizeof(double)));
  return ARB_OK;
}

// span[X, BX, ..., B^q X] as an orthonormal block Krylov basis: U_0 = orth(X); for
// i = 1..q, W = B U_{i-1} (kept as the block AU_{i-1}), W is projected against Q_c and
// U_0..U_{i-1} twice (block classical Gram-Schmidt with reorthogonalisation), and
// U_i = orth(W).  In exact arithmetic span{U_0..U_q} = span{X, BX, ..., B^q X} of
// Algorithm 5; building it block by block keeps the small residual directions that
// columns of [X, BX, ...] carry at full relative accuracy.  Then AU_q = B U_q and
// H = U^T (B U) (Algorithm 1) is formed from its block-tridiagonal part and diagonalised.
template <typename T>
arb_status arr_basis_and_eig(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, int64_t n, T* X,
                             int64_t ldx, int32_t w, const T* Qc, int64_t ldqc, int32_t nl, int32_t q,
                             const ArrWork<T>& wk, int32_t* m_out, double* theta, double* V) {
  *m_out = 0;
  if (q > 15) return set_error(ctx, ARB_INVALID_ARG, "ARR: at most 15 augmentation blocks");
  if (sizeof(T) == 4) ARB_TRY(ensure_val32(ctx, mat));
  if (nl > 0) ARB_TRY(project_out<T>(ctx, n, Qc, ldqc, nl, X, ldx, w));
  int32_t r0 = 0;
  // FP32 blocks resolve no more than their Gram pass does (the recovery threshold 64 m u32
  // of the largest column is about the pass's own cut), so only FP64 bases recover
  ARB_TRY(orth(ctx, n, static_cast<const T*>(X), ldx, w, wk.U, wk.ldu, wk.T1, wk.ldt, &r0,
               std::is_same<T, double>::value));
  if (r0 == 0) return set_error(ctx, ARB_BREAKDOWN, "ARR: iterate has no numerical rank");
  std::vector<int32_t> off{0}, rk{r0};
  int32_t m = r0;
  for (int i = 1; i <= q; ++i) {
    const int32_t o = off.back(), r = rk.back();
    SpmmArgs<T> s;
    s.A = mat;
    s.ncols = r;
    s.Yin = wk.U + o;
    s.ldy = wk.ldu;
    s.alpha = op_scale;
    s.beta = op_shift;
    s.out = wk.AU + o;
    s.ldo = wk.ldau;
    ARB_TRY(spmm_fused(ctx, s));
    ARB_TRY((copy_block<T, T>(ctx, n, wk.AU + o, wk.ldau, r, wk.T2, wk.ldt2)));
    for (int pass = 0; pass < 2; ++pass) {
      if (nl > 0) ARB_TRY(project_out<T>(ctx, n, Qc, ldqc, nl, wk.T2, wk.ldt2, r));
      ARB_TRY(project_out<T>(ctx, n, wk.U, wk.ldu, m, wk.T2, wk.ldt2, r));
    }
    int32_t ri = 0;
    ARB_TRY(orth(ctx, n, static_cast<const T*>(wk.T2), wk.ldt2, r, wk.U + m, wk.ldu, wk.T1, wk.ldt, &ri));
    if (ri == 0) break;  // the Krylov space is exhausted
    off.push_back(m);
    rk.push_back(ri);
    m += ri;
  }
  {
    // B U for the last block (the earlier blocks were formed during the augmentation)
    const int32_t o = off.back(), r = rk.back();
    SpmmArgs<T> s;
    s.A = mat;
    s.ncols = r;
    s.Yin = wk.U + o;
    s.ldy = wk.ldu;
    s.alpha = op_scale;
    s.beta = op_shift;
    s.out = wk.AU + o;
    s.ldo = wk.ldau;
    ARB_TRY(spmm_fused(ctx, s));
  }
  // H = U^T (B U) is block tridiagonal for this basis: B U_i lies in span{U_0..U_{i+1}}
  // up to the directions orth truncated (below its threshold), so only the blocks
  // H_ii and H_{i,i+1} are formed (H_{i+1,i} = H_{i,i+1}^T, the rest zero) - 3q+1 of the
  // (q+1)^2 block products of the full U^T (BU)
  double* H;
  ARB_TRY(ws<double>(ctx, WS_SMALL0, static_cast<size_t>(m) * m, &H));
  ARB_TRY(fill(ctx, H, static_cast<int64_t>(m) * m, 0.0));
  const int nblk = static_cast<int>(off.size());
  for (int bi = 0; bi < nblk; ++bi) {
    for (int bj = bi; bj < std::min(nblk, bi + 2); ++bj) {
      double* Hij = H + static_cast<size_t>(off[bi]) * m + off[bj];
      ARB_TRY(gram<T>(ctx, n, wk.U + off[bi], wk.ldu, rk[bi], wk.AU + off[bj], wk.ldau, rk[bj], Hij, m));
    }
  }
  ARB_TRY(symmetrize_upper_blocks(ctx, m, H, m, off.data(), rk.data(), nblk));
  ARB_TRY(syevj(ctx, m, H, m, theta, V, m, nullptr, jac_tol<T>(ctx), jac_df<T>(ctx)));
  *m_out = m;
  return ARB_OK;
}

template arb_status filter_apply<double>(arb_ctx, arb_mat, const FilterPlan&, const double*, int64_t, int32_t,
                                         const double*, double*, double*, int64_t, double*, int64_t, double*,
                                         double**);
template arb_status filter_apply<float>(arb_ctx, arb_mat, const FilterPlan&, const float*, int64_t, int32_t,
                                        const double*, float*, float*, int64_t, float*, int64_t, double*, float**);
template arb_status filter_apply<df2>(arb_ctx, arb_mat, const FilterPlan&, const df2*, int64_t, int32_t, const double*,
                                      df2*, df2*, int64_t, df2*, int64_t, double*, df2**);
template arb_status orth<double>(arb_ctx, int64_t, const double*, int64_t, int32_t, double*, int64_t, double*,
                                 int64_t, int32_t*, bool);
template arb_status orth<float>(arb_ctx, int64_t, const float*, int64_t, int32_t, float*, int64_t, float*,
                                int64_t, int32_t*, bool);
template arb_status rcond_gram<double>(arb_ctx, int64_t, const double*, int64_t, int32_t, const double*, double*);
template arb_status rcond_gram<float>(arb_ctx, int64_t, const float*, int64_t, int32_t, const double*, double*);
template arb_status project_out<double>(arb_ctx, int64_t, const double*, int64_t, int32_t, double*, int64_t,
                                        int32_t);
template arb_status project_out<float>(arb_ctx, int64_t, const float*, int64_t, int32_t, float*, int64_t, int32_t);
template arb_status arr_basis_and_eig<double>(arb_ctx, arb_mat, double, double, int64_t, double*, int64_t,
                                              int32_t, const double*, int64_t, int32_t, int32_t,
                                              const ArrWork<double>&, int32_t*, double*, double*);
template arb_status arr_basis_and_eig<float>(arb_ctx, arb_mat, double, double, int64_t, float*, int64_t, int32_t,
                                             const float*, int64_t, int32_t, int32_t, const ArrWork<float>&,
                                             int32_t*, double*, double*);

}  // namespace arb
