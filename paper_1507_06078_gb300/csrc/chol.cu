// FP64 Cholesky factorisation and triangular inverse of small symmetric positive definite
// matrices on the device: the factor step of CholeskyQR (orth(Z) of Algorithm 1 as
// G = Z^T Z = R^T R, U = Z R^{-1}) and the inverse behind rcond(X^T X) of the inner stop
// rule (eq. inn-stop).  G is m x m, row-major; only its upper triangle is read.
//
// Blocked right-looking factorisation with panels of 32 columns, three launches per
// panel, all on the context's stream with no host synchronisation:
//   1. the 32 x 32 diagonal block is factored in shared memory by one CTA (pivots checked
//      against a threshold; a breakdown sets a device status word that every later kernel
//      reads first), and its triangular inverse is formed there too;
//   2. the panel's block row to the right is solved with that inverse (R_kj = R_kk^{-T} A_kj);
//   3. the trailing upper triangle is updated, A_ij -= R_ki^T R_kj, one 32 x 32 tile per CTA.
// The inverse of the whole factor is then one warp per column (back substitution with
// warp-wide dot products).
#include <algorithm>
#include <cmath>

#include "arb_internal.h"

namespace arb {
namespace {

constexpr int CB = 32;  // panel width

__global__ void __launch_bounds__(256) potrf_diag_kernel(int m, double* __restrict__ A, int64_t lda, int k0,
                                                         double thr, double* __restrict__ tinv,
                                                         int32_t* __restrict__ status) {
  __shared__ double s[CB][CB + 1];
  __shared__ double t[CB][CB + 1];
  __shared__ int bad;
  if (*status) return;
  const int kb = min(CB, m - k0);
  const int tid = threadIdx.x;
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int i = e / CB, j = e % CB;
    double v = 0.0;
    if (i < kb && j < kb) {
      const int a = min(i, j), b = max(i, j);
      v = A[static_cast<int64_t>(k0 + a) * lda + k0 + b];
    }
    s[i][j] = v;
    t[i][j] = 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      const double d = s[j][j];
      if (!(d > thr) || !isfinite(d)) {
        bad = 1;
        status[0] = 1;
        status[1] = k0 + j;
      }
      s[j][j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    if (bad) return;  // shared: the whole CTA leaves together
    const double r = s[j][j];
    for (int c = j + 1 + tid; c < kb; c += blockDim.x) s[j][c] /= r;
    __syncthreads();
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      const int a = e / kb, b = e % kb;
      if (a > j && b >= a) s[a][b] -= s[j][a] * s[j][b];
    }
    __syncthreads();
  }
  // T = R_kk^{-1} (upper), one column per thread: T_cc = 1 / R_cc and, upwards,
  // T_ic = -(sum_{l = i+1..c} R_il T_lc) / R_ii
  if (tid < kb) {
    const int c = tid;
    t[c][c] = 1.0 / s[c][c];
    for (int i = c - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int l = i + 1; l <= c; ++l) acc = fma(s[i][l], t[l][c], acc);
      t[i][c] = -acc / s[i][i];
    }
  }
  __syncthreads();
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    if (j >= i) A[static_cast<int64_t>(k0 + i) * lda + k0 + j] = s[i][j];
    tinv[i * CB + j] = t[i][j];
  }
}

// R_kj = T^T A_kj for the columns right of the panel: each CTA takes 8 columns, thread
// (a, c) forms sum_{b <= a} T_ba A_{k0+b, j}.
__global__ void __launch_bounds__(256) trsm_panel_kernel(int m, double* __restrict__ A, int64_t lda, int k0,
                                                         const double* __restrict__ tinv,
                                                         const int32_t* __restrict__ status) {
  __shared__ double t[CB][CB + 1];
  __shared__ double col[CB][8];
  if (*status) return;
  const int kb = min(CB, m - k0);
  const int j0 = k0 + kb + blockIdx.x * 8;
  const int tid = threadIdx.x;
  for (int e = tid; e < CB * CB; e += blockDim.x) t[e / CB][e % CB] = tinv[e];
  const int a = tid / 8, c = tid % 8;
  const int j = j0 + c;
  col[a][c] = (a < kb && j < m) ? A[static_cast<int64_t>(k0 + a) * lda + j] : 0.0;
  __syncthreads();
  if (a < kb && j < m) {
    double acc = 0.0;
    for (int b = 0; b <= a; ++b) acc = fma(t[b][a], col[b][c], acc);
    A[static_cast<int64_t>(k0 + a) * lda + j] = acc;
  }
}

// Trailing update of the upper triangle: A_ij -= sum_a R_{k0+a, i} R_{k0+a, j} for
// i, j >= k0 + kb, j >= i; one 32 x 32 tile per CTA (tiles wholly below the diagonal exit).
__global__ void __launch_bounds__(256) syrk_trailing_kernel(int m, double* __restrict__ A, int64_t lda, int k0,
                                                            const int32_t* __restrict__ status) {
  __shared__ double pi[CB][CB + 1];
  __shared__ double pj[CB][CB + 1];
  if (*status) return;
  const int kb = min(CB, m - k0);
  const int base = k0 + kb;
  const int i0 = base + blockIdx.y * CB, j0 = base + blockIdx.x * CB;
  if (j0 + CB - 1 < i0) return;  // below the diagonal
  const int tid = threadIdx.x;
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int a = e / CB, x = e % CB;
    const bool ra = a < kb;
    pi[a][x] = (ra && i0 + x < m) ? A[static_cast<int64_t>(k0 + a) * lda + i0 + x] : 0.0;
    pj[a][x] = (ra && j0 + x < m) ? A[static_cast<int64_t>(k0 + a) * lda + j0 + x] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int x = e / CB, y = e % CB;
    const int i = i0 + x, j = j0 + y;
    if (i >= m || j >= m || j < i) continue;
    double acc = 0.0;
    for (int a = 0; a < kb; ++a) acc = fma(pi[a][x], pj[a][y], acc);
    A[static_cast<int64_t>(i) * lda + j] -= acc;
  }
}

// M = diag(d) R^{-1} (or R^{-1} when d is NULL) of the upper factor R (its upper triangle;
// m x m, row-major lda), M row-major m x m with zeros below the diagonal.  One warp per
// column j: x_j = 1 / R_jj, then upwards x_i = -(sum_{l > i} R_il x_l) / R_ii, the sum a
// warp-wide dot product over the row of R (coalesced), x kept in shared memory.
constexpr int TRINV_WARPS = 4;
__global__ void __launch_bounds__(TRINV_WARPS * 32) trinv_kernel(int m, const double* __restrict__ R, int64_t lda,
                                                                 const double* __restrict__ d,
                                                                 double* __restrict__ M,
                                                                 const int32_t* __restrict__ status) {
  extern __shared__ double sx[];  // [TRINV_WARPS][m]
  if (*status) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * TRINV_WARPS + warp;
  if (j >= m) return;
  double* x = sx + static_cast<size_t>(warp) * m;
  if (lane == 0) x[j] = 1.0 / R[static_cast<int64_t>(j) * lda + j];
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    const double* Ri = R + static_cast<int64_t>(i) * lda;
    double acc = 0.0;
    for (int l = i + 1 + lane; l <= j; l += 32) acc = fma(Ri[l], x[l], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[i] = -acc / Ri[i];
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) {
    const double v = i <= j ? x[i] * (d ? d[i] : 1.0) : 0.0;
    M[static_cast<int64_t>(i) * m + j] = v;
  }
}

// Ginv = Rinv Rinv^T (symmetric, both triangles written): entry (i, j), j >= i, is the dot
// product of rows i and j of the upper Rinv over k >= j.
__global__ void inverse_from_factor_kernel(int m, const double* __restrict__ Rinv, double* __restrict__ Ginv,
                                           const int32_t* __restrict__ status) {
  if (*status) return;
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(m) * m) return;
  const int i = static_cast<int>(t / m), j = static_cast<int>(t % m);
  if (j < i) return;
  const double* ri = Rinv + static_cast<int64_t>(i) * m;
  const double* rj = Rinv + static_cast<int64_t>(j) * m;
  double s = 0.0;
  for (int k = j; k < m; ++k) s = fma(ri[k], rj[k], s);
  Ginv[static_cast<int64_t>(i) * m + j] = s;
  Ginv[static_cast<int64_t>(j) * m + i] = s;
}

// rc = 1 / (||G||_1 ||G^{-1}||_1), 0 when the factorisation broke down
__global__ void rcond_chol_kernel(int m, const double* __restrict__ G, int64_t ldg, const double* __restrict__ Ginv,
                                  const int32_t* __restrict__ status, double* __restrict__ rc) {
  __shared__ double sg[256], si[256];
  const bool ok = *status == 0;
  double mg = 0.0, mi = 0.0;
  if (ok) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      double cg = 0.0, ci = 0.0;
      for (int i = 0; i < m; ++i) {
        cg += fabs(G[static_cast<int64_t>(i) * ldg + j]);
        ci += fabs(Ginv[static_cast<int64_t>(i) * m + j]);
      }
      mg = fmax(mg, cg);
      mi = fmax(mi, ci);
    }
  }
  sg[threadIdx.x] = mg;
  si[threadIdx.x] = mi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sg[threadIdx.x] = fmax(sg[threadIdx.x], sg[threadIdx.x + s]);
      si[threadIdx.x] = fmax(si[threadIdx.x], si[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double r = 0.0;
    if (ok && isfinite(si[0]) && si[0] > 0.0 && sg[0] > 0.0) r = 1.0 / (sg[0] * si[0]);
    *rc = r;
  }
}

// M[i][i] += s
__global__ void add_diagonal_kernel(int m, double* __restrict__ M, int64_t ldm, double s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) M[static_cast<int64_t>(i) * ldm + i] += s;
}

__global__ void clear_status_kernel(int32_t* status) {
  if (threadIdx.x < 2) status[threadIdx.x] = 0;
}

}  // namespace

int cholesky_max_order() { return 4096; }

arb_status cholesky_upper(arb_ctx ctx, int32_t m, double* A, int64_t lda, double thr, int32_t* status) {
  if (m <= 0) return ARB_OK;
  if (m > cholesky_max_order()) return set_error(ctx, ARB_INVALID_ARG, "cholesky: order too large");
  double* tinv;
  ARB_TRY(ws<double>(ctx, WS_CHOL, CB * CB, &tinv));
  clear_status_kernel<<<1, 32, 0, ctx->stream>>>(status);
  ARB_LAUNCHED(ctx);
  for (int k0 = 0; k0 < m; k0 += CB) {
    potrf_diag_kernel<<<1, 256, 0, ctx->stream>>>(m, A, lda, k0, thr, tinv, status);
    ARB_LAUNCHED(ctx);
    const int rest = m - std::min(m, k0 + CB);
    if (rest <= 0) break;
    trsm_panel_kernel<<<(rest + 7) / 8, 256, 0, ctx->stream>>>(m, A, lda, k0, tinv, status);
    ARB_LAUNCHED(ctx);
    const int tiles = (rest + CB - 1) / CB;
    syrk_trailing_kernel<<<dim3(tiles, tiles), 256, 0, ctx->stream>>>(m, A, lda, k0, status);
    ARB_LAUNCHED(ctx);
  }
  return ARB_OK;
}

arb_status triangular_inverse(arb_ctx ctx, int32_t m, const double* R, int64_t lda, const double* d, double* M,
                              const int32_t* status) {
  if (m <= 0) return ARB_OK;
  const size_t smem = static_cast<size_t>(TRINV_WARPS) * m * sizeof(double);
  if (smem > 48 * 1024) ARB_CUDA(ctx, cudaFuncSetAttribute(trinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           static_cast<int>(smem)));
  trinv_kernel<<<(m + TRINV_WARPS - 1) / TRINV_WARPS, TRINV_WARPS * 32, smem, ctx->stream>>>(m, R, lda, d, M, status);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status rcond_from_cholesky(arb_ctx ctx, int32_t m, const double* G, int64_t ldg, double* R, double* Rinv,
                               double* Ginv, int32_t* status, double* rc_dev) {
  ARB_CUDA(ctx, cudaMemcpy2DAsync(R, m * sizeof(double), G, ldg * sizeof(double), m * sizeof(double), m,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  ARB_TRY(cholesky_upper(ctx, m, R, m, 0.0, status));
  ARB_TRY(triangular_inverse(ctx, m, R, m, nullptr, Rinv, status));
  const int64_t mm = static_cast<int64_t>(m) * m;
  inverse_from_factor_kernel<<<static_cast<int>((mm + 255) / 256), 256, 0, ctx->stream>>>(m, Rinv, Ginv, status);
  ARB_LAUNCHED(ctx);
  rcond_chol_kernel<<<1, 256, 0, ctx->stream>>>(m, G, ldg, Ginv, status, rc_dev);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

}  // namespace arb

namespace arb {

arb_status spd_inverse(arb_ctx ctx, int32_t m, const double* G, int64_t ldg, double* R, double* Rinv, double* Ginv,
                       int32_t* status) {
  ARB_CUDA(ctx, cudaMemcpy2DAsync(R, m * sizeof(double), G, ldg * sizeof(double), m * sizeof(double), m,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  ARB_TRY(cholesky_upper(ctx, m, R, m, 0.0, status));
  ARB_TRY(triangular_inverse(ctx, m, R, m, nullptr, Rinv, status));
  const int64_t mm = static_cast<int64_t>(m) * m;
  inverse_from_factor_kernel<<<static_cast<int>((mm + 255) / 256), 256, 0, ctx->stream>>>(m, Rinv, Ginv, status);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status add_diagonal(arb_ctx ctx, int32_t m, double* M, int64_t ldm, double s) {
  if (m <= 0) return ARB_OK;
  add_diagonal_kernel<<<(m + 127) / 128, 128, 0, ctx->stream>>>(m, M, ldm, s);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

}  // namespace arb
