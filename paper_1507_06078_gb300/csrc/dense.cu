// Dense FP64 kernels of the subspace step: tall-skinny Gram products X^T Y (inner stop
// rule eq. inn-stop, orth(Z) and H = U^T A U of Algorithm 1), tall-skinny products
// X W (projection X - Q_c(Q_c^T X) of Algorithm 8, basis change in orth, Ritz rotation
// Y = U V of Algorithm 1), and the small helpers around the dense eigensolver.
//
// GB300 executes FP64 at a small fraction of its FP32/tensor rate, so these FP64 kernels
// are bound by the FP64 pipe; they are register-tiled (4x4 outputs per thread, operands
// staged in shared memory) so that the pipe, not memory, is the limit.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "arb_internal.h"
#include "df_arith.cuh"

namespace arb {
namespace {

constexpr int KSTEP = 16;

// part[s][i][j] = sum over the rows of split s of X[r][i] * Y[r][j].  One (16R)x(16R) tile
// per CTA of 256 threads, each thread owning R x R outputs strided by 16 (R = 1, 2, 4 so
// that small blocks do not pay for a 64-wide tile of FP64 multiply-adds).  For FP32
// inputs the products are summed in FP32 over runs of 64 rows and the run sums in FP64:
// a run's rounding error is ~64 u32 of its own (short) sum, so an n-row Gram entry is
// accurate to ~64 u32 / sqrt(n) relative (~3e-9 at n = 2M) instead of ~u32 sqrt(n).
template <typename T, int R>
__global__ void __launch_bounds__(256)
gram_kernel(int64_t n, const T* __restrict__ X, int64_t ldx, int na, const T* __restrict__ Y,
            int64_t ldy, int nb, int64_t rows_per_split, int symmetric, double* __restrict__ part) {
  constexpr int TT = 16 * R;
  constexpr int FLUSH = 4;  // k-steps (of 16 rows) per FP32 run
  const int ti = blockIdx.x, tj = blockIdx.y, s = blockIdx.z;
  if (symmetric && tj < ti) return;
  __shared__ T Xs[KSTEP][TT + 1];
  __shared__ T Ys[KSTEP][TT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = ti * TT, j0 = tj * TT;
  const int64_t r0 = s * rows_per_split;
  const int64_t r1 = min(n, r0 + rows_per_split);
  double acc[R][R] = {};
  T accT[R][R] = {};
  int steps = 0;
  for (int64_t rb = r0; rb < r1; rb += KSTEP) {
    for (int t = threadIdx.x; t < KSTEP * TT; t += 256) {
      const int rr = t / TT, cc = t % TT;
      const int64_t r = rb + rr;
      const bool rok = r < r1;
      Xs[rr][cc] = (rok && i0 + cc < na) ? X[r * ldx + i0 + cc] : T(0);
      Ys[rr][cc] = (rok && j0 + cc < nb) ? Y[r * ldy + j0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KSTEP; ++k) {
      T a[R], b[R];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        a[u] = Xs[k][ty + 16 * u];
        b[u] = Ys[k][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < R; ++v) accT[u][v] = fma(a[u], b[v], accT[u][v]);
    }
    __syncthreads();
    if (sizeof(T) == 4 && ++steps == FLUSH) {
      steps = 0;
#pragma unroll
      for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < R; ++v) {
          acc[u][v] += static_cast<double>(accT[u][v]);
          accT[u][v] = T(0);
        }
    }
  }
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int v = 0; v < R; ++v) acc[u][v] += static_cast<double>(accT[u][v]);
  double* P = part + static_cast<size_t>(s) * na * nb;
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = i0 + ty + 16 * u;
    if (i >= na) continue;
#pragma unroll
    for (int v = 0; v < R; ++v) {
      const int j = j0 + tx + 16 * v;
      if (j < nb) P[static_cast<size_t>(i) * nb + j] = acc[u][v];
    }
  }
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int nsplit, int na, int nb,
                                   int symmetric, int tile, double* __restrict__ C, int64_t ldc) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<int64_t>(na) * nb) return;
  int i = static_cast<int>(idx / nb), j = static_cast<int>(idx % nb);
  int si = i, sj = j;
  // symmetric products: every entry below the diagonal takes its mirror's partial sums
  // (computed: the tiles with tj >= ti hold every i <= j), so C is exactly symmetric even
  // when the two orders of a product round differently
  if (symmetric && j < i) {
    si = j;
    sj = i;
  }
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[static_cast<size_t>(k) * na * nb + static_cast<size_t>(si) * nb + sj];
  C[static_cast<int64_t>(i) * ldc + j] = s;
}

// w <- w - a v - b u (the three-term recurrence of Lanczos)
__global__ void lin3_kernel(int64_t n, double* __restrict__ w, double a, const double* __restrict__ v, double b,
                            const double* __restrict__ u) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) w[i] = w[i] - a * v[i] - b * u[i];
}

__global__ void scale_vec_kernel(int64_t n, double* __restrict__ dst, const double* __restrict__ src, double s) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) dst[i] = src[i] * s;
}

// Out[r][c] = alpha * sum_k In[r][k] W[k][c] + beta * Out[r][c]; a 64 x (16 RN) output tile
// per CTA, each thread owning 4 x RN outputs; W (FP64) is rounded to T as it is staged.
template <typename T, int RN>
__global__ void __launch_bounds__(256)
gemm_tall_kernel(int64_t n, const T* __restrict__ In, int64_t ldi, int na, const double* __restrict__ W,
                 int64_t ldw, int nb, T alpha, T beta, T* __restrict__ Out, int64_t ldo) {
  constexpr int TR = 64, TC = 16 * RN;
  __shared__ T Is[KSTEP][TR + 1];
  __shared__ T Ws[KSTEP][TC + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * TR;
  const int c0 = blockIdx.y * TC;
  T acc[4][RN] = {};
  for (int k0 = 0; k0 < na; k0 += KSTEP) {
    for (int t = threadIdx.x; t < KSTEP * TR; t += 256) {
      const int kk = t % KSTEP, rr = t / KSTEP;
      const int64_t r = r0 + rr;
      Is[kk][rr] = (r < n && k0 + kk < na) ? In[r * ldi + k0 + kk] : T(0);
    }
    for (int t = threadIdx.x; t < KSTEP * TC; t += 256) {
      const int kw = t / TC, cw = t % TC;
      Ws[kw][cw] = (k0 + kw < na && c0 + cw < nb) ? static_cast<T>(W[static_cast<int64_t>(k0 + kw) * ldw + c0 + cw])
                                                  : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KSTEP; ++k) {
      T a[4], b[RN];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Is[k][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < RN; ++v) b[v] = Ws[k][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < RN; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t r = r0 + ty + 16 * u;
    if (r >= n) continue;
#pragma unroll
    for (int v = 0; v < RN; ++v) {
      const int c = c0 + tx + 16 * v;
      if (c >= nb) continue;
      T* o = Out + r * ldo + c;
      const T val = alpha * acc[u][v];
      *o = (beta == T(0)) ? val : fma(beta, *o, val);
    }
  }
}

// ---------------------------------------------------------------- double-float products
// The FP64 Gram and tall-skinny products of a context in double-float mode: operands are
// split into (hi, lo) FP32 pairs as they are staged in shared memory (split_f64, integer
// operations only), products and sums run on the FP32 pipe by Dot2 (dot2p, two outputs per
// packed instruction), and every 64 terms the compensated pair is folded into a running
// double-float sum.  Results are written in FP64.  GB300 executes FP64 at about 1/64 of
// its FP32 rate; these kernels trade ~12 FP32 operations per multiply-add for that.
constexpr int DF_FOLD = 4;  // k-steps of 16 terms per fold into the running sum

// running double-float sum (Ah, Al) += (S + E), two outputs at once; S = E = 0 after
__device__ __forceinline__ void df_fold(float2& Ah, float2& Al, float2& S, float2& E) {
  const dfp t = fast_two_sum2(S, E);
  const float2 s = __fadd2_rn(Ah, t.hi);
  const float2 bb = sub2(s, Ah);
  const float2 err = __fadd2_rn(sub2(Ah, sub2(s, bb)), sub2(t.hi, bb));
  const dfp r = fast_two_sum2(s, __fadd2_rn(err, __fadd2_rn(Al, t.lo)));
  Ah = r.hi;
  Al = r.lo;
  S = make_float2(0.f, 0.f);
  E = make_float2(0.f, 0.f);
}

// part[s][i][j] = sum over the rows of split s of X[r][i] * Y[r][j] (the tiling of
// gram_kernel; R >= 2 so that a thread's outputs pair up along j).
template <int R>
__global__ void __launch_bounds__(256)
gram_df_kernel(int64_t n, const double* __restrict__ X, int64_t ldx, int na, const double* __restrict__ Y,
               int64_t ldy, int nb, int64_t rows_per_split, int symmetric, double* __restrict__ part) {
  constexpr int TT = 16 * R, H = R / 2;
  const int ti = blockIdx.x, tj = blockIdx.y, s = blockIdx.z;
  if (symmetric && tj < ti) return;
  __shared__ float Xh[KSTEP][TT + 1], Xl[KSTEP][TT + 1], Yh[KSTEP][TT + 1], Yl[KSTEP][TT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = ti * TT, j0 = tj * TT;
  const int64_t r0 = s * rows_per_split;
  const int64_t r1 = min(n, r0 + rows_per_split);
  float2 S[R][H], E[R][H], Ah[R][H], Al[R][H];
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int v = 0; v < H; ++v) S[u][v] = E[u][v] = Ah[u][v] = Al[u][v] = make_float2(0.f, 0.f);
  int steps = 0;
  for (int64_t rb = r0; rb < r1; rb += KSTEP) {
    for (int t = threadIdx.x; t < KSTEP * TT; t += 256) {
      const int rr = t / TT, cc = t % TT;
      const int64_t r = rb + rr;
      const bool rok = r < r1;
      split_f64((rok && i0 + cc < na) ? X[r * ldx + i0 + cc] : 0.0, Xh[rr][cc], Xl[rr][cc]);
      split_f64((rok && j0 + cc < nb) ? Y[r * ldy + j0 + cc] : 0.0, Yh[rr][cc], Yl[rr][cc]);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KSTEP; ++k) {
      dfp b[H];
#pragma unroll
      for (int v = 0; v < H; ++v)
        b[v] = dfp{make_float2(Yh[k][tx + 32 * v], Yh[k][tx + 32 * v + 16]),
                   make_float2(Yl[k][tx + 32 * v], Yl[k][tx + 32 * v + 16])};
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const float ah = Xh[k][ty + 16 * u], al = Xl[k][ty + 16 * u];
        const dfp a{make_float2(ah, ah), make_float2(al, al)};
        const dfp na{make_float2(-ah, -ah), make_float2(-al, -al)};
#pragma unroll
        for (int v = 0; v < H; ++v) dot2p(S[u][v], E[u][v], a, na, b[v]);
      }
    }
    __syncthreads();
    if (++steps == DF_FOLD) {
      steps = 0;
#pragma unroll
      for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < H; ++v) df_fold(Ah[u][v], Al[u][v], S[u][v], E[u][v]);
    }
  }
  double* P = part + static_cast<size_t>(s) * na * nb;
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = i0 + ty + 16 * u;
    if (i >= na) continue;
#pragma unroll
    for (int v = 0; v < H; ++v) {
      df_fold(Ah[u][v], Al[u][v], S[u][v], E[u][v]);
      const int j = j0 + tx + 32 * v;
      if (j < nb) P[static_cast<size_t>(i) * nb + j] = static_cast<double>(Ah[u][v].x) + static_cast<double>(Al[u][v].x);
      if (j + 16 < nb)
        P[static_cast<size_t>(i) * nb + j + 16] = static_cast<double>(Ah[u][v].y) + static_cast<double>(Al[u][v].y);
    }
  }
}

// Out[r][c] = alpha * sum_k In[r][k] W[k][c] + beta * Out[r][c] (the tiling of
// gemm_tall_kernel, RN >= 2); the sum in double-float, the final update in FP64.
template <int RN>
__global__ void __launch_bounds__(256)
gemm_df_kernel(int64_t n, const double* __restrict__ In, int64_t ldi, int na, const double* __restrict__ W,
               int64_t ldw, int nb, double alpha, double beta, double* __restrict__ Out, int64_t ldo) {
  constexpr int TR = 64, TC = 16 * RN, H = RN / 2;
  __shared__ float Ih[KSTEP][TR + 1], Il[KSTEP][TR + 1], Wh[KSTEP][TC + 1], Wl[KSTEP][TC + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * TR;
  const int c0 = blockIdx.y * TC;
  float2 S[4][H], E[4][H], Ah[4][H], Al[4][H];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < H; ++v) S[u][v] = E[u][v] = Ah[u][v] = Al[u][v] = make_float2(0.f, 0.f);
  int steps = 0;
  for (int k0 = 0; k0 < na; k0 += KSTEP) {
    for (int t = threadIdx.x; t < KSTEP * TR; t += 256) {
      const int kk = t % KSTEP, rr = t / KSTEP;
      const int64_t r = r0 + rr;
      split_f64((r < n && k0 + kk < na) ? In[r * ldi + k0 + kk] : 0.0, Ih[kk][rr], Il[kk][rr]);
    }
    for (int t = threadIdx.x; t < KSTEP * TC; t += 256) {
      const int kw = t / TC, cw = t % TC;
      split_f64((k0 + kw < na && c0 + cw < nb) ? W[static_cast<int64_t>(k0 + kw) * ldw + c0 + cw] : 0.0, Wh[kw][cw],
                Wl[kw][cw]);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KSTEP; ++k) {
      dfp b[H];
#pragma unroll
      for (int v = 0; v < H; ++v)
        b[v] = dfp{make_float2(Wh[k][tx + 32 * v], Wh[k][tx + 32 * v + 16]),
                   make_float2(Wl[k][tx + 32 * v], Wl[k][tx + 32 * v + 16])};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float ah = Ih[k][ty + 16 * u], al = Il[k][ty + 16 * u];
        const dfp a{make_float2(ah, ah), make_float2(al, al)};
        const dfp na{make_float2(-ah, -ah), make_float2(-al, -al)};
#pragma unroll
        for (int v = 0; v < H; ++v) dot2p(S[u][v], E[u][v], a, na, b[v]);
      }
    }
    __syncthreads();
    if (++steps == DF_FOLD) {
      steps = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < H; ++v) df_fold(Ah[u][v], Al[u][v], S[u][v], E[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t r = r0 + ty + 16 * u;
    if (r >= n) continue;
#pragma unroll
    for (int v = 0; v < H; ++v) {
      df_fold(Ah[u][v], Al[u][v], S[u][v], E[u][v]);
      const double val[2] = {static_cast<double>(Ah[u][v].x) + static_cast<double>(Al[u][v].x),
                             static_cast<double>(Ah[u][v].y) + static_cast<double>(Al[u][v].y)};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = c0 + tx + 32 * v + 16 * h;
        if (c >= nb) continue;
        double* o = Out + r * ldo + c;
        const double x = alpha * val[h];
        *o = (beta == 0.0) ? x : fma(beta, *o, x);
      }
    }
  }
}

template <typename T>
__global__ void gather_cols_kernel(int64_t n, const T* __restrict__ src, int64_t lds,
                                   const int32_t* __restrict__ idx, int ncols, T* __restrict__ dst,
                                   int64_t ldd) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * ncols) return;
  const int64_t r = t / ncols;
  const int c = static_cast<int>(t % ncols);
  dst[r * ldd + c] = src[r * lds + idx[c]];
}

template <typename T>
__global__ void gather_cols2_kernel(int64_t n, const T* __restrict__ srcA, int64_t ldA,
                                    const T* __restrict__ srcB, int64_t ldB,
                                    const int32_t* __restrict__ idx, int ncols, T* __restrict__ dst,
                                    int64_t ldd) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * ncols) return;
  const int64_t r = t / ncols;
  const int c = static_cast<int>(t % ncols);
  const int s = idx[c];
  dst[r * ldd + c] = s >= 0 ? srcA[r * ldA + s] : srcB[r * ldB + (-s - 1)];
}

__global__ void residual_finish_kernel(int p, const double* __restrict__ ss, const double* __restrict__ mu,
                                       int smallest, double sigma, double* __restrict__ res) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  const double lam = smallest ? sigma - mu[c] : mu[c];
  res[c] = sqrt(fmax(ss[c], 0.0)) / fmax(1.0, fabs(lam));
}

// one block per column: largest |x| and its (smallest) row index
__global__ void column_signs_kernel(int64_t n, const double* __restrict__ X, int64_t ldx,
                                    double* __restrict__ sign) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  const int c = blockIdx.x;
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = fabs(X[r * ldx + c]);
    if (v > best) {
      best = v;
      bi = r;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double v2 = sv[threadIdx.x + s];
      const int64_t i2 = si[threadIdx.x + s];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sign[c] = X[si[0] * ldx + c] < 0.0 ? -1.0 : 1.0;
}

__global__ void write_colmajor_kernel(int64_t n, const double* __restrict__ X, int64_t ldx,
                                      const int32_t* __restrict__ perm, const double* __restrict__ sign,
                                      int k, double* __restrict__ out, int64_t ldq) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * k) return;
  const int c = static_cast<int>(t / n);
  const int64_t r = t % n;
  out[c * ldq + r] = sign[c] * X[r * ldx + perm[c]];
}

template <typename Ti, typename To>
__global__ void copy_block_kernel(int64_t n, const Ti* __restrict__ src, int64_t lds, int ncols,
                                  To* __restrict__ dst, int64_t ldd) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * ncols) return;
  const int64_t r = t / ncols;
  const int c = static_cast<int>(t % ncols);
  dst[r * ldd + c] = static_cast<To>(src[r * lds + c]);
}

__global__ void fill_kernel(double* p, int64_t count, double v) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < count) p[t] = v;
}

__global__ void symmetrize_kernel(int m, double* H, int64_t ldh) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(m) * m) return;
  const int i = static_cast<int>(t / m), j = static_cast<int>(t % m);
  if (j <= i) return;
  const double v = 0.5 * (H[static_cast<int64_t>(i) * ldh + j] + H[static_cast<int64_t>(j) * ldh + i]);
  H[static_cast<int64_t>(i) * ldh + j] = v;
  H[static_cast<int64_t>(j) * ldh + i] = v;
}

struct BlockOffsets {
  int n;
  int off[17];  // block starts, off[n] = m
};

// H (i < j): the average of H_ij and H_ji inside a diagonal block (both computed), their
// sum across blocks (one of the two was left zero)
__global__ void symmetrize_blocks_kernel(int m, double* H, int64_t ldh, BlockOffsets bo) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(m) * m) return;
  const int i = static_cast<int>(t / m), j = static_cast<int>(t % m);
  if (j <= i) return;
  int bi = 0, bj = 0;
  for (int b = 1; b < bo.n; ++b) {
    bi += (i >= bo.off[b]);
    bj += (j >= bo.off[b]);
  }
  const double a = H[static_cast<int64_t>(i) * ldh + j], c = H[static_cast<int64_t>(j) * ldh + i];
  const double v = (bi == bj) ? 0.5 * (a + c) : a + c;
  H[static_cast<int64_t>(i) * ldh + j] = v;
  H[static_cast<int64_t>(j) * ldh + i] = v;
}

__global__ void scale_sym_kernel(int m, double* G, int64_t ldg, const double* __restrict__ s) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(m) * m) return;
  const int i = static_cast<int>(t / m), j = static_cast<int>(t % m);
  G[static_cast<int64_t>(i) * ldg + j] *= s[i] * s[j];
}

__global__ void inv_sqrt_kernel(int m, const double* __restrict__ ss, double* __restrict__ s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) s[i] = ss[i] > 0.0 ? 1.0 / sqrt(ss[i]) : 0.0;
}

__global__ void svqb_prep_kernel(int m, const double* __restrict__ G, int64_t ldg,
                                 double* __restrict__ Gh, double* __restrict__ d) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(m) * m) return;
  const int i = static_cast<int>(t / m), j = static_cast<int>(t % m);
  const double gi = G[static_cast<int64_t>(i) * ldg + i];
  const double gj = G[static_cast<int64_t>(j) * ldg + j];
  const double di = gi > 0.0 ? 1.0 / sqrt(gi) : 0.0;
  const double dj = gj > 0.0 ? 1.0 / sqrt(gj) : 0.0;
  Gh[static_cast<int64_t>(i) * m + j] = G[static_cast<int64_t>(i) * ldg + j] * di * dj;
  if (j == 0) d[i] = di;
}

// number of leading theta_j > tau * theta_0 (theta descending)
__device__ int svqb_rank(int m, const double* theta, double tau) {
  const double t0 = theta[0];
  if (!(t0 > 0.0)) return 0;
  const double thr = tau * t0;
  int lo = 0, hi = m;  // first index with !(theta > thr)
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (theta[mid] > thr) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void svqb_finish_kernel(int m, const double* __restrict__ theta, const double* __restrict__ W,
                                   int64_t ldw, const double* __restrict__ d, double tau,
                                   double* __restrict__ M, int32_t* rank_dev) {
  __shared__ int r_s;
  if (threadIdx.x == 0) r_s = svqb_rank(m, theta, tau);
  __syncthreads();
  const int r = r_s;
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t == 0) *rank_dev = r;
  if (t >= static_cast<int64_t>(m) * m) return;
  const int i = static_cast<int>(t / m), j = static_cast<int>(t % m);
  M[static_cast<int64_t>(i) * m + j] = (j < r) ? d[i] * W[static_cast<int64_t>(i) * ldw + j] / sqrt(theta[j]) : 0.0;
}

// Ginv[i][j] = sum_k W[i][k] W[j][k] / theta_k
__global__ void inverse_from_eig_kernel(int m, const double* __restrict__ theta,
                                        const double* __restrict__ W, int64_t ldw,
                                        double* __restrict__ Ginv) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(m) * m) return;
  const int i = static_cast<int>(t / m), j = static_cast<int>(t % m);
  double s = 0.0;
  for (int k = 0; k < m; ++k)
    s = fma(W[static_cast<int64_t>(i) * ldw + k] * W[static_cast<int64_t>(j) * ldw + k], 1.0 / theta[k], s);
  Ginv[t] = s;
}

__global__ void rcond_final_kernel(int m, const double* __restrict__ G, int64_t ldg,
                                   const double* __restrict__ Ginv, const double* __restrict__ theta,
                                   double* __restrict__ rc) {
  __shared__ double sg[256], si[256];
  double mg = 0.0, mi = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double cg = 0.0, ci = 0.0;
    for (int i = 0; i < m; ++i) {
      cg += fabs(G[static_cast<int64_t>(i) * ldg + j]);
      ci += fabs(Ginv[static_cast<int64_t>(i) * m + j]);
    }
    mg = fmax(mg, cg);
    mi = fmax(mi, ci);
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
    const double tmin = theta[m - 1];
    double r = 0.0;
    if (tmin > 0.0 && isfinite(si[0]) && si[0] > 0.0 && sg[0] > 0.0) r = 1.0 / (sg[0] * si[0]);
    *rc = r;
  }
}

__device__ __forceinline__ double nan_to_neginf(double v) { return isnan(v) ? -INFINITY : v; }

__global__ void select_top_kernel(const double* __restrict__ vl, int nl, const double* __restrict__ vn,
                                  int nn, int p, int32_t* __restrict__ map, double* __restrict__ val) {
  const int N = nl + nn;
  for (int s = threadIdx.x; s < p; s += blockDim.x) map[s] = -1;
  __syncthreads();
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const double ve = nan_to_neginf(e < nl ? vl[e] : vn[e - nl]);
    int rank = 0;
    for (int f = 0; f < N; ++f) {
      const double vf = nan_to_neginf(f < nl ? vl[f] : vn[f - nl]);
      rank += (vf > ve) || (vf == ve && f < e);
    }
    if (rank < p) {
      map[rank] = e;
      val[rank] = ve;
    }
  }
}

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) on counter (c0, c1, 0, 0).
__device__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t c[4] = {c0, c1, 0u, 0u};
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

template <typename T>
__global__ void gaussian_fill_kernel(int64_t n, int ncols, uint64_t seed, T* X, int64_t ldx) {
  const int64_t pair = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t total = n * ncols;
  if (2 * pair >= total) return;
  uint32_t o[4];
  philox4x32_10(static_cast<uint32_t>(pair & 0xffffffffu), static_cast<uint32_t>(pair >> 32),
                static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32), o);
  const double two53 = 9007199254740992.0;
  const double u1 = ((double)(o[0] >> 5) * 67108864.0 + (double)(o[1] >> 6) + 0.5) / two53;
  const double u2 = ((double)(o[2] >> 5) * 67108864.0 + (double)(o[3] >> 6)) / two53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  const int64_t e0 = 2 * pair;
  X[(e0 / ncols) * ldx + (e0 % ncols)] = static_cast<T>(r * cs);
  if (e0 + 1 < total) X[((e0 + 1) / ncols) * ldx + ((e0 + 1) % ncols)] = static_cast<T>(r * sn);
}

inline int blocks_for(int64_t count, int threads) {
  return static_cast<int>(std::max<int64_t>(1, (count + threads - 1) / threads));
}

}  // namespace

// Split-K plan of a Gram product: tile size and the number of row splits, limited so the
// partial sums fit in `max_part` doubles (0: no limit).
struct GramPlan {
  int R = 4, TT = 64, gi = 1, gj = 1, symmetric = 0;
  int64_t nsplit = 1, rows = 0;
};

template <typename T>
static GramPlan gram_plan(arb_ctx ctx, int64_t n, const T* X, int64_t ldx, int32_t na, const T* Y, int64_t ldy,
                          int32_t nb, size_t max_part) {
  GramPlan g;
  g.symmetric = (X == Y && ldx == ldy && na == nb) ? 1 : 0;
  const int mx = std::max(na, nb);
  g.R = mx <= 16 ? 1 : (mx <= 32 ? 2 : 4);
  if (std::is_same<T, double>::value && ctx->dense_df) g.R = std::max(g.R, 2);  // outputs in pairs
  g.TT = 16 * g.R;
  g.gi = (na + g.TT - 1) / g.TT;
  g.gj = (nb + g.TT - 1) / g.TT;
  const int tiles = g.symmetric ? g.gi * (g.gi + 1) / 2 : g.gi * g.gj;
  const int64_t target = static_cast<int64_t>(ctx->num_sms) * 3;
  int64_t nsplit = std::max<int64_t>(1, (target + tiles - 1) / tiles);
  nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, n / (4 * KSTEP)));
  nsplit = std::min<int64_t>(nsplit, 4096);
  if (max_part > 0) {
    const int64_t per = static_cast<int64_t>(na) * nb;
    nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, static_cast<int64_t>(max_part) / per));
  }
  int64_t rows = (n + nsplit - 1) / nsplit;
  rows = ((rows + KSTEP - 1) / KSTEP) * KSTEP;
  g.rows = rows;
  g.nsplit = std::max<int64_t>(1, (n + rows - 1) / rows);
  return g;
}

// The two launches of a Gram product given a partial-sum buffer of g.nsplit * na * nb.
template <typename T>
static arb_status gram_launch(arb_ctx ctx, const GramPlan& g, int64_t n, const T* X, int64_t ldx, int32_t na,
                              const T* Y, int64_t ldy, int32_t nb, double* part, double* C, int64_t ldc) {
  dim3 grid(g.gi, g.gj, static_cast<unsigned>(g.nsplit));
  if constexpr (std::is_same<T, double>::value) {
    if (ctx->dense_df) {
      if (g.R == 2)
        gram_df_kernel<2><<<grid, 256, 0, ctx->stream>>>(n, X, ldx, na, Y, ldy, nb, g.rows, g.symmetric, part);
      else
        gram_df_kernel<4><<<grid, 256, 0, ctx->stream>>>(n, X, ldx, na, Y, ldy, nb, g.rows, g.symmetric, part);
      ARB_LAUNCHED(ctx);
      gram_reduce_kernel<<<blocks_for(static_cast<int64_t>(na) * nb, 256), 256, 0, ctx->stream>>>(
          part, static_cast<int>(g.nsplit), na, nb, g.symmetric, g.TT, C, ldc);
      ARB_LAUNCHED(ctx);
      return ARB_OK;
    }
  }
  if (g.R == 1)
    gram_kernel<T, 1><<<grid, 256, 0, ctx->stream>>>(n, X, ldx, na, Y, ldy, nb, g.rows, g.symmetric, part);
  else if (g.R == 2)
    gram_kernel<T, 2><<<grid, 256, 0, ctx->stream>>>(n, X, ldx, na, Y, ldy, nb, g.rows, g.symmetric, part);
  else
    gram_kernel<T, 4><<<grid, 256, 0, ctx->stream>>>(n, X, ldx, na, Y, ldy, nb, g.rows, g.symmetric, part);
  ARB_LAUNCHED(ctx);
  gram_reduce_kernel<<<blocks_for(static_cast<int64_t>(na) * nb, 256), 256, 0, ctx->stream>>>(
      part, static_cast<int>(g.nsplit), na, nb, g.symmetric, g.TT, C, ldc);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

// FP32 Gram products on the tensor cores (tc.cu): split-K over row ranges that are whole
// multiples of the kernel's 256-row fold, about two CTAs per SM.
static arb_status gram_f32_tc(arb_ctx ctx, int64_t n, const float* X, int64_t ldx, int32_t na, const float* Y,
                              int64_t ldy, int32_t nb, double* C, int64_t ldc) {
  const int symmetric = (X == Y && ldx == ldy && na == nb) ? 1 : 0;
  const int tm = gram_tc_tile_m(), tn = gram_tc_tile_n(), al = gram_tc_rows_align();
  const int64_t tiles = static_cast<int64_t>((na + tm - 1) / tm) * ((nb + tn - 1) / tn);
  int64_t nsplit = std::max<int64_t>(1, (2 * static_cast<int64_t>(ctx->num_sms) + tiles - 1) / tiles);
  nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, n / al));
  int64_t rows = (n + nsplit - 1) / nsplit;
  rows = ((rows + al - 1) / al) * al;
  nsplit = (n + rows - 1) / rows;
  double* part;
  int* err;
  ARB_TRY(ws<double>(ctx, WS_GRAM_PART, static_cast<size_t>(nsplit) * na * nb, &part));
  ARB_TRY(ws<int>(ctx, WS_TC_ERR, 1, &err));
  ARB_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  ARB_TRY(gram_tc_launch(ctx, n, X, ldx, na, Y, ldy, nb, symmetric, part, nsplit, rows, err));
  gram_reduce_kernel<<<blocks_for(static_cast<int64_t>(na) * nb, 256), 256, 0, ctx->stream>>>(
      part, static_cast<int>(nsplit), na, nb, symmetric, 0, C, ldc);
  ARB_LAUNCHED(ctx);
  int herr = 0;
  ARB_TRY(d2h_sync(ctx, &herr, err, sizeof(int)));
  if (herr) return set_error(ctx, ARB_CUDA_ERROR, "gram (tensor cores): a pipeline wait timed out");
  return ARB_OK;
}

template <typename T>
arb_status gram(arb_ctx ctx, int64_t n, const T* X, int64_t ldx, int32_t na, const T* Y, int64_t ldy,
                int32_t nb, double* C, int64_t ldc) {
  if (na <= 0 || nb <= 0) return ARB_OK;
  if constexpr (std::is_same<T, float>::value) {
    if (gram_tc_supported(n, ldx, ldy, X, Y)) return gram_f32_tc(ctx, n, X, ldx, na, Y, ldy, nb, C, ldc);
  }
  const GramPlan g = gram_plan<T>(ctx, n, X, ldx, na, Y, ldy, nb, 0);
  double* part;
  ARB_TRY(ws<double>(ctx, WS_GRAM_PART, static_cast<size_t>(g.nsplit) * na * nb, &part));
  return gram_launch<T>(ctx, g, n, X, ldx, na, Y, ldy, nb, part, C, ldc);
}

arb_status gram_into(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t na, const double* Y,
                     int64_t ldy, int32_t nb, double* C, int64_t ldc, double* part, size_t part_capacity) {
  if (na <= 0 || nb <= 0) return ARB_OK;
  if (static_cast<size_t>(na) * static_cast<size_t>(nb) > part_capacity)
    return set_error(ctx, ARB_INVALID_ARG, "gram: na * nb exceeds the partial-sum capacity");
  const GramPlan g = gram_plan<double>(ctx, n, X, ldx, na, Y, ldy, nb, part_capacity);
  return gram_launch<double>(ctx, g, n, X, ldx, na, Y, ldy, nb, part, C, ldc);
}

template <typename T>
arb_status gemm_tall(arb_ctx ctx, int64_t n, const T* In, int64_t ldi, int32_t na, const double* W,
                     int64_t ldw, int32_t nb, double alpha, double beta, T* Out, int64_t ldo) {
  if (n <= 0 || nb <= 0) return ARB_OK;
  if (na <= 0) {
    if (beta == 1.0) return ARB_OK;
    return set_error(ctx, ARB_INVALID_ARG, "gemm_tall: empty inner dimension with beta != 1");
  }
  if constexpr (std::is_same<T, double>::value) {
    if (ctx->dense_df) {
      const int RN = nb <= 32 ? 2 : 4;
      const int TC = 16 * RN;
      dim3 grid(static_cast<unsigned>((n + 63) / 64), static_cast<unsigned>((nb + TC - 1) / TC));
      if (RN == 2)
        gemm_df_kernel<2><<<grid, 256, 0, ctx->stream>>>(n, In, ldi, na, W, ldw, nb, alpha, beta, Out, ldo);
      else
        gemm_df_kernel<4><<<grid, 256, 0, ctx->stream>>>(n, In, ldi, na, W, ldw, nb, alpha, beta, Out, ldo);
      ARB_LAUNCHED(ctx);
      return ARB_OK;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    // the tensor cores for every product with an inner dimension of a full MMA step
    if (na >= 8 && gemm_tc_supported(ldi, ldo, In, Out)) {
      float* img;
      int* err;
      ARB_TRY(ws<float>(ctx, WS_TC_IMG, gemm_tc_image_floats(na, nb), &img));
      ARB_TRY(ws<int>(ctx, WS_TC_ERR, 1, &err));
      ARB_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
      ARB_TRY(gemm_tc_launch(ctx, n, In, ldi, na, W, ldw, nb, static_cast<float>(alpha), static_cast<float>(beta), Out,
                             ldo, img, err));
      int herr = 0;
      ARB_TRY(d2h_sync(ctx, &herr, err, sizeof(int)));
      if (herr) return set_error(ctx, ARB_CUDA_ERROR, "tall product (tensor cores): a pipeline wait timed out");
      return ARB_OK;
    }
  }
  const int RN = nb <= 16 ? 1 : (nb <= 32 ? 2 : 4);
  const int TC = 16 * RN;
  dim3 grid(static_cast<unsigned>((n + 63) / 64), static_cast<unsigned>((nb + TC - 1) / TC));
  const T al = static_cast<T>(alpha), be = static_cast<T>(beta);
  if (RN == 1)
    gemm_tall_kernel<T, 1><<<grid, 256, 0, ctx->stream>>>(n, In, ldi, na, W, ldw, nb, al, be, Out, ldo);
  else if (RN == 2)
    gemm_tall_kernel<T, 2><<<grid, 256, 0, ctx->stream>>>(n, In, ldi, na, W, ldw, nb, al, be, Out, ldo);
  else
    gemm_tall_kernel<T, 4><<<grid, 256, 0, ctx->stream>>>(n, In, ldi, na, W, ldw, nb, al, be, Out, ldo);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

// out[c] = sum_r X[r][c]^2, FP64 sums, one CTA per column and a fixed reduction tree
template <typename T>
__global__ void col_norm2_kernel(int64_t n, const T* __restrict__ X, int64_t ldx, double* __restrict__ out) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double x = static_cast<double>(X[r * ldx + c]);
    s = fma(x, x, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

template <typename T>
arb_status col_norms2(arb_ctx ctx, int64_t n, const T* X, int64_t ldx, int32_t m, double* out) {
  if (m <= 0) return ARB_OK;
  col_norm2_kernel<T><<<static_cast<unsigned>(m), 256, 0, ctx->stream>>>(n, X, ldx, out);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

template <typename T>
arb_status gather_cols(arb_ctx ctx, int64_t n, const T* src, int64_t lds, const int32_t* idx, int32_t ncols,
                       T* dst, int64_t ldd) {
  if (ncols <= 0 || n <= 0) return ARB_OK;
  gather_cols_kernel<T><<<blocks_for(n * ncols, 256), 256, 0, ctx->stream>>>(n, src, lds, idx, ncols, dst, ldd);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

template <typename T>
arb_status gather_cols2(arb_ctx ctx, int64_t n, const T* srcA, int64_t ldA, const T* srcB, int64_t ldB,
                        const int32_t* idx, int32_t ncols, T* dst, int64_t ldd) {
  if (ncols <= 0 || n <= 0) return ARB_OK;
  gather_cols2_kernel<T><<<blocks_for(n * ncols, 256), 256, 0, ctx->stream>>>(n, srcA, ldA, srcB, ldB, idx,
                                                                              ncols, dst, ldd);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

template <typename Ti, typename To>
arb_status copy_block(arb_ctx ctx, int64_t n, const Ti* src, int64_t lds, int32_t ncols, To* dst, int64_t ldd) {
  if (ncols <= 0 || n <= 0) return ARB_OK;
  copy_block_kernel<Ti, To><<<blocks_for(n * ncols, 256), 256, 0, ctx->stream>>>(n, src, lds, ncols, dst, ldd);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

template arb_status gram<double>(arb_ctx, int64_t, const double*, int64_t, int32_t, const double*, int64_t,
                                 int32_t, double*, int64_t);
template arb_status gram<float>(arb_ctx, int64_t, const float*, int64_t, int32_t, const float*, int64_t,
                                int32_t, double*, int64_t);
template arb_status gemm_tall<double>(arb_ctx, int64_t, const double*, int64_t, int32_t, const double*, int64_t,
                                      int32_t, double, double, double*, int64_t);
template arb_status gemm_tall<float>(arb_ctx, int64_t, const float*, int64_t, int32_t, const double*, int64_t,
                                     int32_t, double, double, float*, int64_t);
template arb_status col_norms2<double>(arb_ctx, int64_t, const double*, int64_t, int32_t, double*);
template arb_status col_norms2<float>(arb_ctx, int64_t, const float*, int64_t, int32_t, double*);
template arb_status gather_cols<double>(arb_ctx, int64_t, const double*, int64_t, const int32_t*, int32_t,
                                        double*, int64_t);
template arb_status gather_cols<float>(arb_ctx, int64_t, const float*, int64_t, const int32_t*, int32_t, float*,
                                       int64_t);
template arb_status gather_cols2<double>(arb_ctx, int64_t, const double*, int64_t, const double*, int64_t,
                                         const int32_t*, int32_t, double*, int64_t);
template arb_status gather_cols2<float>(arb_ctx, int64_t, const float*, int64_t, const float*, int64_t,
                                        const int32_t*, int32_t, float*, int64_t);
template arb_status copy_block<double, double>(arb_ctx, int64_t, const double*, int64_t, int32_t, double*,
                                               int64_t);
template arb_status copy_block<float, float>(arb_ctx, int64_t, const float*, int64_t, int32_t, float*, int64_t);
template arb_status copy_block<float, double>(arb_ctx, int64_t, const float*, int64_t, int32_t, double*,
                                              int64_t);
template arb_status copy_block<double, float>(arb_ctx, int64_t, const double*, int64_t, int32_t, float*,
                                              int64_t);

arb_status residual_finish(arb_ctx ctx, int32_t p, const double* ss, const double* mu, int smallest,
                           double sigma, double* res) {
  if (p <= 0) return ARB_OK;
  residual_finish_kernel<<<blocks_for(p, 128), 128, 0, ctx->stream>>>(p, ss, mu, smallest, sigma, res);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status column_signs(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t ncols,
                        double* sign) {
  if (ncols <= 0) return ARB_OK;
  column_signs_kernel<<<ncols, 256, 0, ctx->stream>>>(n, X, ldx, sign);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status write_colmajor(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, const int32_t* perm,
                          const double* sign, int32_t k, double* out, int64_t ldq) {
  if (k <= 0 || n <= 0) return ARB_OK;
  write_colmajor_kernel<<<blocks_for(n * k, 256), 256, 0, ctx->stream>>>(n, X, ldx, perm, sign, k, out, ldq);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}


arb_status fill(arb_ctx ctx, double* p, int64_t count, double v) {
  if (count <= 0) return ARB_OK;
  fill_kernel<<<blocks_for(count, 256), 256, 0, ctx->stream>>>(p, count, v);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status symmetrize(arb_ctx ctx, int32_t m, double* H, int64_t ldh) {
  if (m <= 1) return ARB_OK;
  symmetrize_kernel<<<blocks_for(static_cast<int64_t>(m) * m, 256), 256, 0, ctx->stream>>>(m, H, ldh);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status symmetrize_upper_blocks(arb_ctx ctx, int32_t m, double* H, int64_t ldh, const int32_t* off,
                                  const int32_t* rk, int32_t nblk) {
  if (m <= 1) return ARB_OK;
  if (nblk < 1 || nblk > 16) return set_error(ctx, ARB_INVALID_ARG, "symmetrize: 1..16 blocks");
  BlockOffsets bo{};
  bo.n = nblk;
  for (int b = 0; b < nblk; ++b) bo.off[b] = off[b];
  bo.off[nblk] = off[nblk - 1] + rk[nblk - 1];
  symmetrize_blocks_kernel<<<blocks_for(static_cast<int64_t>(m) * m, 256), 256, 0, ctx->stream>>>(m, H, ldh, bo);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status lin3(arb_ctx ctx, int64_t n, double* w, double a, const double* v, double b, const double* u) {
  lin3_kernel<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(n, w, a, v, b, u);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status scale_vec(arb_ctx ctx, int64_t n, double* dst, const double* src, double s) {
  scale_vec_kernel<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(n, dst, src, s);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status scale_sym(arb_ctx ctx, int32_t m, double* G, int64_t ldg, const double* s) {
  if (m <= 0) return ARB_OK;
  scale_sym_kernel<<<blocks_for(static_cast<int64_t>(m) * m, 256), 256, 0, ctx->stream>>>(m, G, ldg, s);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status inv_sqrt(arb_ctx ctx, int32_t m, const double* ss, double* s) {
  if (m <= 0) return ARB_OK;
  inv_sqrt_kernel<<<blocks_for(m, 256), 256, 0, ctx->stream>>>(m, ss, s);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status svqb_prep(arb_ctx ctx, int32_t m, const double* G, int64_t ldg, double* Ghat, double* d) {
  svqb_prep_kernel<<<blocks_for(static_cast<int64_t>(m) * m, 256), 256, 0, ctx->stream>>>(m, G, ldg, Ghat, d);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status svqb_finish(arb_ctx ctx, int32_t m, const double* theta, const double* W, int64_t ldw,
                       const double* d, double tau, double* M, int32_t* rank_dev) {
  svqb_finish_kernel<<<blocks_for(static_cast<int64_t>(m) * m, 256), 256, 0, ctx->stream>>>(
      m, theta, W, ldw, d, tau, M, rank_dev);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status rcond_from_eig(arb_ctx ctx, int32_t m, const double* G, int64_t ldg, const double* theta,
                          const double* W, int64_t ldw, double* rc_dev) {
  double* Ginv;
  ARB_TRY(ws<double>(ctx, WS_SMALL3, static_cast<size_t>(m) * m, &Ginv));
  inverse_from_eig_kernel<<<blocks_for(static_cast<int64_t>(m) * m, 256), 256, 0, ctx->stream>>>(
      m, theta, W, ldw, Ginv);
  ARB_LAUNCHED(ctx);
  rcond_final_kernel<<<1, 256, 0, ctx->stream>>>(m, G, ldg, Ginv, theta, rc_dev);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status select_top(arb_ctx ctx, const double* vlock, int32_t nl, const double* vnew, int32_t nn,
                      int32_t p, int32_t* map, double* val) {
  select_top_kernel<<<1, 1024, 0, ctx->stream>>>(vlock, nl, vnew, nn, p, map, val);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

template <typename T>
arb_status gaussian_fill(arb_ctx ctx, int64_t n, int32_t ncols, uint64_t seed, T* X, int64_t ldx) {
  const int64_t pairs = (n * ncols + 1) / 2;
  gaussian_fill_kernel<T><<<blocks_for(pairs, 256), 256, 0, ctx->stream>>>(n, ncols, seed, X, ldx);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}
template arb_status gaussian_fill<double>(arb_ctx, int64_t, int32_t, uint64_t, double*, int64_t);
template arb_status gaussian_fill<float>(arb_ctx, int64_t, int32_t, uint64_t, float*, int64_t);

}  // namespace arb
