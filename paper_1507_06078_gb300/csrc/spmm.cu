// Fused CSR block SpMM: the A-product of the filter recurrence (Algorithm 7 / Clenshaw),
// of the augmentation [X, AX, ..., A^q X] (Algorithm 5), of U^T A U (Algorithm 1) and
// of the residuals A x_i - mu_i x_i (eq. resi), with the per-step vector update and the
// column reductions fused into the epilogue.
//
// Layout: A in CSR (int32 rowptr/col, float64 val); every block is row-major with a
// leading dimension, so the row of the iterate that a nonzero a_ij gathers is one
// contiguous run of `ncols` doubles.  One warp owns one row at a time; its 32 lanes
// cover 32*VEC consecutive columns per chunk, so each gathered row segment is a fully
// coalesced 256/512-byte transaction.  Column indices and values of a row are loaded
// once per 32 nonzeros (one per lane) and broadcast with shuffles.
#include <algorithm>

#include "arb_internal.h"

namespace arb {
namespace {

constexpr int SPMM_THREADS = 256;
constexpr int SPMM_WARPS = SPMM_THREADS / 32;

template <typename T>
struct KParams {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const T* val;
  int32_t ncols;
  const T* Yin;
  int64_t ldy;
  T alpha, beta;
  const double* sy;
  const T* X;
  int64_t ldx;
  const double* sx;
  const T* Z;
  int64_t ldz;
  const double* sz;
  T* out;
  int64_t ldo;
  double* red_part;  // [gridDim.x][ncols] per-block partial column reductions, or NULL
  int dot_with_yin;
};

// VEC consecutive elements as one 8/16-byte access
template <typename T, int VEC>
struct VecIO;
// ld/st: default caching (the gathered block, reused by neighbouring rows through L1/L2);
// lds/sts: evict-first streaming access for the blocks each row touches once (X, the
// b_{j+2} term and the output), so that they do not push the gathered block out of L2.
template <>
struct VecIO<double, 1> {
  __device__ static void ld(const double* p, double* r) { r[0] = *p; }
  __device__ static void st(double* p, const double* r) { *p = r[0]; }
  __device__ static void lds(const double* p, double* r) { r[0] = __ldcs(p); }
  __device__ static void sts(double* p, const double* r) { __stcs(p, r[0]); }
};
template <>
struct VecIO<double, 2> {
  __device__ static void ld(const double* p, double* r) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    r[0] = t.x;
    r[1] = t.y;
  }
  __device__ static void st(double* p, const double* r) { *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]); }
  __device__ static void lds(const double* p, double* r) {
    const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    r[0] = t.x;
    r[1] = t.y;
  }
  __device__ static void sts(double* p, const double* r) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(r[0], r[1]));
  }
};
template <>
struct VecIO<float, 1> {
  __device__ static void ld(const float* p, float* r) { r[0] = *p; }
  __device__ static void st(float* p, const float* r) { *p = r[0]; }
  __device__ static void lds(const float* p, float* r) { r[0] = __ldcs(p); }
  __device__ static void sts(float* p, const float* r) { __stcs(p, r[0]); }
};
template <>
struct VecIO<float, 2> {
  __device__ static void ld(const float* p, float* r) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    r[0] = t.x;
    r[1] = t.y;
  }
  __device__ static void st(float* p, const float* r) { *reinterpret_cast<float2*>(p) = make_float2(r[0], r[1]); }
  __device__ static void lds(const float* p, float* r) {
    const float2 t = __ldcs(reinterpret_cast<const float2*>(p));
    r[0] = t.x;
    r[1] = t.y;
  }
  __device__ static void sts(float* p, const float* r) { __stcs(reinterpret_cast<float2*>(p), make_float2(r[0], r[1])); }
};
template <>
struct VecIO<float, 4> {
  __device__ static void ld(const float* p, float* r) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r[0] = t.x;
    r[1] = t.y;
    r[2] = t.z;
    r[3] = t.w;
  }
  __device__ static void st(float* p, const float* r) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
  }
  __device__ static void lds(const float* p, float* r) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    r[0] = t.x;
    r[1] = t.y;
    r[2] = t.z;
    r[3] = t.w;
  }
  __device__ static void sts(float* p, const float* r) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(r[0], r[1], r[2], r[3]));
  }
};

// T is the storage and arithmetic type of the blocks and of A's values (FP64 path or
// the FP32 filter of the mixed path); column reductions always accumulate in FP64.
//
// A warp owns one row at a time and covers its columns in NC chunks of 32*VEC (all chunks
// of a chunk group in flight together): for every nonzero a_ij it issues NC independent
// vector loads of row j of Yin, and the rows of X and Z that the epilogue needs are
// requested before the gather loop, so each warp keeps 7*NC + 2*NC loads in flight on a
// 7-point stencil.  The grid is sized to the CTAs that are resident at once (a single
// wave); rows are dealt out in a fixed grid-stride order.
//
// The per-column multipliers depend only on the lane's columns: the FP32 kernel converts
// them once per chunk group into registers (an FP64->FP32 conversion per row would run on
// GB300's narrow FP64 pipe).  RED selects the column reduction (sum of out^2 or out*Yin),
// kept in FP64 registers per lane and reduced across the CTA at the end.
template <typename T, int VEC, int NC, bool RED>
__global__ void __launch_bounds__(SPMM_THREADS) spmm_fused_kernel(KParams<T> P) {
  extern __shared__ double s_red[];  // [SPMM_WARPS][ncols] when RED
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ncols = P.ncols;
  constexpr int CH = 32 * VEC;
  constexpr bool HOIST = sizeof(T) == 4;
  const int64_t first = static_cast<int64_t>(blockIdx.x) * SPMM_WARPS + warp;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * SPMM_WARPS;
  for (int g0 = 0; g0 < ncols; g0 += NC * CH) {
    int cc[NC];
    bool act[NC];
#pragma unroll
    for (int h = 0; h < NC; ++h) {
      cc[h] = g0 + h * CH + lane * VEC;
      act[h] = cc[h] < ncols;
    }
    T csy[HOIST ? NC : 1][VEC], csx[HOIST ? NC : 1][VEC], csz[HOIST ? NC : 1][VEC];
    if constexpr (HOIST) {
#pragma unroll
      for (int h = 0; h < NC; ++h)
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          const int c = act[h] ? cc[h] + u : 0;
          csy[h][u] = P.sy ? static_cast<T>(P.sy[c]) : T(1);
          csx[h][u] = P.X ? static_cast<T>(P.sx[c]) : T(0);
          csz[h][u] = P.Z ? static_cast<T>(P.sz[c]) : T(0);
        }
    }
    double red[RED ? NC : 1][VEC];
#pragma unroll
    for (int h = 0; h < (RED ? NC : 1); ++h)
#pragma unroll
      for (int u = 0; u < VEC; ++u) red[h][u] = 0.0;
    for (int64_t row = first; row < P.n; row += stride) {
      const int beg = __ldg(P.rowptr + row);
      const int end = __ldg(P.rowptr + row + 1);
      // epilogue operands first: their latency overlaps the gathers
      T xv[NC][VEC], zv[NC][VEC];
#pragma unroll
      for (int h = 0; h < NC; ++h) {
        if (P.X && act[h]) VecIO<T, VEC>::lds(P.X + row * P.ldx + cc[h], xv[h]);
        if (P.Z && act[h]) VecIO<T, VEC>::lds(P.Z + row * P.ldz + cc[h], zv[h]);
      }
      T acc[NC][VEC];
#pragma unroll
      for (int h = 0; h < NC; ++h)
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[h][u] = T(0);
      for (int base = beg; base < end; base += 32) {
        const int e = base + lane;
        int jc = 0;
        T av = T(0);
        if (e < end) {
          jc = __ldg(P.col + e);
          av = __ldg(P.val + e);
        }
        const int cnt = min(32, end - base);
#pragma unroll 2
        for (int t = 0; t < cnt; ++t) {
          const int j = __shfl_sync(0xffffffffu, jc, t);
          const T v = __shfl_sync(0xffffffffu, av, t);
          const T* yrow = P.Yin + static_cast<int64_t>(j) * P.ldy;
          T y[NC][VEC];
#pragma unroll
          for (int h = 0; h < NC; ++h)
            if (act[h]) VecIO<T, VEC>::ld(yrow + cc[h], y[h]);
#pragma unroll
          for (int h = 0; h < NC; ++h)
            if (act[h]) {
#pragma unroll
              for (int u = 0; u < VEC; ++u) acc[h][u] = fma(v, y[h][u], acc[h][u]);
            }
        }
      }
#pragma unroll
      for (int h = 0; h < NC; ++h) {
        if (!act[h]) continue;
        const int c = cc[h];
        T yi[VEC], o[VEC];
        if (P.beta != T(0) || (RED && P.dot_with_yin)) {
          VecIO<T, VEC>::ld(P.Yin + row * P.ldy + c, yi);
        } else {
#pragma unroll
          for (int u = 0; u < VEC; ++u) yi[u] = T(0);
        }
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          const T sy = HOIST ? csy[HOIST ? h : 0][u] : (P.sy ? static_cast<T>(P.sy[c + u]) : T(1));
          o[u] = sy * fma(P.alpha, acc[h][u], P.beta * yi[u]);
        }
        if (P.X) {
#pragma unroll
          for (int u = 0; u < VEC; ++u) {
            const T sx = HOIST ? csx[HOIST ? h : 0][u] : static_cast<T>(P.sx[c + u]);
            o[u] = fma(sx, xv[h][u], o[u]);
          }
        }
        if (P.Z) {
#pragma unroll
          for (int u = 0; u < VEC; ++u) {
            const T sz = HOIST ? csz[HOIST ? h : 0][u] : static_cast<T>(P.sz[c + u]);
            o[u] = fma(sz, zv[h][u], o[u]);
          }
        }
        if (P.out) VecIO<T, VEC>::sts(P.out + row * P.ldo + c, o);
        if constexpr (RED) {
#pragma unroll
          for (int u = 0; u < VEC; ++u) {
            const double od = static_cast<double>(o[u]);
            red[h][u] += P.dot_with_yin ? od * static_cast<double>(yi[u]) : od * od;
          }
        }
      }
    }
    if constexpr (RED) {
      double* my_red = s_red + static_cast<size_t>(warp) * ncols;
#pragma unroll
      for (int h = 0; h < NC; ++h)
        if (act[h])
#pragma unroll
          for (int u = 0; u < VEC; ++u) my_red[cc[h] + u] = red[h][u];
    }
  }
  if constexpr (RED) {
    __syncthreads();
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
      double s = 0.0;
      for (int w = 0; w < SPMM_WARPS; ++w) s += s_red[static_cast<size_t>(w) * ncols + c];
      P.red_part[static_cast<size_t>(blockIdx.x) * ncols + c] = s;
    }
  }
}

__global__ void to_float_kernel(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < n) dst[t] = static_cast<float>(src[t]);
}

// out[c] = sum_b part[b][c]: one block per column, fixed strided partial sums and a fixed
// tree, so the result does not depend on scheduling (deterministic).
__global__ void reduce_partials_kernel(const double* __restrict__ part, int nb, int ncols,
                                       double* __restrict__ out) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[static_cast<size_t>(b) * ncols + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// Per-block Gershgorin bounds: lo = min(a_ii - r_i), hi = max(a_ii + r_i).
__global__ void gershgorin_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                  double* __restrict__ part) {
  __shared__ double slo[256], shi[256];
  double lo = 1e308, hi = -1e308;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double d = 0.0, r = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      if (col[e] == i) d += val[e];
      else r += fabs(val[e]);
    }
    lo = fmin(lo, d - r);
    hi = fmax(hi, d + r);
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = slo[0];
    part[2 * blockIdx.x + 1] = shi[0];
  }
}

__global__ void gershgorin_final_kernel(const double* __restrict__ part, int nb,
                                        double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double lo = 1e308, hi = -1e308;
  for (int b = 0; b < nb; ++b) {
    lo = fmin(lo, part[2 * b]);
    hi = fmax(hi, part[2 * b + 1]);
  }
  out[0] = lo;
  out[1] = hi;
}

// Per-block column sums of squares of rows [b*rows, (b+1)*rows).
__global__ void col_sumsq_kernel(int64_t n, const double* __restrict__ X, int64_t ldx, int ncols,
                                 int64_t rows_per_block, double* __restrict__ part) {
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      const double x = X[r * ldx + c];
      s = fma(x, x, s);
    }
    part[static_cast<size_t>(blockIdx.x) * ncols + c] = s;
  }
}

// One wave: as many CTAs as are resident at once (at most the rows need), so no second,
// partly empty wave of CTAs runs at the end.  With want_red, the per-CTA partial column
// sums go to a workspace of grid x ncols doubles (returned with the grid).
template <typename T, int VEC, int NC>
arb_status launch_spmm(arb_ctx ctx, KParams<T> P, size_t smem, bool want_red, int* grid_out,
                       double** part_out) {
  void (*kern)(KParams<T>) = want_red ? spmm_fused_kernel<T, VEC, NC, true> : spmm_fused_kernel<T, VEC, NC, false>;
  ARB_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  int per_sm = 0;
  ARB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SPMM_THREADS, smem));
  const int64_t want = (P.n + SPMM_WARPS - 1) / SPMM_WARPS;
  int grid = static_cast<int>(std::min<int64_t>(want, static_cast<int64_t>(ctx->num_sms) * std::max(per_sm, 1)));
  grid = std::max(grid, 1);
  P.red_part = nullptr;
  if (want_red) ARB_TRY(ws<double>(ctx, WS_SS_PART, static_cast<size_t>(grid) * P.ncols, &P.red_part));
  kern<<<grid, SPMM_THREADS, smem, ctx->stream>>>(P);
  ARB_LAUNCHED(ctx);
  *grid_out = grid;
  *part_out = P.red_part;
  return ARB_OK;
}

template <typename T, int VEC>
arb_status launch_spmm_nc(arb_ctx ctx, const KParams<T>& P, size_t smem, bool want_red, int* grid,
                          double** part) {
  constexpr int CH = 32 * VEC;
  const int chunks = (P.ncols + CH - 1) / CH;
  // wider blocks loop over groups of (at most) 4 chunks: more would spill registers
  if (chunks <= 1) return launch_spmm<T, VEC, 1>(ctx, P, smem, want_red, grid, part);
  if (chunks <= 2) return launch_spmm<T, VEC, 2>(ctx, P, smem, want_red, grid, part);
  return launch_spmm<T, VEC, 4>(ctx, P, smem, want_red, grid, part);
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <typename T>
const T* values_of(const arb_mat_s* A);
template <>
const double* values_of<double>(const arb_mat_s* A) {
  return A->val;
}
template <>
const float* values_of<float>(const arb_mat_s* A) {
  return A->val32;
}

}  // namespace

arb_status ensure_val32(arb_ctx ctx, arb_mat mat) {
  if (mat->val32) return ARB_OK;
  ARB_CUDA(ctx, cudaMalloc(&mat->val32, std::max<int64_t>(mat->nnz, 1) * sizeof(float)));
  if (mat->nnz > 0) {
    to_float_kernel<<<static_cast<int>((mat->nnz + 255) / 256), 256, 0, ctx->stream>>>(mat->nnz, mat->val,
                                                                                     mat->val32);
    ARB_LAUNCHED(ctx);
  }
  return ARB_OK;
}

template <typename T>
arb_status spmm_fused(arb_ctx ctx, const SpmmArgs<T>& a) {
  const arb_mat_s* A = a.A;
  if (a.ncols <= 0 || A->n <= 0) return ARB_OK;
  if (a.ncols > 6000) return set_error(ctx, ARB_INVALID_ARG, "spmm: ncols too large");
  if (!values_of<T>(A)) return set_error(ctx, ARB_INVALID_ARG, "spmm: matrix has no values of this precision");
  KParams<T> P;
  P.n = A->n;
  P.rowptr = A->rowptr;
  P.col = A->col;
  P.val = values_of<T>(A);
  P.ncols = a.ncols;
  P.Yin = a.Yin;
  P.ldy = a.ldy;
  P.alpha = static_cast<T>(a.alpha);
  P.beta = static_cast<T>(a.beta);
  P.sy = a.sy;
  P.X = a.X;
  P.ldx = a.ldx;
  P.sx = a.sx;
  P.Z = a.Z;
  P.ldz = a.ldz;
  P.sz = a.sz;
  P.out = a.out;
  P.ldo = a.ldo;
  P.dot_with_yin = a.dot_with_yin ? 1 : 0;
  P.red_part = nullptr;
  size_t smem = 0;
  const bool want_red = a.colred != nullptr;
  if (want_red) {
    smem = static_cast<size_t>(SPMM_WARPS) * a.ncols * sizeof(double);
    if (smem > 200 * 1024) return set_error(ctx, ARB_INVALID_ARG, "spmm: too many columns for reduction");
  }
  // widest vector access that the column count, leading dimensions and bases allow
  auto fits = [&](int v) {
    const size_t bytes = v * sizeof(T);
    bool ok = (a.ncols % v == 0) && (a.ldy % v == 0) && aligned(a.Yin, bytes);
    if (a.X) ok = ok && (a.ldx % v == 0) && aligned(a.X, bytes);
    if (a.Z) ok = ok && (a.ldz % v == 0) && aligned(a.Z, bytes);
    if (a.out) ok = ok && (a.ldo % v == 0) && aligned(a.out, bytes);
    return ok && a.ncols > 32 * (v / 2);
  };
  int grid = 0;
  double* part = nullptr;
  if constexpr (sizeof(T) == 4) {
    if (fits(4)) {
      ARB_TRY((launch_spmm_nc<T, 4>(ctx, P, smem, want_red, &grid, &part)));
    } else if (fits(2)) {
      ARB_TRY((launch_spmm_nc<T, 2>(ctx, P, smem, want_red, &grid, &part)));
    } else {
      ARB_TRY((launch_spmm_nc<T, 1>(ctx, P, smem, want_red, &grid, &part)));
    }
  } else {
    if (fits(2)) {
      ARB_TRY((launch_spmm_nc<T, 2>(ctx, P, smem, want_red, &grid, &part)));
    } else {
      ARB_TRY((launch_spmm_nc<T, 1>(ctx, P, smem, want_red, &grid, &part)));
    }
  }
  if (want_red) {
    reduce_partials_kernel<<<a.ncols, 256, 0, ctx->stream>>>(part, grid, a.ncols, a.colred);
    ARB_LAUNCHED(ctx);
  }
  return ARB_OK;
}

template arb_status spmm_fused<double>(arb_ctx, const SpmmArgs<double>&);
template arb_status spmm_fused<float>(arb_ctx, const SpmmArgs<float>&);

arb_status gershgorin(arb_ctx ctx, arb_mat mat, double* lo, double* hi) {
  if (mat->gersh_valid) {
    *lo = mat->gersh_lo;
    *hi = mat->gersh_hi;
    return ARB_OK;
  }
  const int grid = std::max(1, std::min(ctx->num_sms * 4, static_cast<int>((mat->n + 255) / 256)));
  double* part;
  ARB_TRY(ws<double>(ctx, WS_VEC2, 2 * static_cast<size_t>(grid) + 2, &part));
  gershgorin_kernel<<<grid, 256, 0, ctx->stream>>>(mat->n, mat->rowptr, mat->col, mat->val, part);
  ARB_LAUNCHED(ctx);
  gershgorin_final_kernel<<<1, 32, 0, ctx->stream>>>(part, grid, part + 2 * grid);
  ARB_LAUNCHED(ctx);
  double h[2];
  ARB_TRY(d2h_sync(ctx, h, part + 2 * grid, sizeof(h)));
  mat->gersh_lo = h[0];
  mat->gersh_hi = h[1];
  mat->gersh_valid = true;
  *lo = h[0];
  *hi = h[1];
  return ARB_OK;
}

arb_status col_sumsq(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t ncols,
                     double* out) {
  if (ncols <= 0) return ARB_OK;
  const int64_t target = static_cast<int64_t>(ctx->num_sms) * 4;
  int64_t rows = std::max<int64_t>(1, (n + target - 1) / target);
  const int grid = static_cast<int>((n + rows - 1) / rows);
  double* part;
  ARB_TRY(ws<double>(ctx, WS_SS_PART, static_cast<size_t>(grid) * ncols, &part));
  col_sumsq_kernel<<<grid, 256, 0, ctx->stream>>>(n, X, ldx, ncols, rows, part);
  ARB_LAUNCHED(ctx);
  reduce_partials_kernel<<<ncols, 256, 0, ctx->stream>>>(part, grid, ncols, out);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

}  // namespace arb
