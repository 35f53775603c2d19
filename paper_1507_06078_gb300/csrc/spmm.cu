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
#include <type_traits>

#include "arb_internal.h"

namespace arb {
namespace {

constexpr int SPMM_THREADS = 256;
constexpr int SPMM_WARPS = SPMM_THREADS / 32;
// Tuning defaults (measured on the 128^3 x 240 filter): widest FP32 vector access per lane,
// gathers issued per batch, and the CTAs per SM the register budget must allow.
#ifndef ARB_SPMM_F32_MAX_VEC
#define ARB_SPMM_F32_MAX_VEC 4
#endif
#ifndef ARB_SPMM_UNROLL
#define ARB_SPMM_UNROLL 4
#endif
#ifndef ARB_SPMM_MIN_BLOCKS
#define ARB_SPMM_MIN_BLOCKS 3
#endif
#ifndef ARB_SPMM_SHORT_UNROLL
#define ARB_SPMM_SHORT_UNROLL 4
#endif
// 1: short-row FP32 products by the bulk-copy pipelined kernel (spmm_bulk.cu); measured at
// 2.6-2.8 ms per 128^3 x 240 filter pass against 2.0 ms for this kernel, so off by default
#ifndef ARB_SPMM_BULK
#define ARB_SPMM_BULK 0
#endif
// 1: every CTA walks a contiguous range of rows (neighbouring rows' gathers meet in its L1)
// instead of the grid sweeping the rows as one interleaved front
#ifndef ARB_SPMM_CONTIG
#define ARB_SPMM_CONTIG 0
#endif


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
  // SELL-C-sigma (MODE 2): sorted position i holds block row perm[i], of slen[i] nonzeros
  // stored at slots scptr[i / sellC] + i % sellC + e * sellC (e = 0 .. slen[i] - 1)
  const int32_t* perm;
  const int32_t* slen;
  const int64_t* scptr;
  int sellC;
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
// Work split: a row's columns are cut into nch chunks of 32*VEC; every warp owns one
// fixed chunk (warp id mod nch) and walks the rows dealt to it in a fixed grid-stride
// order, so its lanes always touch the same columns and the per-column multipliers are
// loaded (and, for FP32, converted) once into registers instead of once per row.  For
// every row the warp first requests the epilogue rows of X and Z, then gathers the rows
// of Yin named by the row's nonzeros in batches of UNR loads issued back to back before
// any of them is used: on a 7-point stencil all 7 gathers and both epilogue rows are in
// flight together.  The grid is the number of CTAs resident at once (one wave).
// RED adds the column reduction (sum of out^2 or out*Yin) in FP64 registers, combined per
// CTA through shared memory.
//
// MODE 0: CSR.  MODE 2: SELL-C-sigma - rows taken in their sorted order (longest first within
// each sigma window, so the warps of a CTA get rows of similar length), each row's indices
// and values read from its chunk's column-major slots; the block rows it reads and writes
// are the original ones (perm), so the result is the same, summed in the same order.
// MODE 1, SHORT (every row has at most 32 nonzeros, e.g. stencils, and every block has fewer than
// 2^31 elements): the index loads of a row are software-pipelined across the warp's rows -
// the row pointers two rows ahead, the column indices and values one row ahead - so a row
// waits only on its gathers, not on the chain rowptr -> col -> Yin of three dependent
// loads; element offsets are 32-bit products.
template <typename T, int VEC, bool RED, int MODE>
__global__ void __launch_bounds__(SPMM_THREADS, ARB_SPMM_MIN_BLOCKS) spmm_fused_kernel(KParams<T> P) {
  constexpr bool SHORT = MODE == 1, SELL = MODE == 2;
  extern __shared__ double s_red[];  // [SPMM_WARPS][ncols] when RED
  constexpr int CH = 32 * VEC;
  constexpr int UNR = SHORT ? ARB_SPMM_SHORT_UNROLL : ARB_SPMM_UNROLL;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ncols = P.ncols;
  const int nch = (ncols + CH - 1) / CH;
  if constexpr (RED) {
    for (int c = lane; c < ncols; c += 32) s_red[static_cast<size_t>(warp) * ncols + c] = 0.0;
    __syncwarp();
  }
  // ARB_SPMM_CONTIG: every CTA walks its own contiguous range of rows, SPMM_WARPS / nch rows
  // at a time (when every chunk gets a warp); otherwise the grid sweeps the rows as one
  // interleaved front, warp gw taking rows gw / nch + k (nwarps / nch)
  const bool contig = ARB_SPMM_CONTIG && nch <= SPMM_WARPS;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * SPMM_WARPS + warp;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * SPMM_WARPS;
  const int wpc = SPMM_WARPS / nch;  // warps per chunk in a CTA (contiguous ranges)
  const int64_t rows_per_cta = (P.n + gridDim.x - 1) / gridDim.x;
  const int chunk = contig ? warp % nch : static_cast<int>(gw % nch);
  const int64_t r_first = contig ? static_cast<int64_t>(blockIdx.x) * rows_per_cta + warp / nch : gw / nch;
  const int64_t rstride = contig ? static_cast<int64_t>(wpc) : nwarps / nch;
  const int64_t r_end = contig ? min(P.n, static_cast<int64_t>(blockIdx.x + 1) * rows_per_cta) : P.n;
  const bool live = contig ? warp < wpc * nch : r_first < rstride;
  const int c = chunk * CH + lane * VEC;
  const bool act = live && (c < ncols);
  // lanes past the last column load column 0 of the same rows (always in bounds) and
  // discard the result, so the gathers need no per-lane predicate
  const int cl = act ? c : 0;
  T csy[VEC], csx[VEC], csz[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) {
    const int cu = act ? c + u : 0;
    csy[u] = P.sy ? static_cast<T>(P.sy[cu]) : T(1);
    csx[u] = P.X ? static_cast<T>(P.sx[cu]) : T(0);
    csz[u] = P.Z ? static_cast<T>(P.sz[cu]) : T(0);
  }
  // column reductions: FP64 for FP64 blocks; for FP32 blocks double-float pairs (FP32 hi,
  // lo with error-free product and sum transforms), which keep the FP64 pipe (a small
  // fraction of the FP32 rate on this GPU) out of the row loop
  double red[VEC];
  float rhi[VEC], rlo[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) {
    red[u] = 0.0;
    rhi[u] = rlo[u] = 0.f;
  }
  // SHORT pipeline state: indices of the next row, row pointers of the one after
  int n_jc = 0, n_cnt = 0, p_beg = 0, p_end = 0;
  T n_av = T(0);
  if (SHORT && live && r_first < r_end) {
    const int b0 = __ldg(P.rowptr + r_first), e0 = __ldg(P.rowptr + r_first + 1);
    n_cnt = e0 - b0;
    if (lane < n_cnt) {
      n_jc = __ldg(P.col + b0 + lane);
      n_av = __ldg(P.val + b0 + lane);
    }
    if (r_first + rstride < r_end) {
      p_beg = __ldg(P.rowptr + r_first + rstride);
      p_end = __ldg(P.rowptr + r_first + rstride + 1);
    }
  }
  if (live) {
    for (int64_t row = r_first; row < r_end; row += rstride) {
      int beg = 0, end = 0, s_jc = 0;
      T s_av = T(0);
      int64_t orow = row;  // the block row (SELL: the sorted position's original row)
      int64_t sbase = 0;   // SELL: slot of the row's first nonzero
      if constexpr (SHORT) {
        s_jc = n_jc;
        s_av = n_av;
        end = n_cnt;  // the row's nonzeros are lanes 0..n_cnt-1 of (s_jc, s_av)
        const int64_t r1 = row + rstride, r2 = row + 2 * rstride;
        n_cnt = 0;
        n_jc = 0;
        n_av = T(0);
        if (r1 < r_end) {
          n_cnt = p_end - p_beg;
          if (lane < n_cnt) {
            n_jc = __ldg(P.col + p_beg + lane);
            n_av = __ldg(P.val + p_beg + lane);
          }
        }
        if (r2 < r_end) {
          p_beg = __ldg(P.rowptr + r2);
          p_end = __ldg(P.rowptr + r2 + 1);
        }
      } else if constexpr (SELL) {
        orow = __ldg(P.perm + row);
        end = __ldg(P.slen + row);
        sbase = __ldg(P.scptr + row / P.sellC) + row % P.sellC;
      } else {
        beg = __ldg(P.rowptr + row);
        end = __ldg(P.rowptr + row + 1);
      }
      // element offset of (r, c) in a block of leading dimension ld
      auto off = [&](int64_t r, int64_t ld) -> int64_t {
        if constexpr (SHORT) return static_cast<int64_t>(static_cast<uint32_t>(r) * static_cast<uint32_t>(ld));
        else return r * ld;
      };
      T xv[VEC], zv[VEC], yi[VEC];
      if (P.X) VecIO<T, VEC>::lds(P.X + off(orow, P.ldx) + cl, xv);
      if (P.Z) VecIO<T, VEC>::lds(P.Z + off(orow, P.ldz) + cl, zv);
      // the row's own entries of Yin with them, ahead of the gathers (not after the sums)
      const bool need_yi = P.beta != T(0) || (RED && P.dot_with_yin);
      if (need_yi) VecIO<T, VEC>::ld(P.Yin + off(orow, P.ldy) + cl, yi);
      T acc[VEC];
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[u] = T(0);
      for (int base = beg; base < end; base += 32) {
        int jc = 0;
        T av = T(0);
        if constexpr (SHORT) {
          jc = s_jc;
          av = s_av;
        } else {
          const int e = base + lane;
          if (e < end) {
            const int64_t idx = SELL ? sbase + static_cast<int64_t>(e) * P.sellC : static_cast<int64_t>(e);
            jc = __ldg(P.col + idx);
            av = __ldg(P.val + idx);
          }
        }
        const int cnt = __shfl_sync(0xffffffffu, min(32, end - base), 0);  // warp-uniform
        for (int t0 = 0; t0 < cnt; t0 += UNR) {
          int jj[UNR];
          T vv[UNR];
#pragma unroll
          for (int t = 0; t < UNR; ++t) {
            jj[t] = __shfl_sync(0xffffffffu, jc, t0 + t < 32 ? t0 + t : 31);
            vv[t] = __shfl_sync(0xffffffffu, av, t0 + t < 32 ? t0 + t : 31);
          }
          T y[UNR][VEC];
#pragma unroll
          for (int t = 0; t < UNR; ++t)
            if (t0 + t < cnt) VecIO<T, VEC>::ld(P.Yin + off(jj[t], P.ldy) + cl, y[t]);
#pragma unroll
          for (int t = 0; t < UNR; ++t) {
            if (t0 + t < cnt) {
              if constexpr (std::is_same<T, float>::value && VEC % 2 == 0) {
                // packed FP32 (two lanes of one FFMA2 instruction): half the issue slots
                const float2 v2 = make_float2(vv[t], vv[t]);
#pragma unroll
                for (int u = 0; u < VEC; u += 2) {
                  const float2 r = __ffma2_rn(v2, make_float2(y[t][u], y[t][u + 1]), make_float2(acc[u], acc[u + 1]));
                  acc[u] = r.x;
                  acc[u + 1] = r.y;
                }
              } else {
#pragma unroll
                for (int u = 0; u < VEC; ++u) acc[u] = fma(vv[t], y[t][u], acc[u]);
              }
            }
          }
        }
      }
      if (!act) continue;
      T o[VEC];
      if (!need_yi) {
#pragma unroll
        for (int u = 0; u < VEC; ++u) yi[u] = T(0);
      }
      if constexpr (std::is_same<T, float>::value && VEC % 2 == 0) {
        // the same operations, two columns per packed instruction
        const float2 al2 = make_float2(P.alpha, P.alpha), be2 = make_float2(P.beta, P.beta);
#pragma unroll
        for (int u = 0; u < VEC; u += 2) {
          float2 r = __fmul2_rn(be2, make_float2(yi[u], yi[u + 1]));
          r = __ffma2_rn(al2, make_float2(acc[u], acc[u + 1]), r);
          r = __fmul2_rn(make_float2(csy[u], csy[u + 1]), r);
          if (P.X) r = __ffma2_rn(make_float2(csx[u], csx[u + 1]), make_float2(xv[u], xv[u + 1]), r);
          if (P.Z) r = __ffma2_rn(make_float2(csz[u], csz[u + 1]), make_float2(zv[u], zv[u + 1]), r);
          o[u] = r.x;
          o[u + 1] = r.y;
        }
      } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u) o[u] = csy[u] * fma(P.alpha, acc[u], P.beta * yi[u]);
        if (P.X) {
#pragma unroll
          for (int u = 0; u < VEC; ++u) o[u] = fma(csx[u], xv[u], o[u]);
        }
        if (P.Z) {
#pragma unroll
          for (int u = 0; u < VEC; ++u) o[u] = fma(csz[u], zv[u], o[u]);
        }
      }
      if (P.out) VecIO<T, VEC>::sts(P.out + off(orow, P.ldo) + c, o);
      if constexpr (RED) {
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          if constexpr (std::is_same<T, float>::value) {
            const float b = P.dot_with_yin ? yi[u] : o[u];
            const float pr = o[u] * b;
            const float pe = fmaf(o[u], b, -pr);
            const float sm = rhi[u] + pr;
            const float bp = sm - rhi[u];
            rlo[u] += ((rhi[u] - (sm - bp)) + (pr - bp)) + pe;
            rhi[u] = sm;
          } else {
            const double od = static_cast<double>(o[u]);
            red[u] += P.dot_with_yin ? od * static_cast<double>(yi[u]) : od * od;
          }
        }
      }
    }
  }
  if constexpr (RED) {
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
      for (int u = 0; u < VEC; ++u) red[u] = static_cast<double>(rhi[u]) + static_cast<double>(rlo[u]);
    }
    if (act)
#pragma unroll
      for (int u = 0; u < VEC; ++u) s_red[static_cast<size_t>(warp) * ncols + c + u] = red[u];
    __syncthreads();
    for (int cc = threadIdx.x; cc < ncols; cc += blockDim.x) {
      double sum = 0.0;
      for (int w = 0; w < SPMM_WARPS; ++w) sum += s_red[static_cast<size_t>(w) * ncols + cc];
      P.red_part[static_cast<size_t>(blockIdx.x) * ncols + cc] = sum;
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

// One wave: as many CTAs as are resident at once (at most what the rows need), so no
// second, partly empty wave of CTAs runs at the end.  With want_red, the per-CTA partial
// column sums go to a workspace of grid x ncols doubles (returned with the grid).
template <typename T, int VEC>
arb_status launch_spmm(arb_ctx ctx, KParams<T> P, size_t smem, bool want_red, int mode, int* grid_out,
                       double** part_out) {
  void (*kern)(KParams<T>) =
      mode == 2   ? (want_red ? spmm_fused_kernel<T, VEC, true, 2> : spmm_fused_kernel<T, VEC, false, 2>)
      : mode == 1 ? (want_red ? spmm_fused_kernel<T, VEC, true, 1> : spmm_fused_kernel<T, VEC, false, 1>)
                  : (want_red ? spmm_fused_kernel<T, VEC, true, 0> : spmm_fused_kernel<T, VEC, false, 0>);
  ARB_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  int per_sm = 0;
  ARB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SPMM_THREADS, smem));
  const int nch = (P.ncols + 32 * VEC - 1) / (32 * VEC);
  const int64_t want = (P.n * nch + SPMM_WARPS - 1) / SPMM_WARPS;
  int grid = static_cast<int>(std::min<int64_t>(want, static_cast<int64_t>(ctx->num_sms) * std::max(per_sm, 1)));
  // every chunk needs at least one warp
  grid = std::max(grid, (nch + SPMM_WARPS - 1) / SPMM_WARPS);
  P.red_part = nullptr;
  if (want_red) ARB_TRY(ws<double>(ctx, WS_SS_PART, static_cast<size_t>(grid) * P.ncols, &P.red_part));
  kern<<<grid, SPMM_THREADS, smem, ctx->stream>>>(P);
  ARB_LAUNCHED(ctx);
  *grid_out = grid;
  *part_out = P.red_part;
  return ARB_OK;
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <typename T>
const T* values_of(const arb_mat_s* A);
template <>
const double* values_of<double>(const arb_mat_s* A) {
  return A->sell_C > 0 ? A->sell_val : A->val;
}
template <>
const float* values_of<float>(const arb_mat_s* A) {
  return A->sell_C > 0 ? A->sell_val32 : A->val32;
}

}  // namespace

arb_status ensure_val32(arb_ctx ctx, arb_mat mat) {
  std::lock_guard<std::mutex> lock(mat->mu);
  if (mat->val32) return ARB_OK;
  float* v = nullptr;
  ARB_CUDA(ctx, cudaMalloc(&v, std::max<int64_t>(mat->nnz, 1) * sizeof(float)));
  if (mat->nnz > 0) {
    to_float_kernel<<<static_cast<int>((mat->nnz + 255) / 256), 256, 0, ctx->stream>>>(mat->nnz, mat->val, v);
    ARB_LAUNCHED(ctx);
  }
  // other contexts (other streams) may use the copy next: make it complete first
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  mat->val32 = v;
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
  P.col = A->sell_C > 0 ? A->sell_col : A->col;
  P.val = values_of<T>(A);
  P.perm = A->sell_perm;
  P.slen = A->sell_len;
  P.scptr = A->sell_cptr;
  P.sellC = A->sell_C;
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
    // the matrix's tuned width caps the access (arb_matrix_autotune)
    if (A->tune_vec > 0 && v > A->tune_vec) return false;
    return ok && a.ncols > 32 * (v / 2);
  };
  int grid = 0;
  double* part = nullptr;
  int64_t ld_max = a.ldy;
  if (a.X) ld_max = std::max(ld_max, a.ldx);
  if (a.Z) ld_max = std::max(ld_max, a.ldz);
  if (a.out) ld_max = std::max(ld_max, a.ldo);
  const bool short_rows = A->max_row_nnz >= 0 && A->max_row_nnz <= 32 && A->n * ld_max < (int64_t(1) << 31);
  const int mode = A->sell_C > 0 ? 2 : (short_rows ? 1 : 0);
  if constexpr (sizeof(T) == 4) {
    bool bulk = false;
#if ARB_SPMM_BULK
    if (mode == 1) ARB_TRY(spmm_bulk_f32(ctx, A, a, P.val, want_red, &bulk, &grid, &part));
#endif
    if (bulk) {
      // done by the bulk-copy pipelined kernel
    } else if (ARB_SPMM_F32_MAX_VEC >= 4 && fits(4)) {
      ARB_TRY((launch_spmm<T, 4>(ctx, P, smem, want_red, mode, &grid, &part)));
    } else if (fits(2)) {
      ARB_TRY((launch_spmm<T, 2>(ctx, P, smem, want_red, mode, &grid, &part)));
    } else {
      ARB_TRY((launch_spmm<T, 1>(ctx, P, smem, want_red, mode, &grid, &part)));
    }
  } else {
    if (fits(2)) {
      ARB_TRY((launch_spmm<T, 2>(ctx, P, smem, want_red, mode, &grid, &part)));
    } else {
      ARB_TRY((launch_spmm<T, 1>(ctx, P, smem, want_red, mode, &grid, &part)));
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
  std::lock_guard<std::mutex> lock(mat->mu);
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
