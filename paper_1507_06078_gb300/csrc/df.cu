// Double-float ("df") blocks for the refinement filter of the mixed path.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so an FP64 filter pass is bound by
// the FP64 pipe (about 5x its HBM time).  A df element stores a value as an unevaluated
// sum hi + lo of two FP32 numbers (8 bytes, the same traffic as FP64) and the arithmetic
// uses only the FP32 pipe: products by the FMA-based exact product (Dekker / Kahan:
// p = a*b, e = fma(a, b, -p)), sums by Knuth's two-sum followed by a fast renormalising
// two-sum.  That carries about 2^-44 relative accuracy per operation, far below the
// 1e-8 residuals and 1e-10 eigenvalue errors the solver is run to; the Rayleigh-Ritz
// steps, residuals and reported eigenvalues stay in true FP64.
//
// Block layout ("paired planar"): row-major with an even leading dimension ld (in df
// elements); the columns 2j and 2j+1 of a row are the four floats
// [hi(2j), hi(2j+1), lo(2j), lo(2j+1)], so one 16-byte load gives a lane the hi parts and
// the lo parts of its two columns as float2 pairs, the operands of the packed FP32x2
// instructions (FFMA2 / FADD2 / FMUL2) that do the arithmetic of both columns at once.
#include <algorithm>

#include "arb_internal.h"
#include "df_arith.cuh"

namespace arb {
namespace {

constexpr int DF_THREADS = 256;
constexpr int DF_WARPS = DF_THREADS / 32;

struct DfParams {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const df2* val;
  int32_t ncols;
  const df2* Yin;
  int64_t ldy;
  double alpha, beta;
  const double* sy;
  const df2* X;
  int64_t ldx;
  const double* sx;
  const df2* Z;
  int64_t ldz;
  const double* sz;
  df2* out;
  int64_t ldo;
  double* red_part;
  int dot_with_yin;
  const int32_t* perm;  // SELL-C-sigma (MODE 2), as in the FP32/FP64 kernel
  const int32_t* slen;
  const int64_t* scptr;
  int sellC;
};

// one 16-byte load of a column pair of a paired planar block
__device__ __forceinline__ dfp ldp(const df2* p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  return dfp{make_float2(t.x, t.y), make_float2(t.z, t.w)};
}
__device__ __forceinline__ dfp ldps(const df2* p) {
  const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
  return dfp{make_float2(t.x, t.y), make_float2(t.z, t.w)};
}

// Tuning defaults (measured on the 128^3 x 240 filter): gathers in flight per lane, the CTAs
// per SM the register budget must allow, and column pairs per lane.  Measured and dropped:
// parking the epilogue multipliers in shared memory and splitting the sum over two
// accumulators (both slower at this occupancy), 3 CTAs per SM (spills), 2 pairs per lane.
#ifndef ARB_DF_BATCH
#define ARB_DF_BATCH 8
#endif
#ifndef ARB_DF_MIN_BLOCKS
#define ARB_DF_MIN_BLOCKS 2
#endif
#ifndef ARB_DF_NP
#define ARB_DF_NP 1
#endif
constexpr int DF_BATCH = ARB_DF_BATCH;
constexpr int DF_NP = ARB_DF_NP;
constexpr int DF_CH = 64 * DF_NP;  // columns per warp chunk

__device__ __forceinline__ float4 pack4(const dfp& a) { return make_float4(a.hi.x, a.hi.y, a.lo.x, a.lo.y); }

// A warp owns a fixed chunk of 64 DF_NP columns - DF_NP column pairs per lane, pair u at
// columns chunk * DF_CH + 64 u + 2 lane, so every 16-byte load of a pair is one coalesced
// 512-byte warp access - and walks its rows, gathers issued DF_BATCH at a time, as in the
// FP32/FP64 fused kernel.  Leading dimensions are even and bases 16-byte aligned; for odd
// ncols the pad column (ld >= ncols + 1) is read and written but never reduced.
// MODE 0: CSR; MODE 2: SELL-C-sigma (rows in sorted order, indices and values from the chunk
// slots, block rows through perm).
// MODE 1, SHORT (rows of at most 32 nonzeros, blocks below 2^31 elements): row pointers loaded two
// rows ahead, column indices and values one row ahead, 32-bit element offsets.
template <bool RED, int MODE>
__global__ void __launch_bounds__(DF_THREADS, ARB_DF_MIN_BLOCKS) spmm_df_kernel(DfParams P) {
  constexpr bool SHORT = MODE == 1, SELL = MODE == 2;
  extern __shared__ double s_red[];  // RED: [DF_WARPS][ncols]
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ncols = P.ncols;
  const int nch = (ncols + DF_CH - 1) / DF_CH;
  if constexpr (RED) {
    for (int c = lane; c < ncols; c += 32) s_red[static_cast<size_t>(warp) * ncols + c] = 0.0;
    __syncwarp();
  }
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * DF_WARPS + warp;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * DF_WARPS;
  const int64_t rstride = nwarps / nch;
  const int chunk = static_cast<int>(gw % nch);
  const int64_t r_first = gw / nch;
  const bool live = r_first < rstride;
  int cp[DF_NP], cl[DF_NP];
  bool act[DF_NP], act1[DF_NP];
#pragma unroll
  for (int u = 0; u < DF_NP; ++u) {
    cp[u] = chunk * DF_CH + 64 * u + lane * 2;
    act[u] = live && (cp[u] < ncols);
    act1[u] = act[u] && (cp[u] + 1 < ncols);  // odd ncols: the pad column is carried, not reduced
    // lanes past the last column load columns 0-1 of the same rows (always in bounds) and
    // discard the result, so the gathers need no per-lane predicate
    cl[u] = act[u] ? cp[u] : 0;
  }
  // out = ka (A Yin) + kb Yin + kx X + kz Z with ka = sy alpha, kb = sy beta, kx = sx, kz = sz
  dfp kmul[4][DF_NP];
  {
    const df2 alpha = df_from(P.alpha), beta = df_from(P.beta);
#pragma unroll
    for (int u = 0; u < DF_NP; ++u) {
      df2 a[2], b[2], x[2], z[2];
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int cu = (act[u] && cp[u] + v < ncols) ? cp[u] + v : 0;
        const df2 sy = df_from(P.sy ? P.sy[cu] : 1.0);
        a[v] = df_mul(sy, alpha);
        b[v] = df_mul(sy, beta);
        x[v] = df_from(P.X ? P.sx[cu] : 0.0);
        z[v] = df_from(P.Z ? P.sz[cu] : 0.0);
      }
      kmul[0][u] = dfp_of(a[0], a[1]);
      kmul[1][u] = dfp_of(b[0], b[1]);
      kmul[2][u] = dfp_of(x[0], x[1]);
      kmul[3][u] = dfp_of(z[0], z[1]);
    }
  }
  auto off = [&](int64_t r, int64_t ld) -> int64_t {
    if constexpr (SHORT) return static_cast<int64_t>(static_cast<uint32_t>(r) * static_cast<uint32_t>(ld));
    else return r * ld;
  };
  const bool has_beta = P.beta != 0.0;  // one FP64 compare per thread, not one per row
  const bool need_yi = has_beta || (RED && P.dot_with_yin);
  const dfp zero{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  double red[DF_NP][2];
#pragma unroll
  for (int u = 0; u < DF_NP; ++u) red[u][0] = red[u][1] = 0.0;
  int n_jc = 0, n_cnt = 0, p_beg = 0, p_end = 0;
  float n_ah = 0.f, n_al = 0.f;
  if (SHORT && live && r_first < P.n) {
    const int b0 = __ldg(P.rowptr + r_first), e0 = __ldg(P.rowptr + r_first + 1);
    n_cnt = e0 - b0;
    if (lane < n_cnt) {
      n_jc = __ldg(P.col + b0 + lane);
      const float2 v = __ldg(reinterpret_cast<const float2*>(P.val) + b0 + lane);
      n_ah = v.x;
      n_al = v.y;
    }
    if (r_first + rstride < P.n) {
      p_beg = __ldg(P.rowptr + r_first + rstride);
      p_end = __ldg(P.rowptr + r_first + rstride + 1);
    }
  }
  if (live) {
    for (int64_t row = r_first; row < P.n; row += rstride) {
      int beg = 0, end = 0, s_jc = 0;
      float s_ah = 0.f, s_al = 0.f;
      int64_t orow = row;  // the block row (SELL: the sorted position's original row)
      int64_t sbase = 0;   // SELL: slot of the row's first nonzero
      if constexpr (SHORT) {
        s_jc = n_jc;
        s_ah = n_ah;
        s_al = n_al;
        end = n_cnt;
        const int64_t r1 = row + rstride, r2 = row + 2 * rstride;
        n_cnt = 0;
        n_jc = 0;
        n_ah = n_al = 0.f;
        if (r1 < P.n) {
          n_cnt = p_end - p_beg;
          if (lane < n_cnt) {
            n_jc = __ldg(P.col + p_beg + lane);
            const float2 v = __ldg(reinterpret_cast<const float2*>(P.val) + p_beg + lane);
            n_ah = v.x;
            n_al = v.y;
          }
        }
        if (r2 < P.n) {
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
      // the row's own streams first, so their latency overlaps the gathers
      dfp xv[DF_NP], zv[DF_NP], yi[DF_NP];
#pragma unroll
      for (int u = 0; u < DF_NP; ++u) {
        xv[u] = zv[u] = yi[u] = zero;
        if (P.X) xv[u] = ldps(P.X + off(orow, P.ldx) + cl[u]);
        if (P.Z) zv[u] = ldps(P.Z + off(orow, P.ldz) + cl[u]);
        if (need_yi) yi[u] = ldp(P.Yin + off(orow, P.ldy) + cl[u]);
      }
      float2 S[DF_NP], E[DF_NP];
#pragma unroll
      for (int u = 0; u < DF_NP; ++u) S[u] = E[u] = make_float2(0.f, 0.f);
      for (int base = beg; base < end; base += 32) {
        int jc = 0;
        float ah = 0.f, al = 0.f;
        if constexpr (SHORT) {
          jc = s_jc;
          ah = s_ah;
          al = s_al;
        } else {
          const int e = base + lane;
          if (e < end) {
            const int64_t idx = SELL ? sbase + static_cast<int64_t>(e) * P.sellC : static_cast<int64_t>(e);
            jc = __ldg(P.col + idx);
            const float2 v = __ldg(reinterpret_cast<const float2*>(P.val) + idx);
            ah = v.x;
            al = v.y;
          }
        }
        const int cnt = __shfl_sync(0xffffffffu, min(32, end - base), 0);  // warp-uniform
        for (int t0 = 0; t0 < cnt; t0 += DF_BATCH) {
          int jj[DF_BATCH];
#pragma unroll
          for (int t = 0; t < DF_BATCH; ++t) jj[t] = __shfl_sync(0xffffffffu, jc, t0 + t < 32 ? t0 + t : 31);
          dfp y[DF_BATCH][DF_NP];
#pragma unroll
          for (int t = 0; t < DF_BATCH; ++t)
            if (t0 + t < cnt) {
              const df2* yr = P.Yin + off(jj[t], P.ldy);
#pragma unroll
              for (int u = 0; u < DF_NP; ++u) y[t][u] = ldp(yr + cl[u]);
            }
          // the multipliers are fetched only as each product is formed (not with the indices,
          // before the loads), which keeps the batch's live registers to its loads
#pragma unroll
          for (int t = 0; t < DF_BATCH; ++t) {
            const int src = t0 + t < 32 ? t0 + t : 31;
            const float h = __shfl_sync(0xffffffffu, ah, src);
            const float l = __shfl_sync(0xffffffffu, al, src);
            if (t0 + t < cnt) {
              const dfp a{make_float2(h, h), make_float2(l, l)};
              const dfp na{make_float2(-h, -h), make_float2(-l, -l)};
#pragma unroll
              for (int u = 0; u < DF_NP; ++u) dot2p(S[u], E[u], a, na, y[t][u]);
            }
          }
        }
      }
      if (!act[0]) continue;
#pragma unroll
      for (int u = 0; u < DF_NP; ++u) {
        const dfp acc = fast_two_sum2(S[u], E[u]);
        float2 So = make_float2(0.f, 0.f), Eo = make_float2(0.f, 0.f);
        dot2p(So, Eo, kmul[0][u], neg(kmul[0][u]), acc);
        if (has_beta) dot2p(So, Eo, kmul[1][u], neg(kmul[1][u]), yi[u]);
        if (P.X) dot2p(So, Eo, kmul[2][u], neg(kmul[2][u]), xv[u]);
        if (P.Z) dot2p(So, Eo, kmul[3][u], neg(kmul[3][u]), zv[u]);
        const dfp o = fast_two_sum2(So, Eo);
        if (P.out && act[u])
          __stcs(reinterpret_cast<float4*>(P.out + off(orow, P.ldo) + cp[u]), pack4(o));
        if constexpr (RED) {
          const double o0 = static_cast<double>(o.hi.x) + static_cast<double>(o.lo.x);
          const double o1 = static_cast<double>(o.hi.y) + static_cast<double>(o.lo.y);
          if (P.dot_with_yin) {
            if (act[u]) red[u][0] += o0 * (static_cast<double>(yi[u].hi.x) + static_cast<double>(yi[u].lo.x));
            if (act1[u]) red[u][1] += o1 * (static_cast<double>(yi[u].hi.y) + static_cast<double>(yi[u].lo.y));
          } else {
            if (act[u]) red[u][0] += o0 * o0;
            if (act1[u]) red[u][1] += o1 * o1;
          }
        }
      }
    }
  }
  if constexpr (RED) {
#pragma unroll
    for (int u = 0; u < DF_NP; ++u) {
      if (act[u]) s_red[static_cast<size_t>(warp) * ncols + cp[u]] = red[u][0];
      if (act1[u]) s_red[static_cast<size_t>(warp) * ncols + cp[u] + 1] = red[u][1];
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < ncols; cc += blockDim.x) {
      double sum = 0.0;
      for (int w = 0; w < DF_WARPS; ++w) sum += s_red[static_cast<size_t>(w) * ncols + cc];
      P.red_part[static_cast<size_t>(blockIdx.x) * ncols + cc] = sum;
    }
  }
}

__global__ void reduce_cols_kernel(const double* __restrict__ part, int nb, int ncols, double* __restrict__ out) {
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

// one thread per (row, column pair): FP64 -> paired planar double-float
__global__ void to_df_kernel(int64_t n, const double* __restrict__ src, int64_t lds, int ncols, df2* __restrict__ dst,
                             int64_t ldd) {
  const int npair = (ncols + 1) / 2;
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * npair) return;
  const int64_t r = t / npair;
  const int c = 2 * static_cast<int>(t % npair);
  const df2 a = df_from(src[r * lds + c]);
  const df2 b = df_from(c + 1 < ncols ? src[r * lds + c + 1] : 0.0);
  *reinterpret_cast<float4*>(dst + r * ldd + c) = make_float4(a.hi, b.hi, a.lo, b.lo);
}

__global__ void from_df_kernel(int64_t n, const df2* __restrict__ src, int64_t lds, int ncols, double* __restrict__ dst,
                               int64_t ldd) {
  const int npair = (ncols + 1) / 2;
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * npair) return;
  const int64_t r = t / npair;
  const int c = 2 * static_cast<int>(t % npair);
  const float4 v = *reinterpret_cast<const float4*>(src + r * lds + c);
  dst[r * ldd + c] = static_cast<double>(v.x) + static_cast<double>(v.z);
  if (c + 1 < ncols) dst[r * ldd + c + 1] = static_cast<double>(v.y) + static_cast<double>(v.w);
}

__global__ void val_df_kernel(int64_t nnz, const double* __restrict__ v, df2* __restrict__ out) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < nnz) out[t] = df_from(v[t]);
}

inline int blocks_of(int64_t count, int threads) {
  return static_cast<int>(std::max<int64_t>(1, (count + threads - 1) / threads));
}

}  // namespace

arb_status ensure_valdf(arb_ctx ctx, arb_mat mat) {
  std::lock_guard<std::mutex> lock(mat->mu);
  if (mat->valdf) return ARB_OK;
  df2* v = nullptr;
  ARB_CUDA(ctx, cudaMalloc(&v, std::max<int64_t>(mat->nnz, 1) * sizeof(df2)));
  if (mat->nnz > 0) {
    val_df_kernel<<<blocks_of(mat->nnz, 256), 256, 0, ctx->stream>>>(mat->nnz, mat->val, v);
    ARB_LAUNCHED(ctx);
  }
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  mat->valdf = v;
  return ARB_OK;
}

arb_status to_df(arb_ctx ctx, int64_t n, const double* src, int64_t lds, int32_t ncols, df2* dst, int64_t ldd) {
  if (n <= 0 || ncols <= 0) return ARB_OK;
  if (ldd % 2) return set_error(ctx, ARB_INVALID_ARG, "to_df: leading dimension must be even");
  to_df_kernel<<<blocks_of(n * ((ncols + 1) / 2), 256), 256, 0, ctx->stream>>>(n, src, lds, ncols, dst, ldd);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

arb_status from_df(arb_ctx ctx, int64_t n, const df2* src, int64_t lds, int32_t ncols, double* dst, int64_t ldd) {
  if (n <= 0 || ncols <= 0) return ARB_OK;
  if (lds % 2) return set_error(ctx, ARB_INVALID_ARG, "from_df: leading dimension must be even");
  from_df_kernel<<<blocks_of(n * ((ncols + 1) / 2), 256), 256, 0, ctx->stream>>>(n, src, lds, ncols, dst, ldd);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

template <>
arb_status spmm_fused<df2>(arb_ctx ctx, const SpmmArgs<df2>& a) {
  const arb_mat_s* A = a.A;
  if (a.ncols <= 0 || A->n <= 0) return ARB_OK;
  const bool sell = A->sell_C > 0;
  if (!(sell ? A->sell_valdf : A->valdf))
    return set_error(ctx, ARB_INVALID_ARG, "spmm(df): matrix has no double-float values");
  const bool even = (a.ldy % 2 == 0) && (!a.X || a.ldx % 2 == 0) && (!a.Z || a.ldz % 2 == 0) &&
                    (!a.out || a.ldo % 2 == 0);
  if (!even) return set_error(ctx, ARB_INVALID_ARG, "spmm(df): leading dimensions must be even");
  DfParams P;
  P.n = A->n;
  P.rowptr = A->rowptr;
  P.col = sell ? A->sell_col : A->col;
  P.val = sell ? A->sell_valdf : A->valdf;
  P.perm = A->sell_perm;
  P.slen = A->sell_len;
  P.scptr = A->sell_cptr;
  P.sellC = A->sell_C;
  P.ncols = a.ncols;
  P.Yin = a.Yin;
  P.ldy = a.ldy;
  P.alpha = a.alpha;
  P.beta = a.beta;
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
  const bool want_red = a.colred != nullptr;
  const size_t smem = want_red ? static_cast<size_t>(DF_WARPS) * a.ncols * sizeof(double) : 0;
  if (smem > 200 * 1024) return set_error(ctx, ARB_INVALID_ARG, "spmm(df): too many columns for reduction");
  int64_t ld_max = a.ldy;
  if (a.X) ld_max = std::max(ld_max, a.ldx);
  if (a.Z) ld_max = std::max(ld_max, a.ldz);
  if (a.out) ld_max = std::max(ld_max, a.ldo);
  const bool short_rows = A->max_row_nnz >= 0 && A->max_row_nnz <= 32 && A->n * ld_max < (int64_t(1) << 31);
  const int mode = sell ? 2 : (short_rows ? 1 : 0);
  void (*kern)(DfParams) = mode == 2   ? (want_red ? spmm_df_kernel<true, 2> : spmm_df_kernel<false, 2>)
                           : mode == 1 ? (want_red ? spmm_df_kernel<true, 1> : spmm_df_kernel<false, 1>)
                                       : (want_red ? spmm_df_kernel<true, 0> : spmm_df_kernel<false, 0>);
  ARB_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  int per_sm = 0;
  ARB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DF_THREADS, smem));
  const int nch = (a.ncols + DF_CH - 1) / DF_CH;
  const int64_t want = (P.n * nch + DF_WARPS - 1) / DF_WARPS;
  int grid = static_cast<int>(std::min<int64_t>(want, static_cast<int64_t>(ctx->num_sms) * std::max(per_sm, 1)));
  grid = std::max(grid, (nch + DF_WARPS - 1) / DF_WARPS);
  if (want_red) ARB_TRY(ws<double>(ctx, WS_SS_PART, static_cast<size_t>(grid) * a.ncols, &P.red_part));
  kern<<<grid, DF_THREADS, smem, ctx->stream>>>(P);
  ARB_LAUNCHED(ctx);
  if (want_red) {
    reduce_cols_kernel<<<a.ncols, 256, 0, ctx->stream>>>(P.red_part, grid, a.ncols, a.colred);
    ARB_LAUNCHED(ctx);
  }
  return ARB_OK;
}

}  // namespace arb
