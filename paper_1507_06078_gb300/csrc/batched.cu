// Batched filter: the Chebyshev-interpolant filter (Algorithm 7, evaluated by Clenshaw's
// recurrence) applied to many independent instances - different matrices, block widths,
// degrees and precisions - in ONE persistent cooperative launch.
//
// Every pass t of the recurrence is a set of work items: (instance, row, column chunk)
// for each instance whose degree exceeds t.  The items of pass t are numbered by
// per-pass prefix sums over the instances; warps take items in grid-stride order, find
// the instance by binary search, and run the same fused gather + Clenshaw epilogue as
// the single-instance kernel.  A grid-wide barrier separates passes (pass t+1 gathers
// rows that pass t wrote).  Each instance's multipliers are tabulated per pass in its
// own element type, and its buffer rotation (b_j over b_{j+2}) is fixed in a pass table,
// so the kernel reads plain pointers.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "arb_internal.h"

namespace cg = cooperative_groups;

namespace arb {
namespace {

constexpr int BT_THREADS = 256;
constexpr int BT_WARPS = BT_THREADS / 32;

struct BJob {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  int32_t ncols, nch, vec, fp32;
};

struct BPass {
  const void* Yin;
  const void* X;
  const void* Z;
  void* out;
  const void* sy;  // per-column multipliers in the job's element type
  const void* sx;
  const void* sz;
  int64_t ldy, ldx, ldz, ldo;
  double alpha, beta;
};

template <typename T, int VEC>
__device__ __forceinline__ void vload(const T* p, T (&r)[VEC]) {
#pragma unroll
  for (int u = 0; u < VEC; ++u) r[u] = p[u];
}

template <>
__device__ __forceinline__ void vload<float, 4>(const float* p, float (&r)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  r[0] = t.x;
  r[1] = t.y;
  r[2] = t.z;
  r[3] = t.w;
}

template <>
__device__ __forceinline__ void vload<double, 2>(const double* p, double (&r)[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  r[0] = t.x;
  r[1] = t.y;
}

template <typename T, int VEC>
__device__ __forceinline__ void vstore(T* p, const T (&r)[VEC]) {
#pragma unroll
  for (int u = 0; u < VEC; ++u) p[u] = r[u];
}

template <>
__device__ __forceinline__ void vstore<float, 4>(float* p, const float (&r)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
}

template <>
__device__ __forceinline__ void vstore<double, 2>(double* p, const double (&r)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
}

// out[row, chunk] = sy*(alpha*(A Yin)[row] + beta*Yin[row]) + sx*X[row] + sz*Z[row]
template <typename T, int VEC>
__device__ void batched_item(const BJob& J, const BPass& P, int64_t row, int chunk, int lane) {
  const int c = chunk * 32 * VEC + lane * VEC;
  const bool act = c < J.ncols;
  const T* Yin = static_cast<const T*>(P.Yin);
  const T* X = static_cast<const T*>(P.X);
  const T* Z = static_cast<const T*>(P.Z);
  const T* val = static_cast<const T*>(J.val);
  T xv[VEC], zv[VEC];
  if (X && act) vload<T, VEC>(X + row * P.ldx + c, xv);
  if (Z && act) vload<T, VEC>(Z + row * P.ldz + c, zv);
  T acc[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) acc[u] = T(0);
  const int beg = J.rowptr[row], end = J.rowptr[row + 1];
  for (int base = beg; base < end; base += 32) {
    const int e = base + lane;
    int jc = 0;
    T av = T(0);
    if (e < end) {
      jc = J.col[e];
      av = val[e];
    }
    const int cnt = min(32, end - base);
    for (int t0 = 0; t0 < cnt; t0 += 4) {
      int jj[4];
      T vv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        jj[t] = __shfl_sync(0xffffffffu, jc, t0 + t < 32 ? t0 + t : 31);
        vv[t] = __shfl_sync(0xffffffffu, av, t0 + t < 32 ? t0 + t : 31);
      }
      T y[4][VEC];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (act && t0 + t < cnt) vload<T, VEC>(Yin + static_cast<int64_t>(jj[t]) * P.ldy + c, y[t]);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (act && t0 + t < cnt)
#pragma unroll
          for (int u = 0; u < VEC; ++u) acc[u] = fma(vv[t], y[t][u], acc[u]);
    }
  }
  if (!act) return;
  const T alpha = static_cast<T>(P.alpha), beta = static_cast<T>(P.beta);
  const T* sy = static_cast<const T*>(P.sy);
  const T* sx = static_cast<const T*>(P.sx);
  const T* sz = static_cast<const T*>(P.sz);
  T yi[VEC], o[VEC];
  if (beta != T(0)) {
    vload<T, VEC>(Yin + row * P.ldy + c, yi);
  } else {
#pragma unroll
    for (int u = 0; u < VEC; ++u) yi[u] = T(0);
  }
#pragma unroll
  for (int u = 0; u < VEC; ++u) {
    o[u] = sy[c + u] * fma(alpha, acc[u], beta * yi[u]);
    if (X) o[u] = fma(sx[c + u], xv[u], o[u]);
    if (Z) o[u] = fma(sz[c + u], zv[u], o[u]);
  }
  vstore<T, VEC>(static_cast<T*>(P.out) + row * P.ldo + c, o);
}

__global__ void __launch_bounds__(BT_THREADS) batched_filter_kernel(const BJob* __restrict__ jobs,
                                                                     const BPass* __restrict__ passes,
                                                                     const int64_t* __restrict__ offsets, int njobs,
                                                                     int dmax) {
  cg::grid_group g = cg::this_grid();
  const int lane = threadIdx.x & 31;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * BT_WARPS + (threadIdx.x >> 5);
  const int64_t nw = static_cast<int64_t>(gridDim.x) * BT_WARPS;
  for (int t = 0; t < dmax; ++t) {
    const int64_t* off = offsets + static_cast<int64_t>(t) * (njobs + 1);
    const int64_t total = off[njobs];
    for (int64_t item = gw; item < total; item += nw) {
      int lo = 0, hi = njobs - 1;  // last job with off[j] <= item
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (off[mid] <= item) lo = mid;
        else hi = mid - 1;
      }
      const BJob& J = jobs[lo];
      const BPass& P = passes[static_cast<int64_t>(lo) * dmax + t];
      const int64_t local = item - off[lo];
      const int64_t row = local / J.nch;
      const int chunk = static_cast<int>(local % J.nch);
      if (J.fp32) {
        if (J.vec == 4) batched_item<float, 4>(J, P, row, chunk, lane);
        else batched_item<float, 1>(J, P, row, chunk, lane);
      } else {
        if (J.vec == 2) batched_item<double, 2>(J, P, row, chunk, lane);
        else batched_item<double, 1>(J, P, row, chunk, lane);
      }
    }
    g.sync();
  }
}

// table[(3 t + {0,1,2}) * ncols + c] = {sy, sx, sz} of pass t, in the job's element type
template <typename T>
__global__ void batched_table_kernel(int d, CoefTable cc, const double* __restrict__ xs, int ncols, T* table) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<int64_t>(d) * ncols) return;
  const int t = static_cast<int>(idx / ncols), c = static_cast<int>(idx % ncols);
  const double s = xs ? xs[c] : 1.0;
  const int j = d - 1 - t;
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
  table[(3 * static_cast<int64_t>(t) + 0) * ncols + c] = static_cast<T>(sy);
  table[(3 * static_cast<int64_t>(t) + 1) * ncols + c] = static_cast<T>(sx);
  table[(3 * static_cast<int64_t>(t) + 2) * ncols + c] = static_cast<T>(sz);
}

// per-job column sums of squares: block b of job j sums rows [b*R, (b+1)*R)
template <typename T>
__global__ void colss_kernel(int64_t n, const T* __restrict__ Y, int64_t ldy, int ncols, int64_t rows,
                             double* __restrict__ part) {
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rows, r1 = min(n, r0 + rows);
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      const double v = static_cast<double>(Y[r * ldy + c]);
      s = fma(v, v, s);
    }
    part[static_cast<size_t>(blockIdx.x) * ncols + c] = s;
  }
}

__global__ void colss_reduce_kernel(const double* __restrict__ part, int nb, int ncols, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[static_cast<size_t>(b) * ncols + c];
  out[c] = s;
}

inline bool al(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

// The batched filter in two parts: prepare() validates the jobs, sizes the workspaces and
// uploads the descriptors (it synchronises the stream); launch() issues the per-job
// coefficient tables, the one persistent cooperative launch and the per-job column sums -
// kernels only, with no allocation and no synchronisation, so that a caller may capture it
// into a CUDA graph and replay it while the descriptors (re-uploaded by prepare) keep
// their device addresses.
arb_status filter_batched_prepare(arb_ctx ctx, int32_t njobs, const arb_filter_job* jobs, BatchPlan* out) {
  out->njobs = njobs;
  out->jobs.assign(jobs, jobs + njobs);
  out->tables.clear();
  out->coef.clear();
  if (njobs <= 0) return ARB_OK;
  int dmax = 0;
  size_t work_bytes = 0, table_bytes = 0;
  std::vector<int64_t> ldw(njobs);
  for (int j = 0; j < njobs; ++j) {
    const arb_filter_job& J = jobs[j];
    if (!J.mat || !J.coef || !J.X || !J.Y || J.ncols <= 0 || J.ldx < J.ncols || J.ldy < J.ncols || !(J.b > J.a) ||
        J.degree < 1 || J.degree > 60 || J.mat->device != ctx->device)
      return set_error(ctx, ARB_INVALID_ARG, "filter_batched: bad job");
    dmax = std::max(dmax, J.degree);
    const size_t es = J.fp32 ? 4 : 8;
    ldw[j] = (J.ncols + 3) / 4 * 4;
    work_bytes += 2 * static_cast<size_t>(J.mat->n) * ldw[j] * es + 256;
    table_bytes += 3 * static_cast<size_t>(J.degree) * J.ncols * es + 256;
    if (J.fp32) ARB_TRY(ensure_val32(ctx, J.mat));
  }
  char *work, *tables;
  ARB_TRY(ws<char>(ctx, WS_BATCH_WORK, work_bytes, &work));
  ARB_TRY(ws<char>(ctx, WS_BATCH_TABLE, table_bytes, &tables));
  std::vector<BJob> hj(njobs);
  std::vector<BPass> hp(static_cast<size_t>(njobs) * dmax);
  std::vector<int64_t> hoff(static_cast<size_t>(dmax) * (njobs + 1), 0);
  size_t wo = 0, to = 0;
  for (int j = 0; j < njobs; ++j) {
    const arb_filter_job& J = jobs[j];
    const bool f = J.fp32 != 0;
    const size_t es = f ? 4 : 8;
    const int64_t n = J.mat->n;
    char* W1 = work + wo;
    wo += (static_cast<size_t>(n) * ldw[j] * es + 255) / 256 * 256;
    char* W2 = work + wo;
    wo += (static_cast<size_t>(n) * ldw[j] * es + 255) / 256 * 256;
    char* tab = tables + to;
    to += (3 * static_cast<size_t>(J.degree) * J.ncols * es + 255) / 256 * 256;
    const FilterPlan plan = make_filter_plan(J.op_scale, J.op_shift, J.a, J.b, J.degree, J.coef);
    CoefTable cc;
    for (int i = 0; i < 64; ++i) cc.c[i] = (i <= J.degree) ? plan.coef[i] : 0.0;
    const int64_t cnt = static_cast<int64_t>(J.degree) * J.ncols;
    const int tb = static_cast<int>((cnt + 255) / 256);
    out->tables.push_back(BatchPlan::Table{f, J.degree, J.ncols, tb, cc, J.xscale, tab});
    // vector width: 16-byte lanes when the columns, leading dimensions and bases allow
    int vec = 1;
    const int want = f ? 4 : 2;
    if (J.ncols % want == 0 && J.ldx % want == 0 && J.ldy % want == 0 && ldw[j] % want == 0 && al(J.X, 16) &&
        al(J.Y, 16) && J.ncols > 32 * (want / 2) && (J.mat->tune_vec == 0 || J.mat->tune_vec >= want))
      vec = want;
    const int nch = (J.ncols + 32 * vec - 1) / (32 * vec);
    hj[j] = BJob{n, J.mat->rowptr, J.mat->col, f ? static_cast<const void*>(J.mat->val32) : J.mat->val, J.ncols, nch,
                 vec, f ? 1 : 0};
    // buffer rotation of the recurrence (as in the single-instance filter)
    auto tabp = [&](int t, int which) -> const void* { return tab + ((3 * static_cast<size_t>(t) + which) * J.ncols) * es; };
    const int d = J.degree;
    const void* cur = nullptr;
    const void* prev = nullptr;
    for (int t = 0; t < d; ++t) {
      BPass P{};
      P.alpha = plan.alpha;
      P.beta = plan.beta;
      P.sy = tabp(t, 0);
      P.sx = tabp(t, 1);
      P.sz = tabp(t, 2);
      const int jdx = d - 1 - t;
      const bool last = (t == d - 1);
      if (t == 0) {
        P.Yin = J.X;
        P.ldy = J.ldx;
      } else {
        P.Yin = cur;
        P.ldy = ldw[j];
      }
      if (plan.coef[d == 1 ? 0 : jdx] != 0.0) {
        P.X = J.X;
        P.ldx = J.ldx;
      }
      if (t >= 1) {
        if (prev) {
          P.Z = prev;
          P.ldz = ldw[j];
        } else if (plan.coef[d] != 0.0) {
          P.Z = J.X;
          P.ldz = J.ldx;
        }
      }
      if (last) {
        P.out = J.Y;
        P.ldo = J.ldy;
      } else {
        P.out = (t == 0) ? static_cast<void*>(W1) : (prev ? const_cast<void*>(prev) : static_cast<void*>(W2));
        P.ldo = ldw[j];
      }
      hp[static_cast<size_t>(j) * dmax + t] = P;
      prev = (t == 0) ? nullptr : cur;
      cur = P.out;
    }
    for (int t = 0; t < dmax; ++t) {
      int64_t* off = hoff.data() + static_cast<size_t>(t) * (njobs + 1);
      off[j + 1] = (t < d) ? static_cast<int64_t>(n) * nch : 0;
    }
  }
  for (int t = 0; t < dmax; ++t) {
    int64_t* off = hoff.data() + static_cast<size_t>(t) * (njobs + 1);
    for (int j = 0; j < njobs; ++j) off[j + 1] += off[j];
  }
  // descriptors to the device
  const size_t bj = hj.size() * sizeof(BJob), bp = hp.size() * sizeof(BPass), bo = hoff.size() * sizeof(int64_t);
  char* desc;
  ARB_TRY(ws<char>(ctx, WS_BATCH_DESC, bj + bp + bo + 512, &desc));
  void* st;
  ARB_TRY(host_stage(ctx, bj + bp + bo + 512, &st));
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // staging area free
  char* sp = static_cast<char*>(st);
  memcpy(sp, hj.data(), bj);
  memcpy(sp + bj, hp.data(), bp);
  memcpy(sp + bj + bp, hoff.data(), bo);
  ARB_CUDA(ctx, cudaMemcpyAsync(desc, sp, bj + bp + bo, cudaMemcpyHostToDevice, ctx->stream));
  const BJob* dj = reinterpret_cast<const BJob*>(desc);
  const BPass* dp = reinterpret_cast<const BPass*>(desc + bj);
  const int64_t* doff = reinterpret_cast<const int64_t*>(desc + bj + bp);
  out->dmax = dmax;
  int per_sm = 0;
  ARB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_filter_kernel, BT_THREADS, 0));
  out->coop_grid = std::max(1, std::max(1, per_sm) * ctx->num_sms / std::max(1, ctx->coop_share));
  out->dj = dj;
  out->dp = dp;
  out->doff = doff;
  // column-sum partials: the largest any job needs
  size_t part_max = 0;
  for (int j = 0; j < njobs; ++j) {
    if (!jobs[j].colss) continue;
    const int64_t n = jobs[j].mat->n;
    const int64_t rows = std::max<int64_t>(256, (n + 4 * ctx->num_sms - 1) / (4 * ctx->num_sms));
    part_max = std::max(part_max, static_cast<size_t>((n + rows - 1) / rows) * jobs[j].ncols);
  }
  if (part_max) ARB_TRY(ws<double>(ctx, WS_SS_PART, part_max, &out->part));
  return ARB_OK;
}

arb_status filter_batched_launch(arb_ctx ctx, const BatchPlan& plan) {
  const int32_t njobs = plan.njobs;
  if (njobs <= 0) return ARB_OK;
  for (const auto& tb : plan.tables) {
    if (tb.fp32)
      batched_table_kernel<float><<<tb.blocks, 256, 0, ctx->stream>>>(tb.d, tb.cc, tb.xscale, tb.ncols,
                                                                      static_cast<float*>(tb.table));
    else
      batched_table_kernel<double><<<tb.blocks, 256, 0, ctx->stream>>>(tb.d, tb.cc, tb.xscale, tb.ncols,
                                                                       static_cast<double*>(tb.table));
    ARB_LAUNCHED(ctx);
  }
  const BJob* dj = static_cast<const BJob*>(plan.dj);
  const BPass* dp = static_cast<const BPass*>(plan.dp);
  const int64_t* doff = plan.doff;
  int dmax = plan.dmax;
  const arb_filter_job* jobs = plan.jobs.data();
  const int grid = plan.coop_grid;
  int nj = njobs;
  void* args[] = {&dj, &dp, &doff, &nj, &dmax};
  ARB_CUDA(ctx, cudaLaunchCooperativeKernel(reinterpret_cast<void*>(batched_filter_kernel), dim3(grid),
                                            dim3(BT_THREADS), args, 0, ctx->stream));
  ARB_LAUNCHED(ctx);
  // column sums of squares of each result (the MPM normalisation)
  for (int j = 0; j < njobs; ++j) {
    const arb_filter_job& J = jobs[j];
    if (!J.colss) continue;
    const int64_t n = J.mat->n;
    const int64_t rows = std::max<int64_t>(256, (n + 4 * ctx->num_sms - 1) / (4 * ctx->num_sms));
    const int nb = static_cast<int>((n + rows - 1) / rows);
    double* part = plan.part;
    if (J.fp32)
      colss_kernel<float><<<nb, 128, 0, ctx->stream>>>(n, static_cast<const float*>(J.Y), J.ldy, J.ncols, rows, part);
    else
      colss_kernel<double><<<nb, 128, 0, ctx->stream>>>(n, static_cast<const double*>(J.Y), J.ldy, J.ncols, rows, part);
    ARB_LAUNCHED(ctx);
    colss_reduce_kernel<<<(J.ncols + 127) / 128, 128, 0, ctx->stream>>>(part, nb, J.ncols, J.colss);
    ARB_LAUNCHED(ctx);
  }
  return ARB_OK;
}


arb_status filter_batched(arb_ctx ctx, int32_t njobs, const arb_filter_job* jobs) {
  BatchPlan plan;
  ARB_TRY(filter_batched_prepare(ctx, njobs, jobs, &plan));
  return filter_batched_launch(ctx, plan);
}

}  // namespace arb

extern "C" arb_status arb_filter_batched(arb_ctx ctx, int32_t njobs, const arb_filter_job* jobs) {
  if (!ctx || njobs < 0 || (njobs > 0 && !jobs)) return ARB_INVALID_ARG;
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  return arb::filter_batched(ctx, njobs, jobs);
}
