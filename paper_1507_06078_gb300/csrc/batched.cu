// Batched filter: the Chebyshev-interpolant filter (Algorithm 7, evaluated by Clenshaw's
// recurrence) applied to many independent instances - different matrices, block widths,
// degrees and precisions - in persistent cooperative launches, one per element type and
// vector width present in the batch.
//
// Every pass t of the recurrence is a set of tiles: (instance, run of rows) for each
// instance whose degree exceeds t.  The tiles of pass t are numbered by per-pass prefix
// sums over the instances; warps take tiles in grid-stride order and find the instance by
// one binary search per tile.  Inside a tile a warp is split into groups of G lanes (G the
// power of two that covers the block's width in 16-byte vectors, at most 32), one row per
// group, so a 12-column block keeps 8 rows in flight per warp instead of idling 20 lanes.
// A group walks its rows software-pipelined: the nonzeros of the next row and the bounds
// of the one after are fetched while the current row gathers.  Each lane sums its
// columns' products over the row's nonzeros in CSR order and applies the same Clenshaw
// epilogue as the single-instance kernel.  The per-column multipliers of every pass follow
// from the instance's coefficients and column scale in FP64; a prologue of the launch
// tabulates them in the instance's element type, so the row loop runs no FP64 instruction
// for FP32 instances (FP64 issues at a small fraction of the FP32 rate on this GPU).  A
// grid-wide barrier separates passes (pass t+1 gathers rows that pass t wrote).  In an
// instance's last pass every tile also leaves the column sums of squares of its rows (the
// MPM normalisation of Algorithm 7's output; FP32 instances sum in double-float: FP32
// pairs with error-free product and sum transforms); after the last barrier one warp per
// (instance, column) adds the tiles' partial sums in tile order, so the result does not
// depend on the grid.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "arb_internal.h"

namespace cg = cooperative_groups;

namespace arb {
namespace {

constexpr int BT_THREADS = 256;
constexpr int BT_WARPS = BT_THREADS / 32;
// nonzeros of the next row fetched ahead (rows up to this length take one round trip)
#ifndef BT_PF
#define BT_PF 4
#endif
// CTAs per SM the register budget must allow (2: 128 registers a thread)
#ifndef ARB_BATCH_MIN_BLOCKS
#define ARB_BATCH_MIN_BLOCKS 2
#endif

struct BJob {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  const double* coef;  // c_0..c_d of the instance's interpolant in terms of S (device)
  const double* xs;    // per-column scale of X, or NULL
  double* colss;       // column sums of squares of the result, or NULL
  double* part;        // [tiles][ncols] partial sums of the last pass (colss only)
  void* tab;           // [degree][3][ldt] multipliers (sy, sx, sz) of every pass, element type
  int64_t tiles;       // tiles of one pass
  int32_t tile_rows;
  int32_t ncols, nch, vec, fp32;
  int32_t glog;        // lanes per row = 1 << glog
  int32_t degree;
  int32_t ldt;         // ncols rounded up to 4
};

struct BPass {
  const void* Yin;
  const void* X;
  const void* Z;
  void* out;
  int64_t ldy, ldx, ldz, ldo;
  double alpha, beta;
};

// element offset r * ld of row r in a block of leading dimension ld (both below 2^31)
__device__ __forceinline__ int64_t roff(int64_t r, int64_t ld) {
  return static_cast<int64_t>(static_cast<int32_t>(r)) * static_cast<int32_t>(ld);
}

// VEC consecutive elements of a row.  For VEC > 1 the whole vector is read even where the
// row's last vector is ragged (valid < VEC), except in a block's last row (tail = true),
// which may end at the block's last column: the vector classes have leading dimensions
// that are multiples of VEC, so such a read stays inside the row's leading dimension, and
// the extra lanes' results are never stored.  For VEC == 1, valid <= 0 reads nothing.
template <typename T, int VEC>
__device__ __forceinline__ void vload(const T* p, int valid, T (&r)[VEC], bool tail = false) {
  if (valid >= VEC || (VEC > 1 && !tail)) {
    if constexpr (VEC == 4 && sizeof(T) == 4) {
      const float4 t = *reinterpret_cast<const float4*>(p);
      r[0] = t.x;
      r[1] = t.y;
      r[2] = t.z;
      r[3] = t.w;
      return;
    } else if constexpr (VEC == 2 && sizeof(T) == 8) {
      const double2 t = *reinterpret_cast<const double2*>(p);
      r[0] = t.x;
      r[1] = t.y;
      return;
    }
  }
#pragma unroll
  for (int u = 0; u < VEC; ++u) r[u] = u < valid ? p[u] : T(0);
}

template <typename T, int VEC>
__device__ __forceinline__ void vstore(T* p, int valid, const T (&r)[VEC]) {
  if (valid >= VEC) {
    if constexpr (VEC == 4 && sizeof(T) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
      return;
    } else if constexpr (VEC == 2 && sizeof(T) == 8) {
      *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
      return;
    }
  }
#pragma unroll
  for (int u = 0; u < VEC; ++u)
    if (u < valid) p[u] = r[u];
}

// multipliers of column c in pass t (Clenshaw's b_j = 2 S b_{j+1} - b_{j+2} + c_j X with
// the first and last passes folded in), in FP64 as the single-instance filter's tables
__device__ __forceinline__ void pass_multipliers(const BJob& J, int t, int c, double& sy, double& sx, double& sz) {
  const double s = J.xs ? J.xs[c] : 1.0;
  const int d = J.degree;
  const int j = d - 1 - t;
  if (d == 1) {
    sy = J.coef[1] * s;
    sx = J.coef[0] * s;
    sz = 0.0;
  } else {
    sy = (t == 0) ? 2.0 * J.coef[d] * s : (t == d - 1 ? 1.0 : 2.0);
    sx = J.coef[j] * s;
    sz = (j + 2 == d) ? -J.coef[d] * s : -1.0;
  }
}

// (hi, lo) += o^2 with the rounding errors of the product and of the sum carried in lo
__device__ __forceinline__ void df_add_square(float o, float& hi, float& lo) {
  const float p = o * o;
  const float pe = fmaf(o, o, -p);
  const float s = hi + p;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (p - bp);
  hi = s;
  lo += e + pe;
}

__device__ __forceinline__ void df_add(float& hi, float& lo, float h2, float l2) {
  const float s = hi + h2;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (h2 - bp);
  hi = s;
  lo = lo + l2 + e;
}

// one tile of pass t: out[row, c] = sy*(alpha*(A Yin)[row] + beta*Yin[row]) + sx*X[row] + sz*Z[row]
template <typename T, int VEC>
__device__ void batched_tile(const BJob& J, const BPass& P, int t, int64_t tile, int lane, bool last) {
  const int glog = J.glog;
  const int G = 1 << glog;
  const int R = 32 >> glog;
  const int grp = lane >> glog, gl = lane & (G - 1);
  const int64_t r0 = tile * J.tile_rows;
  const int64_t r1 = min(J.n, r0 + J.tile_rows);
  const bool want_ss = last && J.colss != nullptr;  // warp-uniform
  const T* Yin = static_cast<const T*>(P.Yin);
  const T* X = static_cast<const T*>(P.X);
  const T* Z = static_cast<const T*>(P.Z);
  T* out = static_cast<T*>(P.out);
  const T* val = static_cast<const T*>(J.val);
  const T alpha = static_cast<T>(P.alpha), beta = static_cast<T>(P.beta);
  const int nlast = static_cast<int>(J.n - 1);
  // column sums of squares of the tile's rows: FP64 for FP64 instances, double-float
  // (hi, lo) for FP32 ones
  using Acc = typename std::conditional<sizeof(T) == 4, float, double>::type;
  for (int ch = 0; ch < J.nch; ++ch) {
    const int c = (ch * G + gl) * VEC;
    const int valid = min(VEC, J.ncols - c);  // <= 0: the lane has no column here
    Acc ss[VEC], sl[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) ss[u] = sl[u] = Acc(0);
    const T* tab = static_cast<const T*>(J.tab) + static_cast<int64_t>(t) * 3 * J.ldt + c;
    if (valid > 0) {
      int64_t row = r0 + grp;
      int cb = 0, ce = 0, nb = 0, ne = 0;
      int cj[BT_PF];
      T cv[BT_PF];
      if (row < r1) {
        cb = J.rowptr[row];
        ce = J.rowptr[row + 1];
      }
#pragma unroll
      for (int q = 0; q < BT_PF; ++q) {
        const bool in = cb + q < ce;
        cj[q] = in ? J.col[cb + q] : 0;
        cv[q] = in ? val[cb + q] : T(0);
      }
      if (row + R < r1) {
        nb = J.rowptr[row + R];
        ne = J.rowptr[row + R + 1];
      }
      for (; row < r1; row += R) {
        int pb = 0, pe = 0;
        if (row + 2 * R < r1) {
          pb = J.rowptr[row + 2 * R];
          pe = J.rowptr[row + 2 * R + 1];
        }
        int nj[BT_PF];
        T nv[BT_PF];
#pragma unroll
        for (int q = 0; q < BT_PF; ++q) {
          const bool in = nb + q < ne;
          nj[q] = in ? J.col[nb + q] : 0;
          nv[q] = in ? val[nb + q] : T(0);
        }
        const bool tail = row == nlast;
        T xv[VEC], zv[VEC], yi[VEC];
        if (X) vload<T, VEC>(X + roff(row, P.ldx) + c, valid, xv, tail);
        if (Z) vload<T, VEC>(Z + roff(row, P.ldz) + c, valid, zv, tail);
        if (beta != T(0)) vload<T, VEC>(Yin + roff(row, P.ldy) + c, valid, yi, tail);
        T acc[VEC];
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[u] = T(0);
        {
          T y[BT_PF][VEC];
#pragma unroll
          for (int q = 0; q < BT_PF; ++q)
            if (cb + q < ce) vload<T, VEC>(Yin + roff(cj[q], P.ldy) + c, valid, y[q], cj[q] == nlast);
#pragma unroll
          for (int q = 0; q < BT_PF; ++q)
            if (cb + q < ce)
#pragma unroll
              for (int u = 0; u < VEC; ++u) acc[u] = fma(cv[q], y[q][u], acc[u]);
        }
        for (int e = cb + BT_PF; e < ce; e += 4) {  // rows longer than the prefetched part
          int jj[4];
          T vv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const bool in = e + q < ce;
            jj[q] = in ? J.col[e + q] : 0;
            vv[q] = in ? val[e + q] : T(0);
          }
          T y[4][VEC];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (e + q < ce) vload<T, VEC>(Yin + roff(jj[q], P.ldy) + c, valid, y[q], jj[q] == nlast);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (e + q < ce)
#pragma unroll
              for (int u = 0; u < VEC; ++u) acc[u] = fma(vv[q], y[q][u], acc[u]);
        }
        // the pass's multipliers from the table (cached reads, not held in registers
        // across the gathers)
        T my[VEC], mx[VEC], mz[VEC];
        vload<T, VEC>(tab, valid, my);
        vload<T, VEC>(tab + J.ldt, valid, mx);
        vload<T, VEC>(tab + 2 * J.ldt, valid, mz);
        T o[VEC];
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          o[u] = my[u] * fma(alpha, acc[u], beta != T(0) ? beta * yi[u] : T(0));
          if (X) o[u] = fma(mx[u], xv[u], o[u]);
          if (Z) o[u] = fma(mz[u], zv[u], o[u]);
        }
        vstore<T, VEC>(out + roff(row, P.ldo) + c, valid, o);
        if (want_ss) {
#pragma unroll
          for (int u = 0; u < VEC; ++u) {
            if constexpr (sizeof(T) == 4) df_add_square(o[u], ss[u], sl[u]);
            else ss[u] = fma(o[u], o[u], ss[u]);
          }
        }
        cb = nb;
        ce = ne;
        nb = pb;
        ne = pe;
#pragma unroll
        for (int q = 0; q < BT_PF; ++q) {
          cj[q] = nj[q];
          cv[q] = nv[q];
        }
      }
    }
    if (want_ss) {
      // the R groups' sums of the tile's rows, then one lane per column writes them
#pragma unroll
      for (int u = 0; u < VEC; ++u)
        for (int m = G; m < 32; m <<= 1) {
          const Acc h2 = __shfl_xor_sync(0xffffffffu, ss[u], m);
          if constexpr (sizeof(T) == 4) {
            const Acc l2 = __shfl_xor_sync(0xffffffffu, sl[u], m);
            df_add(ss[u], sl[u], h2, l2);
          } else {
            ss[u] += h2;
          }
        }
      if (grp == 0)
#pragma unroll
        for (int u = 0; u < VEC; ++u)
          if (u < valid) J.part[tile * J.ncols + c + u] = static_cast<double>(ss[u]) + static_cast<double>(sl[u]);
    }
  }
}

// one launch per element type and vector width present in the batch: a kernel that held
// all four tile variants would need the registers of their union and spill.
// offsets: dmax rows of per-pass tile offsets, then one row of table-prologue offsets
// (degree x ncols per job), each of njobs + 1 entries; csoff: column-sum offsets.
template <typename T, int VEC>
__global__ void __launch_bounds__(BT_THREADS, ARB_BATCH_MIN_BLOCKS)
    batched_filter_kernel(const BJob* __restrict__ jobs, const BPass* __restrict__ passes,
                          const int64_t* __restrict__ offsets, int njobs, int dmax,
                          const int64_t* __restrict__ csoff, unsigned long long* __restrict__ tickets) {
  cg::grid_group g = cg::this_grid();
  const int lane = threadIdx.x & 31;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * BT_WARPS + (threadIdx.x >> 5);
  const int64_t nw = static_cast<int64_t>(gridDim.x) * BT_WARPS;
  auto job_of = [&](const int64_t* off, int64_t item) {
    int lo = 0, hi = njobs - 1;  // last job with off[j] <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (off[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  // prologue: every job's multiplier table and the passes' tile tickets, then a barrier
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < dmax; i += blockDim.x) tickets[i] = 0ull;
  {
    const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nt = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t* toff = offsets + static_cast<int64_t>(dmax) * (njobs + 1);
    for (int64_t item = gt; item < toff[njobs]; item += nt) {
      const int j = job_of(toff, item);
      const BJob& J = jobs[j];
      const int64_t local = item - toff[j];
      const int tt = static_cast<int>(local / J.ncols), c = static_cast<int>(local % J.ncols);
      double my, mx, mz;
      pass_multipliers(J, tt, c, my, mx, mz);
      T* tab = static_cast<T*>(J.tab) + static_cast<int64_t>(tt) * 3 * J.ldt + c;
      tab[0] = static_cast<T>(my);
      tab[J.ldt] = static_cast<T>(mx);
      tab[2 * J.ldt] = static_cast<T>(mz);
    }
    g.sync();
  }
  for (int t = 0; t < dmax; ++t) {
    const int64_t* off = offsets + static_cast<int64_t>(t) * (njobs + 1);
    const int64_t total = off[njobs];
    // tiles handed out in order by a ticket counter, so warps that drew short tiles take
    // more and the pass ends within about one tile of its average; the next ticket is
    // drawn before the current tile runs
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(tickets + t, 1ull);
    int64_t item = static_cast<int64_t>(__shfl_sync(0xffffffffu, tk, 0));
    while (item < total) {
      if (lane == 0) tk = atomicAdd(tickets + t, 1ull);
      const int j = job_of(off, item);
      const BJob& J = jobs[j];
      const BPass& P = passes[static_cast<int64_t>(j) * dmax + t];
      batched_tile<T, VEC>(J, P, t, item - off[j], lane, t == J.degree - 1);
      item = static_cast<int64_t>(__shfl_sync(0xffffffffu, tk, 0));
    }
    g.sync();
  }
  // column sums of squares: one warp per (job, column), tiles strided over the lanes and
  // added in a fixed tree
  const int64_t ctotal = csoff[njobs];
  for (int64_t item = gw; item < ctotal; item += nw) {
    const int j = job_of(csoff, item);
    const BJob& J = jobs[j];
    const int c = static_cast<int>(item - csoff[j]);
    double s = 0.0;
    for (int64_t tile = lane; tile < J.tiles; tile += 32) s += J.part[tile * J.ncols + c];
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) J.colss[c] = s;
  }
}

inline bool al(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// kernel of a job class: 0 FP32 x4, 1 FP32 x1, 2 FP64 x2, 3 FP64 x1
const void* class_kernel(int cls) {
  switch (cls) {
    case 0: return reinterpret_cast<const void*>(batched_filter_kernel<float, 4>);
    case 1: return reinterpret_cast<const void*>(batched_filter_kernel<float, 1>);
    case 2: return reinterpret_cast<const void*>(batched_filter_kernel<double, 2>);
    default: return reinterpret_cast<const void*>(batched_filter_kernel<double, 1>);
  }
}

}  // namespace

// The batched filter in two parts: prepare() validates the jobs, sizes the workspaces and
// uploads the descriptors (it synchronises the stream); launch() issues the persistent
// cooperative launches (one per job class present) - kernels only, with no allocation and
// no synchronisation, so that a caller may capture them into a CUDA graph and replay it
// while the descriptors (re-uploaded by prepare) keep their device addresses.
arb_status filter_batched_prepare(arb_ctx ctx, int32_t njobs, const arb_filter_job* jobs, BatchPlan* out) {
  out->njobs = njobs;
  out->jobs.assign(jobs, jobs + njobs);
  for (auto& c : out->cls) c = BatchPlan::Class{};
  if (njobs <= 0) return ARB_OK;
  int dmax = 0;
  size_t work_bytes = 0, ncoef = 0;
  for (int j = 0; j < njobs; ++j) {
    const arb_filter_job& J = jobs[j];
    if (!J.mat || !J.coef || !J.X || !J.Y || J.ncols <= 0 || J.ldx < J.ncols || J.ldy < J.ncols || !(J.b > J.a) ||
        J.degree < 1 || J.degree > 60 || J.mat->device != ctx->device)
      return set_error(ctx, ARB_INVALID_ARG, "filter_batched: bad job");
    dmax = std::max(dmax, J.degree);
    const size_t es = J.fp32 ? 4 : 8;
    const size_t ldw = (J.ncols + 3) / 4 * 4;
    work_bytes += 2 * static_cast<size_t>(J.mat->n) * ldw * es + 512;
    work_bytes += 3 * static_cast<size_t>(J.degree) * ldw * es + 256;  // multiplier table
    ncoef += static_cast<size_t>(J.degree) + 1;
    if (J.fp32) ARB_TRY(ensure_val32(ctx, J.mat));
  }
  char* work;
  ARB_TRY(ws<char>(ctx, WS_BATCH_WORK, work_bytes, &work));
  // class of every job (element type; 16-byte lanes when the leading dimensions and bases
  // allow, a ragged last vector of a row being read and written element by element), and
  // the jobs in class order
  std::vector<int> cls(njobs), order;
  for (int j = 0; j < njobs; ++j) {
    const arb_filter_job& J = jobs[j];
    const int want = J.fp32 ? 4 : 2;
    const int64_t ldw = (J.ncols + 3) / 4 * 4;
    const bool wide = J.ldx % want == 0 && J.ldy % want == 0 && ldw % want == 0 && al(J.X, 16) && al(J.Y, 16);
    cls[j] = (J.fp32 ? 0 : 2) + (wide ? 0 : 1);
  }
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < njobs; ++j)
      if (cls[j] == k) order.push_back(j);
  std::vector<BJob> hj(njobs);
  std::vector<BPass> hp(static_cast<size_t>(njobs) * dmax);
  std::vector<double> hcoef;
  hcoef.reserve(ncoef);
  std::vector<size_t> coef_at(njobs), part_at(njobs);
  size_t wo = 0, part_total = 0;
  for (int o = 0; o < njobs; ++o) {
    const int j = order[o];
    const arb_filter_job& J = jobs[j];
    const bool f = J.fp32 != 0;
    const size_t es = f ? 4 : 8;
    const int64_t n = J.mat->n;
    const int64_t ldw = (J.ncols + 3) / 4 * 4;
    char* W1 = work + wo;
    wo += (static_cast<size_t>(n) * ldw * es + 255) / 256 * 256;
    char* W2 = work + wo;
    wo += (static_cast<size_t>(n) * ldw * es + 255) / 256 * 256;
    char* tab = work + wo;
    wo += (3 * static_cast<size_t>(J.degree) * ldw * es + 255) / 256 * 256;
    const FilterPlan plan = make_filter_plan(J.op_scale, J.op_shift, J.a, J.b, J.degree, J.coef);
    coef_at[o] = hcoef.size();
    for (int i = 0; i <= J.degree; ++i) hcoef.push_back(plan.coef[i]);
    const int vec = (cls[j] & 1) ? 1 : (f ? 4 : 2);
    // lanes per row: the power of two covering the row's vectors, at most a warp
    const int lanes = (J.ncols + vec - 1) / vec;
    int glog = 0;
    while ((1 << glog) < lanes && glog < 5) ++glog;
    const int G = 1 << glog, R = 32 >> glog;
    const int nch = (J.ncols + G * vec - 1) / (G * vec);
    // 8 to 64 row steps per tile: the instance lookup is amortised and a large instance
    // leaves at most ~1024 tiles of partial column sums
    const int64_t iters = std::min<int64_t>(64, std::max<int64_t>(8, (n + R * 1024 - 1) / (R * 1024)));
    const int32_t tile_rows = static_cast<int32_t>(R * iters);
    const int64_t tiles = (n + tile_rows - 1) / tile_rows;
    part_at[o] = part_total;
    if (J.colss) part_total += static_cast<size_t>(tiles) * J.ncols;
    BJob& B = hj[o];
    B.n = n;
    B.rowptr = J.mat->rowptr;
    B.col = J.mat->col;
    B.val = f ? static_cast<const void*>(J.mat->val32) : static_cast<const void*>(J.mat->val);
    B.coef = nullptr;  // device addresses below
    B.xs = J.xscale;
    B.colss = J.colss;
    B.part = nullptr;
    B.tab = tab;
    B.tiles = tiles;
    B.tile_rows = tile_rows;
    B.ncols = J.ncols;
    B.nch = nch;
    B.vec = vec;
    B.fp32 = f ? 1 : 0;
    B.glog = glog;
    B.degree = J.degree;
    B.ldt = static_cast<int32_t>(ldw);
    // buffer rotation of the recurrence (as in the single-instance filter)
    const int d = J.degree;
    const void* cur = nullptr;
    const void* prev = nullptr;
    for (int t = 0; t < d; ++t) {
      BPass P{};
      P.alpha = plan.alpha;
      P.beta = plan.beta;
      const int jdx = d - 1 - t;
      const bool last = (t == d - 1);
      if (t == 0) {
        P.Yin = J.X;
        P.ldy = J.ldx;
      } else {
        P.Yin = cur;
        P.ldy = ldw;
      }
      if (plan.coef[d == 1 ? 0 : jdx] != 0.0) {
        P.X = J.X;
        P.ldx = J.ldx;
      }
      if (t >= 1) {
        if (prev) {
          P.Z = prev;
          P.ldz = ldw;
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
        P.ldo = ldw;
      }
      hp[static_cast<size_t>(o) * dmax + t] = P;
      prev = (t == 0) ? nullptr : cur;
      cur = P.out;
    }
  }
  // per class: pass offsets over its tiles (dmax rows), the table prologue's offsets (one
  // row) and column-sum offsets over its columns
  std::vector<int64_t> hoff, hcs;
  size_t off_at[4] = {0, 0, 0, 0}, cs_at[4] = {0, 0, 0, 0};
  int first = 0;
  for (int k = 0; k < 4; ++k) {
    int count = 0;
    while (first + count < njobs && cls[order[first + count]] == k) ++count;
    out->cls[k].first = first;
    out->cls[k].count = count;
    off_at[k] = hoff.size();
    cs_at[k] = hcs.size();
    if (count > 0) {
      for (int t = 0; t < dmax; ++t) {
        int64_t acc = 0;
        hoff.push_back(0);
        for (int o = first; o < first + count; ++o) {
          acc += (t < hj[o].degree) ? hj[o].tiles : 0;
          hoff.push_back(acc);
        }
      }
      int64_t acc = 0;
      hoff.push_back(0);
      for (int o = first; o < first + count; ++o) {
        acc += static_cast<int64_t>(hj[o].degree) * hj[o].ncols;
        hoff.push_back(acc);
      }
      acc = 0;
      hcs.push_back(0);
      for (int o = first; o < first + count; ++o) {
        acc += jobs[order[o]].colss ? hj[o].ncols : 0;
        hcs.push_back(acc);
      }
    }
    first += count;
  }
  double* part = nullptr;
  if (part_total) ARB_TRY(ws<double>(ctx, WS_SS_PART, part_total, &part));
  // descriptors to the device: jobs, passes, offsets, column-sum offsets, coefficients
  const size_t bj = hj.size() * sizeof(BJob), bp = hp.size() * sizeof(BPass), bo = hoff.size() * sizeof(int64_t),
               bc = hcs.size() * sizeof(int64_t), bf = hcoef.size() * sizeof(double);
  const size_t bt = 4 * static_cast<size_t>(dmax) * sizeof(unsigned long long);  // tile tickets, zeroed
  const size_t bytes = bj + bp + bo + bc + bf + bt;
  char* desc;
  ARB_TRY(ws<char>(ctx, WS_BATCH_DESC, bytes + 512, &desc));
  const double* dcoef = reinterpret_cast<const double*>(desc + bj + bp + bo + bc);
  for (int o = 0; o < njobs; ++o) {
    hj[o].coef = dcoef + coef_at[o];
    hj[o].part = jobs[order[o]].colss ? part + part_at[o] : nullptr;
  }
  void* st;
  ARB_TRY(host_stage(ctx, bytes + 512, &st));
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // staging area free
  char* sp = static_cast<char*>(st);
  memcpy(sp, hj.data(), bj);
  memcpy(sp + bj, hp.data(), bp);
  memcpy(sp + bj + bp, hoff.data(), bo);
  memcpy(sp + bj + bp + bo, hcs.data(), bc);
  memcpy(sp + bj + bp + bo + bc, hcoef.data(), bf);
  memset(sp + bj + bp + bo + bc + bf, 0, bt);
  ARB_CUDA(ctx, cudaMemcpyAsync(desc, sp, bytes, cudaMemcpyHostToDevice, ctx->stream));
  out->dmax = dmax;
  out->dj = desc;
  out->dp = desc + bj;
  for (int k = 0; k < 4; ++k) {
    BatchPlan::Class& c = out->cls[k];
    if (c.count == 0) continue;
    c.doff = reinterpret_cast<const int64_t*>(desc + bj + bp) + off_at[k];
    c.dcs = reinterpret_cast<const int64_t*>(desc + bj + bp + bo) + cs_at[k];
    c.tickets = reinterpret_cast<unsigned long long*>(desc + bj + bp + bo + bc + bf) + static_cast<size_t>(k) * dmax;
    int per_sm = 0;
    ARB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, class_kernel(k), BT_THREADS, 0));
    c.grid = std::max(1, std::max(1, per_sm) * ctx->num_sms / std::max(1, ctx->coop_share));
  }
  out->part = part;
  return ARB_OK;
}

arb_status filter_batched_launch(arb_ctx ctx, const BatchPlan& plan) {
  if (plan.njobs <= 0) return ARB_OK;
  for (int k = 0; k < 4; ++k) {
    const BatchPlan::Class& c = plan.cls[k];
    if (c.count == 0) continue;
    const BJob* dj = static_cast<const BJob*>(plan.dj) + c.first;
    const BPass* dp = static_cast<const BPass*>(plan.dp) + static_cast<size_t>(c.first) * plan.dmax;
    const int64_t* doff = c.doff;
    const int64_t* dcs = c.dcs;
    unsigned long long* tk = c.tickets;
    int dmax = plan.dmax;
    int nj = c.count;
    void* args[] = {&dj, &dp, &doff, &nj, &dmax, &dcs, &tk};
    ARB_CUDA(ctx, cudaLaunchCooperativeKernel(class_kernel(k), dim3(c.grid), dim3(BT_THREADS), args, 0, ctx->stream));
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
