// Bulk-copy pipelined form of the fused FP32 block SpMM for matrices with short rows
// (stencils): the same computation as spmm_fused_kernel<float> - out = sy (alpha A Yin +
// beta Yin) + sx X + sz Z with an optional column reduction - for the Clenshaw passes of
// the filter (Algorithm 7 / eq. rhod), the augmentation products (Algorithm 5) and the
// Rayleigh-Ritz products (Algorithm 1) of the mixed path's FP32 phase.
//
// The register-staged kernel keeps the rows it gathers in registers, so the bytes a
// warp has in flight are bounded by its registers, and occupancy by the register file:
// on the 7-point stencil it runs latency-bound at 24 warps per SM.  Here one producer
// warp per CTA moves every row of Yin that a group of G consecutive matrix rows gathers,
// plus their X, Z and own Yin rows, into a shared-memory stage with one-dimensional bulk
// copies (cp.async.bulk, completion counted in bytes on the stage's mbarrier); S stages
// form a ring, so S*G matrix rows (about 16) are in flight per SM without holding a
// register.  Eight consumer warps compute the rows of a full stage from shared memory and
// release it.  Column indices and values of the next groups are prefetched by the producer
// two groups ahead.  Row groups are dealt to the CTAs round robin (group g to CTA
// g mod grid), so the GPU sweeps the rows as one front and the rows a stencil gathers
// from the planes around it stay in L2.
//
// Every mbarrier wait is bounded; a wait that gives up sets the context's device error
// word (read at the next host synchronisation) and the CTA stops; the producer then waits,
// again bounded, for the copies it issued before it returns.
#include <algorithm>

#include "arb_internal.h"

namespace arb {
namespace {

constexpr int BK_CONSUMERS = 8;                       // consumer warps
constexpr int BK_THREADS = (BK_CONSUMERS + 1) * 32;   // + one producer warp
constexpr long long BK_SPIN = 1ll << 26;              // mbarrier polls before giving up
constexpr int BK_MAX_STAGES = 8;

struct BulkParams {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const float* val;
  int32_t ncols;
  const float* Yin;
  int64_t ldy;
  float alpha, beta;
  const double* sy;
  const float* X;
  int64_t ldx;
  const double* sx;
  const float* Z;
  int64_t ldz;
  const double* sz;
  float* out;
  int64_t ldo;
  double* red_part;
  int dot_with_yin;
  int need_yi;
  int G;        // matrix rows per group (stage)
  int S;        // stages
  int slots;    // slots per row: maxnz + 3 (X, Z, own Yin row)
  int maxnz;
  int32_t* err;
};

__device__ __forceinline__ unsigned bk_smem(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void bk_mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bk_smem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bk_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bk_smem(bar)) : "memory");
}
__device__ __forceinline__ void bk_arrive_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bk_smem(bar)), "r"(bytes) : "memory");
}
// bounded wait for the phase of the given parity; false if it gave up
__device__ __forceinline__ bool bk_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = bk_smem(bar);
  for (long long it = 0; it < BK_SPIN; ++it) {
    unsigned done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t"
        "}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// global -> shared bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(bk_smem(dst)),
      "l"(src), "r"(bytes), "r"(bk_smem(bar))
      : "memory");
}

struct BulkLayout {
  int bar_off, coef_off, meta_off, meta_bytes, slot_off, stage_bytes, total;
};

__host__ __device__ inline BulkLayout bulk_layout(int ncols, int G, int S, int slots, int maxnz) {
  BulkLayout L;
  const int rowbytes = ncols * 4;
  L.bar_off = 0;
  L.coef_off = 128;  // 2 S barriers of 8 bytes fit below (S <= 8)
  L.meta_off = L.coef_off + ((3 * ncols * 4 + 127) / 128) * 128;
  L.meta_bytes = ((G * (maxnz + 1) * 4 + 127) / 128) * 128;  // per stage: G counts + G x maxnz values
  L.slot_off = L.meta_off + S * L.meta_bytes;
  L.stage_bytes = G * slots * rowbytes;
  L.total = L.slot_off + S * L.stage_bytes;
  return L;
}

template <bool RED>
__global__ void __launch_bounds__(BK_THREADS, 1) spmm_bulk_f32_kernel(BulkParams P) {
  extern __shared__ __align__(128) unsigned char bk_sm[];
  const int ncols = P.ncols, G = P.G, S = P.S, SL = P.slots, MZ = P.maxnz;
  const int nc4 = ncols / 4;
  const unsigned rowbytes = static_cast<unsigned>(ncols) * 4u;
  const BulkLayout L = bulk_layout(ncols, G, S, SL, MZ);
  uint64_t* full = reinterpret_cast<uint64_t*>(bk_sm + L.bar_off);
  uint64_t* empty = full + BK_MAX_STAGES;
  float* csy = reinterpret_cast<float*>(bk_sm + L.coef_off);
  float* csx = csy + ncols;
  float* csz = csx + ncols;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ngroups = (P.n + G - 1) / G;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      bk_mbar_init(&full[s], 1);
      bk_mbar_init(&empty[s], BK_CONSUMERS);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int c = tid; c < ncols; c += blockDim.x) {
    csy[c] = P.sy ? static_cast<float>(P.sy[c]) : 1.f;
    csx[c] = P.X ? static_cast<float>(P.sx[c]) : 0.f;
    csz[c] = P.Z ? static_cast<float>(P.sz[c]) : 0.f;
  }
  __syncthreads();

  if (warp == BK_CONSUMERS) {
    // ---------------------------------------------------------------- producer warp
    const int nstream = (P.X ? 1 : 0) + (P.Z ? 1 : 0) + (P.need_yi ? 1 : 0);
    // register pipeline: row pointers of group it+1 (lanes 0..G), column index and value
    // of the nonzeros of group it (two per lane: flattened index f = lane, lane + 32)
    int rp_cur = 0, rp_next = 0;
    int c0 = 0, c1 = 0;
    float v0 = 0.f, v1 = 0.f;
    auto load_rp = [&](int64_t g) -> int {
      const int64_t r = g * G + lane;
      if (g < ngroups && lane <= G) return __ldg(P.rowptr + (r < P.n ? r : P.n));
      return 0;
    };
    auto load_cv = [&](int64_t g, int rp, int& ca, int& cb, float& va, float& vb) {
      const int b = __shfl_sync(0xffffffffu, rp, 0), e = __shfl_sync(0xffffffffu, rp, G);
      ca = cb = 0;
      va = vb = 0.f;
      if (g >= ngroups) return;
      if (b + lane < e) {
        ca = __ldg(P.col + b + lane);
        va = __ldg(P.val + b + lane);
      }
      if (b + lane + 32 < e) {
        cb = __ldg(P.col + b + lane + 32);
        vb = __ldg(P.val + b + lane + 32);
      }
    };
    int64_t g = blockIdx.x;
    rp_cur = load_rp(g);
    load_cv(g, rp_cur, c0, c1, v0, v1);
    rp_next = load_rp(g + gridDim.x);
    int it = 0;
    bool ok = true;
    for (; g < ngroups; g += gridDim.x, ++it) {
      const int s = it % S;
      // prefetch: nonzeros of the next group, row pointers of the one after
      int n_c0, n_c1;
      float n_v0, n_v1;
      load_cv(g + gridDim.x, rp_next, n_c0, n_c1, n_v0, n_v1);
      const int rp_next2 = load_rp(g + 2 * static_cast<int64_t>(gridDim.x));
      if (it >= S && !bk_wait(&empty[s], ((it / S) - 1) & 1)) {
        ok = false;
        break;
      }
      if (abort_flag) {
        ok = false;
        break;
      }
      const int64_t r0 = g * G;
      const int nr = static_cast<int>(P.n - r0 < G ? P.n - r0 : G);
      const int b = __shfl_sync(0xffffffffu, rp_cur, 0);
      const int nnzg = __shfl_sync(0xffffffffu, rp_cur, nr) - b;
      int* cnt = reinterpret_cast<int*>(bk_sm + L.meta_off + s * L.meta_bytes);
      float* vals = reinterpret_cast<float*>(cnt + G);
      unsigned char* stage = bk_sm + L.slot_off + static_cast<size_t>(s) * L.stage_bytes;
      // row and position of the flattened nonzero f
      auto place = [&](int f, int& i, int& j) {
        i = 0;
        for (int q = 1; q < nr; ++q)
          if (f >= __shfl_sync(0xffffffffu, rp_cur, q) - b) i = q;
        j = f - (__shfl_sync(0xffffffffu, rp_cur, i) - b);
      };
      int i0, j0, i1, j1;
      place(lane, i0, j0);
      place(lane + 32, i1, j1);
      // every lane takes part in the shuffles; only the first nr lanes store a count
      const int rpa = __shfl_sync(0xffffffffu, rp_cur, lane < G ? lane : G);
      const int rpb = __shfl_sync(0xffffffffu, rp_cur, lane < G ? lane + 1 : G);
      if (lane < nr) cnt[lane] = min(rpb - rpa, MZ);
      if (lane < nnzg && j0 < MZ) vals[i0 * MZ + j0] = v0;
      if (lane + 32 < nnzg && j1 < MZ) vals[i1 * MZ + j1] = v1;
      __syncwarp();
      if (lane == 0) bk_arrive_expect(&full[s], static_cast<unsigned>(nnzg + nstream * nr) * rowbytes);
      __syncwarp();
      // (the host admits only matrices whose rows have at most maxnz nonzeros, so j < MZ and
      // every copy that the expected byte count includes is issued)
      if (lane < nnzg)
        bk_copy(stage + static_cast<size_t>(i0 * SL + min(j0, MZ - 1)) * rowbytes,
                P.Yin + static_cast<int64_t>(c0) * P.ldy, rowbytes, &full[s]);
      if (lane + 32 < nnzg)
        bk_copy(stage + static_cast<size_t>(i1 * SL + min(j1, MZ - 1)) * rowbytes,
                P.Yin + static_cast<int64_t>(c1) * P.ldy, rowbytes, &full[s]);
      for (int t = lane; t < nstream * nr; t += 32) {
        const int kind = t / nr, i = t % nr;
        int which = 0, seen = 0;  // the kind-th present stream: 0 = X, 1 = Z, 2 = own Yin row
        for (int w = 0; w < 3; ++w) {
          const bool present = (w == 0 && P.X) || (w == 1 && P.Z) || (w == 2 && P.need_yi);
          if (present) {
            if (seen == kind) which = w;
            ++seen;
          }
        }
        const int64_t row = r0 + i;
        const float* src = which == 0 ? P.X + row * P.ldx : (which == 1 ? P.Z + row * P.ldz : P.Yin + row * P.ldy);
        bk_copy(stage + static_cast<size_t>(i * SL + MZ + which) * rowbytes, src, rowbytes, &full[s]);
      }
      rp_cur = rp_next;
      rp_next = rp_next2;
      c0 = n_c0;
      c1 = n_c1;
      v0 = n_v0;
      v1 = n_v1;
    }
    if (!ok) {
      if (lane == 0) {
        abort_flag = 1;
        atomicExch(P.err, 1);
      }
      // wait (bounded) for the copies of the stages issued and possibly not yet landed
      for (int back = 1; back <= S && back <= it; ++back) {
        const int ib = it - back;
        bk_wait(&full[ib % S], (ib / S) & 1);
      }
    }
    return;
  }

  // ---------------------------------------------------------------- consumer warps
  const int ctid = tid;  // 0 .. 32 BK_CONSUMERS - 1
  const int nthr = BK_CONSUMERS * 32;
  const int rows_per_pass = max(1, nthr / max(nc4, 1));
  const bool active = ctid < rows_per_pass * nc4;
  const int c4 = active ? ctid % nc4 : 0;
  const int ri = active ? ctid / nc4 : 0;
  const int c = 4 * c4;
  float ky[4], kx[4], kz[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    ky[u] = csy[c + u];
    kx[u] = csx[c + u];
    kz[u] = csz[c + u];
  }
  double red[4] = {0.0, 0.0, 0.0, 0.0};
  int it = 0;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x, ++it) {
    const int s = it % S;
    if (!bk_wait(&full[s], (it / S) & 1) || abort_flag) {
      if (lane == 0) {
        abort_flag = 1;
        atomicExch(P.err, 1);
      }
      break;
    }
    const int64_t r0 = g * G;
    const int nr = static_cast<int>(P.n - r0 < G ? P.n - r0 : G);
    const int* cnt = reinterpret_cast<const int*>(bk_sm + L.meta_off + s * L.meta_bytes);
    const float* vals = reinterpret_cast<const float*>(cnt + G);
    const unsigned char* stage = bk_sm + L.slot_off + static_cast<size_t>(s) * L.stage_bytes;
    if (active) {
      for (int i = ri; i < nr; i += rows_per_pass) {
        const float4* rs = reinterpret_cast<const float4*>(stage + static_cast<size_t>(i * SL) * rowbytes) + c4;
        const int nz = min(cnt[i], MZ);
        float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
        for (int j = 0; j < nz; ++j) {
          const float v = vals[i * MZ + j];
          const float4 y = rs[static_cast<size_t>(j) * (rowbytes / 16)];
          const float2 v2 = make_float2(v, v);
          a01 = __ffma2_rn(v2, make_float2(y.x, y.y), a01);
          a23 = __ffma2_rn(v2, make_float2(y.z, y.w), a23);
        }
        float4 yi = make_float4(0.f, 0.f, 0.f, 0.f), xv = yi, zv = yi;
        if (P.need_yi) yi = rs[static_cast<size_t>(MZ + 2) * (rowbytes / 16)];
        if (P.X) xv = rs[static_cast<size_t>(MZ) * (rowbytes / 16)];
        if (P.Z) zv = rs[static_cast<size_t>(MZ + 1) * (rowbytes / 16)];
        // o = sy (alpha acc + beta yi) + sx x + sz z, as the register-staged kernel forms it
        const float2 al2 = make_float2(P.alpha, P.alpha), be2 = make_float2(P.beta, P.beta);
        float2 r01 = __fmul2_rn(be2, make_float2(yi.x, yi.y));
        float2 r23 = __fmul2_rn(be2, make_float2(yi.z, yi.w));
        r01 = __ffma2_rn(al2, a01, r01);
        r23 = __ffma2_rn(al2, a23, r23);
        r01 = __fmul2_rn(make_float2(ky[0], ky[1]), r01);
        r23 = __fmul2_rn(make_float2(ky[2], ky[3]), r23);
        if (P.X) {
          r01 = __ffma2_rn(make_float2(kx[0], kx[1]), make_float2(xv.x, xv.y), r01);
          r23 = __ffma2_rn(make_float2(kx[2], kx[3]), make_float2(xv.z, xv.w), r23);
        }
        if (P.Z) {
          r01 = __ffma2_rn(make_float2(kz[0], kz[1]), make_float2(zv.x, zv.y), r01);
          r23 = __ffma2_rn(make_float2(kz[2], kz[3]), make_float2(zv.z, zv.w), r23);
        }
        const float4 o = make_float4(r01.x, r01.y, r23.x, r23.y);
        __stcs(reinterpret_cast<float4*>(P.out + (r0 + i) * P.ldo + c), o);
        if constexpr (RED) {
          const float ov[4] = {o.x, o.y, o.z, o.w};
          const float yv[4] = {yi.x, yi.y, yi.z, yi.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const double od = static_cast<double>(ov[u]);
            red[u] += P.dot_with_yin ? od * static_cast<double>(yv[u]) : od * od;
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) bk_arrive(&empty[s]);
  }
  if constexpr (RED) {
    // per-CTA column sums: the threads of one column (one per row slot) in a fixed order
    double* sred = reinterpret_cast<double*>(bk_sm + L.slot_off);  // the stages are free now
    // the producer may still be waiting on a stage only after an abort; results are then void
    __syncwarp();
    asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
    if (active)
#pragma unroll
      for (int u = 0; u < 4; ++u) sred[static_cast<size_t>(ri) * ncols + c + u] = red[u];
    asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
    for (int cc = ctid; cc < ncols; cc += nthr) {
      double sum = 0.0;
      for (int q = 0; q < rows_per_pass; ++q) sum += sred[static_cast<size_t>(q) * ncols + cc];
      P.red_part[static_cast<size_t>(blockIdx.x) * ncols + cc] = sum;
    }
  }
}

inline bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// Launches the bulk-copy kernel when the operands allow it (rows of at most 32 nonzeros,
// ncols a multiple of 4, 16-byte aligned rows, a full ring of at least 3 stages in shared
// memory); *launched says whether it did.  With want_red the per-CTA partial column sums
// go to a grid x ncols workspace returned in *part (grid in *grid_out).
arb_status spmm_bulk_f32(arb_ctx ctx, const arb_mat_s* A, const SpmmArgs<float>& a, const float* val, bool want_red,
                         bool* launched, int* grid_out, double** part) {
  *launched = false;
#if defined(ARB_SPMM_BULK) && ARB_SPMM_BULK == 0
  return ARB_OK;
#endif
  const int maxnz = A->max_row_nnz;
  if (A->sell_C > 0 || maxnz < 0 || maxnz > 32 || !a.out || a.ncols % 4 != 0 || a.ncols > 1024) return ARB_OK;
  auto ok_blk = [](const float* p, int64_t ld) { return !p || (al16(p) && ld % 4 == 0); };
  if (!ok_blk(a.Yin, a.ldy) || !ok_blk(a.X, a.ldx) || !ok_blk(a.Z, a.ldz) || !ok_blk(a.out, a.ldo)) return ARB_OK;
  if (a.X && !a.sx) return ARB_OK;
  if (a.Z && !a.sz) return ARB_OK;
  const int G = std::max(1, std::min(4, 64 / std::max(maxnz, 1)));
  const int slots = std::max(maxnz, 1) + 3;
  const int smem_max = 227 * 1024;
  int S = BK_MAX_STAGES;
  while (S >= 3 && bulk_layout(a.ncols, G, S, slots, std::max(maxnz, 1)).total > smem_max) --S;
  if (S < 3) return ARB_OK;
  BulkParams P;
  P.n = A->n;
  P.rowptr = A->rowptr;
  P.col = A->col;
  P.val = val;
  P.ncols = a.ncols;
  P.Yin = a.Yin;
  P.ldy = a.ldy;
  P.alpha = static_cast<float>(a.alpha);
  P.beta = static_cast<float>(a.beta);
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
  P.need_yi = (a.beta != 0.0 || (want_red && a.dot_with_yin)) ? 1 : 0;
  P.G = G;
  P.S = S;
  P.slots = slots;
  P.maxnz = std::max(maxnz, 1);
  ARB_TRY(device_error_word(ctx, &P.err));
  const BulkLayout L = bulk_layout(a.ncols, G, S, slots, P.maxnz);
  const int64_t ngroups = (A->n + G - 1) / G;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ngroups, ctx->num_sms)));
  // the column reduction reuses the stage area: it must hold rows_per_pass x ncols doubles
  const int rows_per_pass = std::max(1, (BK_CONSUMERS * 32) / (a.ncols / 4));
  if (want_red && static_cast<int64_t>(rows_per_pass) * a.ncols * 8 > static_cast<int64_t>(S) * L.stage_bytes)
    return ARB_OK;
  P.red_part = nullptr;
  if (want_red) ARB_TRY(ws<double>(ctx, WS_SS_PART, static_cast<size_t>(grid) * a.ncols, &P.red_part));
  void (*kern)(BulkParams) = want_red ? spmm_bulk_f32_kernel<true> : spmm_bulk_f32_kernel<false>;
  ARB_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total));
  kern<<<grid, BK_THREADS, L.total, ctx->stream>>>(P);
  ARB_LAUNCHED(ctx);
  *launched = true;
  *grid_out = grid;
  *part = P.red_part;
  return ARB_OK;
}

}  // namespace arb
