// Bulk-copy pipelined form of the fused FP32 block SpMM for matrices with short rows
// (stencils): the same computation as spmm_fused_kernel<float> - out = sy (alpha A Yin +
// beta Yin) + sx X + sz Z with an optional column reduction - for the Clenshaw passes of
// the filter (Algorithm 7 / eq. rhod), the augmentation products (Algorithm 5) and the
// Rayleigh-Ritz products (Algorithm 1) of the mixed path's FP32 phase.
//
// The register-staged kernel keeps the rows it gathers in registers, so the bytes a warp
// has in flight are bounded by its registers, and occupancy by the register file: on the
// 7-point stencil it runs latency-bound at 24 warps per SM.  Here producer warps move
// every row of Yin that a group of G consecutive matrix rows gathers, plus their X, Z
// (and, when the diagonal is not stored, own Yin) rows, into a shared-memory stage with
// one-dimensional bulk copies (cp.async.bulk, completion counted in bytes on the stage's
// mbarrier); S stages form a ring, so S*G matrix rows are in flight per SM without
// holding a register.  Eight consumer warps compute the rows of a full stage from shared
// memory and release it.
//
// The matrix is read through a group table made once per matrix (bulk_table_kernel): for
// every group of G rows one 16-byte aligned record with the distinct rows of Yin the group
// gathers (a row that several of its rows gather - the +-1 neighbours of a stencil - is
// copied once), the map from each nonzero to its distinct row, the row lengths, the
// position of each row's diagonal and the FP32 values.  Producers fetch the record of the
// group S iterations ahead with one more bulk copy into a ring of 2S records, so issuing a
// group's copies waits on no global load.  Row groups are dealt to the CTAs round robin
// (group g to CTA g mod grid), so the GPU sweeps the rows as one front and the rows a
// stencil gathers from the planes around it stay in L2.  Within a row the products are
// summed in CSR order with the operations of the register-staged kernel, so the results
// are bitwise equal to it.
//
// Every mbarrier wait is bounded; a wait that gives up sets the context's device error
// word (read at the next host synchronisation) and the CTA stops; each producer then
// waits, again bounded, for the copies it issued before it returns.
#include <algorithm>

#include "arb_internal.h"

namespace arb {
namespace {

#ifndef ARB_BULK_PRODUCERS
#define ARB_BULK_PRODUCERS 4
#endif
#ifndef ARB_BULK_ROWS
#define ARB_BULK_ROWS 4
#endif
constexpr int BK_CONSUMERS = 8;                       // consumer warps
constexpr int BK_PRODUCERS = ARB_BULK_PRODUCERS;      // producer warps
constexpr int BK_THREADS = (BK_CONSUMERS + BK_PRODUCERS) * 32;
constexpr long long BK_SPIN = 1ll << 26;              // mbarrier polls before giving up
constexpr int BK_MAX_STAGES = 8;

// Group record (int32 words): [0] nu = distinct rows gathered; [1, 1+G) row lengths;
// [1+G, 1+2G) position (distinct-row index) of each row's own Yin row, -1 if its diagonal
// is not stored; then NZG = G*maxnz source rows of the distinct list (padded with 0), NZG
// distinct-row indices of the nonzeros (row i, nonzero j at i*maxnz + j), NZG FP32 values.
__host__ __device__ inline int rec_words(int G, int maxnz) { return ((1 + 2 * G + 3 * G * maxnz) + 3) / 4 * 4; }

struct BulkParams {
  int64_t n;
  const int32_t* tab;  // group records
  int32_t rec;         // words per record
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
  int G;      // matrix rows per group (stage)
  int S;      // stages
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
  int bar_off, coef_off, rec_off, rec_bytes, slot_off, slots, stage_bytes, total;
};

// barriers: full[S], empty[S], ibar[2S] (8 bytes each, 256 bytes for S <= 8); the three
// coefficient rows; 2S records; S stages of NZG + 3G row slots (distinct gathered rows,
// then X, Z and own-Yin rows)
__host__ __device__ inline BulkLayout bulk_layout(int ncols, int G, int S, int maxnz) {
  BulkLayout L;
  const int rowbytes = ncols * 4;
  L.bar_off = 0;
  L.coef_off = 256;
  L.rec_off = L.coef_off + ((3 * ncols * 4 + 127) / 128) * 128;
  L.rec_bytes = rec_words(G, maxnz) * 4;
  L.slot_off = L.rec_off + ((2 * S * L.rec_bytes + 127) / 128) * 128;
  L.slots = G * maxnz + 3 * G;
  L.stage_bytes = L.slots * rowbytes;
  L.total = L.slot_off + S * L.stage_bytes;
  return L;
}

// One thread per group: the record of rows [g G, g G + G) from the CSR arrays.
__global__ void bulk_table_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const float* __restrict__ val, int G, int maxnz, int rec, int32_t* __restrict__ tab) {
  const int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t ngroups = (n + G - 1) / G;
  if (g >= ngroups) return;
  int32_t* r = tab + g * rec;
  const int NZG = G * maxnz;
  int32_t* cnt = r + 1;
  int32_t* yslot = r + 1 + G;
  int32_t* src = r + 1 + 2 * G;
  int32_t* map = src + NZG;
  float* vals = reinterpret_cast<float*>(map + NZG);
  for (int w = 0; w < rec; ++w) r[w] = 0;
  int nu = 0;
  for (int i = 0; i < G; ++i) {
    const int64_t row = g * G + i;
    yslot[i] = -1;
    if (row >= n) continue;
    const int b = rowptr[row], e = rowptr[row + 1];
    const int len = min(e - b, maxnz);
    cnt[i] = len;
    for (int j = 0; j < len; ++j) {
      const int c = col[b + j];
      int u = 0;
      while (u < nu && src[u] != c) ++u;
      if (u == nu) src[nu++] = c;
      map[i * maxnz + j] = u;
      vals[i * maxnz + j] = val[b + j];
      if (c == row) yslot[i] = u;
    }
  }
  r[0] = nu;
}

template <bool RED>
__global__ void __launch_bounds__(BK_THREADS, 1) spmm_bulk_f32_kernel(BulkParams P) {
  extern __shared__ __align__(128) unsigned char bk_sm[];
  const int ncols = P.ncols, G = P.G, S = P.S, MZ = P.maxnz;
  const int NZG = G * MZ;
  const int nc4 = ncols / 4;
  const unsigned rowbytes = static_cast<unsigned>(ncols) * 4u;
  const unsigned rstride = rowbytes / 16;  // float4 per slot
  const BulkLayout L = bulk_layout(ncols, G, S, MZ);
  uint64_t* full = reinterpret_cast<uint64_t*>(bk_sm + L.bar_off);
  uint64_t* empty = full + BK_MAX_STAGES;
  uint64_t* ibar = empty + BK_MAX_STAGES;  // 2 BK_MAX_STAGES
  float* csy = reinterpret_cast<float*>(bk_sm + L.coef_off);
  float* csx = csy + ncols;
  float* csz = csx + ncols;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ngroups = (P.n + G - 1) / G;
  auto record = [&](int it) { return reinterpret_cast<int32_t*>(bk_sm + L.rec_off + (it % (2 * S)) * L.rec_bytes); };
  auto group_of = [&](int it) { return static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(it) * gridDim.x; };
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      bk_mbar_init(&full[s], 1);
      bk_mbar_init(&empty[s], BK_CONSUMERS);
    }
    for (int s = 0; s < 2 * S; ++s) bk_mbar_init(&ibar[s], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int c = tid; c < ncols; c += blockDim.x) {
    csy[c] = P.sy ? static_cast<float>(P.sy[c]) : 1.f;
    csx[c] = P.X ? static_cast<float>(P.sx[c]) : 0.f;
    csz[c] = P.Z ? static_cast<float>(P.sz[c]) : 0.f;
  }
  __syncthreads();

  if (warp >= BK_CONSUMERS) {
    // ---------------------------------------------------------------- producer warps
    // Producer w issues the iterations it = w, w + P, w + 2P, ... (P producers); S is a
    // multiple of P, so every stage and every record slot - and their barriers - belongs
    // to one producer, which uses them in iteration order.  At iteration it the producer
    // fetches the record of iteration it + S into the slot that iteration it - S has
    // released, then issues the row copies of iteration it from its record.
    const int w = warp - BK_CONSUMERS;
    const unsigned recb = static_cast<unsigned>(L.rec_bytes);
    auto fetch_record = [&](int it) {
      const int64_t g = group_of(it);
      if (g >= ngroups) return;
      if (lane == 0) {
        uint64_t* b = &ibar[it % (2 * S)];
        bk_arrive_expect(b, recb);
        bk_copy(record(it), P.tab + g * P.rec, recb, b);
      }
    };
    for (int it = w; it < S; it += BK_PRODUCERS) fetch_record(it);
    int it = w;
    bool ok = true;
    for (; group_of(it) < ngroups; it += BK_PRODUCERS) {
      const int s = it % S;
      if (it >= S && !bk_wait(&empty[s], ((it / S) - 1) & 1)) {
        ok = false;
        break;
      }
      if (abort_flag) {
        ok = false;
        break;
      }
      fetch_record(it + S);
      if (!bk_wait(&ibar[it % (2 * S)], (it / (2 * S)) & 1)) {
        ok = false;
        break;
      }
      const int32_t* rec = record(it);
      const int64_t r0 = group_of(it) * G;
      const int nr = static_cast<int>(P.n - r0 < G ? P.n - r0 : G);
      const int nu = min(rec[0], NZG);
      const int32_t* yslot = rec + 1 + G;
      const int32_t* src = rec + 1 + 2 * G;
      // rows without a stored diagonal take their own Yin row as a stream of its own
      int ny = 0;
      if (P.need_yi)
        for (int i = 0; i < nr; ++i) ny += yslot[i] < 0;
      const int nxz = (P.X ? nr : 0) + (P.Z ? nr : 0);
      unsigned char* stage = bk_sm + L.slot_off + static_cast<size_t>(s) * L.stage_bytes;
      if (lane == 0) bk_arrive_expect(&full[s], static_cast<unsigned>(nu + nxz + ny) * rowbytes);
      __syncwarp();
      for (int f = lane; f < nu; f += 32)
        bk_copy(stage + static_cast<size_t>(f) * rowbytes, P.Yin + static_cast<int64_t>(src[f]) * P.ldy, rowbytes,
                &full[s]);
      for (int t = lane; t < 3 * nr; t += 32) {
        const int kind = t / nr, i = t % nr;
        const int64_t row = r0 + i;
        if (kind == 0 && P.X)
          bk_copy(stage + static_cast<size_t>(NZG + i) * rowbytes, P.X + row * P.ldx, rowbytes, &full[s]);
        if (kind == 1 && P.Z)
          bk_copy(stage + static_cast<size_t>(NZG + G + i) * rowbytes, P.Z + row * P.ldz, rowbytes, &full[s]);
        if (kind == 2 && P.need_yi && yslot[i] < 0)
          bk_copy(stage + static_cast<size_t>(NZG + 2 * G + i) * rowbytes, P.Yin + row * P.ldy, rowbytes, &full[s]);
      }
    }
    if (!ok) {
      if (lane == 0) {
        abort_flag = 1;
        atomicExch(P.err, 1);
      }
      // wait (bounded) for the copies of this producer that may not have landed: the
      // stages of its last S iterations and the records it fetched ahead
      for (int ib = it - BK_PRODUCERS; ib >= 0 && ib >= it - S; ib -= BK_PRODUCERS)
        bk_wait(&full[ib % S], (ib / S) & 1);
      for (int ib = it; ib < it + S; ib += BK_PRODUCERS)
        if (group_of(ib) < ngroups) bk_wait(&ibar[ib % (2 * S)], (ib / (2 * S)) & 1);
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
  for (int it = 0; group_of(it) < ngroups; ++it) {
    const int s = it % S;
    if (!bk_wait(&full[s], (it / S) & 1) || abort_flag) {
      if (lane == 0) {
        abort_flag = 1;
        atomicExch(P.err, 1);
      }
      break;
    }
    const int64_t r0 = group_of(it) * G;
    const int nr = static_cast<int>(P.n - r0 < G ? P.n - r0 : G);
    const int32_t* rec = record(it);
    const int32_t* cnt = rec + 1;
    const int32_t* yslot = rec + 1 + G;
    const int32_t* map = rec + 1 + 2 * G + NZG;
    const float* vals = reinterpret_cast<const float*>(map + NZG);
    const float4* stage = reinterpret_cast<const float4*>(bk_sm + L.slot_off + static_cast<size_t>(s) * L.stage_bytes) + c4;
    if (active) {
      for (int i = ri; i < nr; i += rows_per_pass) {
        const int nz = min(cnt[i], MZ);
        float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
        for (int j = 0; j < nz; ++j) {
          const float v = vals[i * MZ + j];
          const int u = min(max(map[i * MZ + j], 0), NZG - 1);
          const float4 y = stage[static_cast<size_t>(u) * rstride];
          const float2 v2 = make_float2(v, v);
          a01 = __ffma2_rn(v2, make_float2(y.x, y.y), a01);
          a23 = __ffma2_rn(v2, make_float2(y.z, y.w), a23);
        }
        float4 yi = make_float4(0.f, 0.f, 0.f, 0.f), xv = yi, zv = yi;
        if (P.need_yi) {
          const int ys = yslot[i];
          yi = stage[static_cast<size_t>(ys >= 0 ? min(ys, NZG - 1) : NZG + 2 * G + i) * rstride];
        }
        if (P.X) xv = stage[static_cast<size_t>(NZG + i) * rstride];
        if (P.Z) zv = stage[static_cast<size_t>(NZG + G + i) * rstride];
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
    // per-CTA column sums: the threads of one column (one per row slot) in a fixed order,
    // through the stage area (no copy is in flight once every group has been consumed; after
    // an abort the results are void)
    double* sred = reinterpret_cast<double*>(bk_sm + L.slot_off);
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

inline int bulk_rows(int maxnz) { return std::max(1, std::min(ARB_BULK_ROWS, 64 / std::max(maxnz, 1))); }

}  // namespace

void matrix_free_bulk(arb_mat m) {
  if (m->bulk_tab) cudaFree(m->bulk_tab);
  m->bulk_tab = nullptr;
}

// The group table of the matrix for groups of bulk_rows(maxnz) rows (made on first use,
// with the FP32 values, and kept with the matrix).
static arb_status ensure_bulk_table(arb_ctx ctx, arb_mat mat, const float* val32) {
  std::lock_guard<std::mutex> lock(mat->mu);
  if (mat->bulk_tab) return ARB_OK;
  const int maxnz = std::max(mat->max_row_nnz, 1);
  const int G = bulk_rows(maxnz);
  const int rec = rec_words(G, maxnz);
  const int64_t ngroups = (mat->n + G - 1) / G;
  int32_t* tab = nullptr;
  ARB_CUDA(ctx, cudaMalloc(&tab, static_cast<size_t>(ngroups) * rec * sizeof(int32_t)));
  bulk_table_kernel<<<static_cast<int>((ngroups + 127) / 128), 128, 0, ctx->stream>>>(mat->n, mat->rowptr, mat->col,
                                                                                      val32, G, maxnz, rec, tab);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // other contexts may use the table next
  ctx->launches++;
  if (e != cudaSuccess) {
    cudaFree(tab);
    return cuda_error(ctx, e, "bulk group table", __FILE__, __LINE__);
  }
  mat->bulk_tab = tab;
  return ARB_OK;
}

// Launches the bulk-copy kernel when the operands allow it (CSR rows of at most 32
// nonzeros, ncols a multiple of 4, 16-byte aligned rows, a ring of stages in shared
// memory, S a multiple of the producer warps); *launched says whether it did.  With
// want_red the per-CTA partial column sums go to a grid x ncols workspace returned in
// *part (grid in *grid_out).
arb_status spmm_bulk_f32(arb_ctx ctx, const arb_mat_s* A, const SpmmArgs<float>& a, const float* val, bool want_red,
                         bool* launched, int* grid_out, double** part) {
  *launched = false;
#if defined(ARB_SPMM_BULK) && ARB_SPMM_BULK == 0
  return ARB_OK;
#endif
  const int maxnz = A->max_row_nnz;
  if (A->sell_C > 0 || maxnz < 1 || maxnz > 32 || !a.out || a.ncols % 4 != 0 || a.ncols > 1024) return ARB_OK;
  auto ok_blk = [](const float* p, int64_t ld) { return !p || (al16(p) && ld % 4 == 0); };
  if (!ok_blk(a.Yin, a.ldy) || !ok_blk(a.X, a.ldx) || !ok_blk(a.Z, a.ldz) || !ok_blk(a.out, a.ldo)) return ARB_OK;
  if (a.X && !a.sx) return ARB_OK;
  if (a.Z && !a.sz) return ARB_OK;
  const int G = bulk_rows(maxnz);
  const int smem_max = 227 * 1024;
  // stages: a multiple of the producer count (each stage belongs to one producer)
  int S = (BK_MAX_STAGES / BK_PRODUCERS) * BK_PRODUCERS;
  while (S >= BK_PRODUCERS && bulk_layout(a.ncols, G, S, maxnz).total > smem_max) S -= BK_PRODUCERS;
  if (S < BK_PRODUCERS || S < 2) return ARB_OK;
  const BulkLayout L = bulk_layout(a.ncols, G, S, maxnz);
  // the column reduction reuses the stage area: it must hold rows_per_pass x ncols doubles
  const int rows_per_pass = std::max(1, (BK_CONSUMERS * 32) / (a.ncols / 4));
  if (want_red && static_cast<int64_t>(rows_per_pass) * a.ncols * 8 > static_cast<int64_t>(S) * L.stage_bytes)
    return ARB_OK;
  ARB_TRY(ensure_bulk_table(ctx, const_cast<arb_mat>(A), val));
  BulkParams P;
  P.n = A->n;
  P.tab = A->bulk_tab;
  P.rec = rec_words(G, maxnz);
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
  P.maxnz = maxnz;
  ARB_TRY(device_error_word(ctx, &P.err));
  const int64_t ngroups = (A->n + G - 1) / G;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ngroups, ctx->num_sms)));
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
