// Tensor-core (tcgen05) Gram products of FP32 blocks: part[s] = X^T Y over the rows of
// split s, the FP32 phase's Gram products (inner stop rule eq. inn-stop, orth(Z) and
// H = U^T A U of Algorithm 1).
//
// Split-TF32 ("3xTF32"): every FP32 operand x is cut into hi = x rounded to the nearest
// TF32 number and lo = the remainder x - hi rounded to TF32 (x = hi + lo to 2^-23), and
// x*y is formed as hi*hi + hi*lo + lo*hi by tcgen05.mma.kind::tf32 products.  The tensor
// core's FP32 accumulation in tensor memory does not round to nearest, and accumulating
// long runs there biases sums of squares by ~1e-6 relative (measured), so every 32-row
// step gives each K slice of eight rows its own fresh accumulator for hi*hi (the cross
// terms, 2^-11 smaller, share one): the step's partial sums are read back, added in
// registers in FP32 (round to nearest), and folded every 256 rows into double-float sums.
//
// CTA tile: 128 columns of X (the MMA's M, tensor-memory lanes) x 64 columns of Y (N,
// tensor-memory columns), rows of the split in steps of 32.  Operands are staged by all
// 256 threads into shared memory in the canonical K-major layout without swizzling (core
// matrices of 8 rows x 16 bytes; LBO = 128 bytes between the two core matrices of one MMA's
// K = 8, SBO = 1024 bytes between 8-row groups); one elected thread issues the MMAs and
// commits them to an mbarrier.  Every wait on the mbarrier is bounded; a wait that gives
// up sets the error word and the CTA stops issuing work.
#include <algorithm>

#include "arb_internal.h"

namespace arb {
namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;          // columns of X per CTA (MMA M)
constexpr int TC_N = 64;           // columns of Y per CTA (MMA N)
constexpr int TC_KS = 32;          // rows per pipeline step
constexpr int TC_FOLD = 8;         // steps (256 rows) per fold of the FP32 run sums into double-float
constexpr int TC_TMEM_COLS = 512;  // accumulators: 4 leading-product slices + 1 cross-product, 64 columns each
constexpr int TC_A_BYTES = TC_M * TC_KS * 4;   // one operand copy (hi or lo) of the X tile
constexpr int TC_B_BYTES = TC_N * TC_KS * 4;
constexpr int TC_STAGE = 2 * TC_A_BYTES + 2 * TC_B_BYTES;  // hi, lo of both
constexpr int TC_SMEM = TC_STAGE + 1024;                   // one stage + barrier
constexpr long long TC_SPIN = 1ll << 26;                   // mbarrier polls before giving up

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ unsigned long long make_sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= static_cast<unsigned long long>((saddr >> 4) & 0x3fff);
  d |= static_cast<unsigned long long>((lbo >> 4) & 0x3fff) << 16;
  d |= static_cast<unsigned long long>((sbo >> 4) & 0x3fff) << 32;
  d |= 1ull << 46;  // descriptor version of this architecture
  return d;         // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = 64
__host__ __device__ constexpr unsigned make_idesc_tf32(int m, int n) {
  return (1u << 4)                            // D format F32
         | (2u << 7)                          // A format TF32
         | (2u << 10)                         // B format TF32
         | (static_cast<unsigned>(n >> 3) << 17) | (static_cast<unsigned>(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t"
      "}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mbar_init(void* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the phase with the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait(void* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (long long it = 0; it < TC_SPIN; ++it) {
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

__device__ __forceinline__ void mma_commit(void* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row, k) of a K-major no-swizzle operand tile with TC_KS columns of K
__device__ __forceinline__ int kmajor_off(int row, int k) {
  return (row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// x rounded to the nearest TF32 number (ties away from zero): low 13 significand bits
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}
// x = hi + lo + r with hi, lo TF32 numbers and |r| <= 2^-23 |x| (both parts rounded to
// nearest, so the residuals carry no sign bias into long sums of squares)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = round_tf32(x);
  lo = round_tf32(__fsub_rn(x, hi));
}

// running double-float sum (h, l) += v
__device__ __forceinline__ void df_acc(float& h, float& l, float v) {
  const float s = __fadd_rn(h, v);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  const float t = __fadd_rn(l, e);
  h = __fadd_rn(s, t);
  l = __fsub_rn(t, __fsub_rn(h, s));
}

__global__ void __launch_bounds__(TC_THREADS, 1)
gram_tc_kernel(int64_t n, const float* __restrict__ X, int64_t ldx, int na, const float* __restrict__ Y,
               int64_t ldy, int nb, int64_t rows_per_split, int symmetric, double* __restrict__ part,
               int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ti = blockIdx.x, tj = blockIdx.y, s = blockIdx.z;
  const int i0 = ti * TC_M, j0 = tj * TC_N;
  // symmetric products need every entry with i <= j: skip tiles entirely below the diagonal
  if (symmetric && j0 + TC_N - 1 < i0) return;
  unsigned char* Ahi = smem;
  unsigned char* Alo = Ahi + TC_A_BYTES;
  unsigned char* Bhi = Alo + TC_A_BYTES;
  unsigned char* Blo = Bhi + TC_B_BYTES;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + TC_STAGE);  // MMAs of a step done
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(smem + TC_STAGE + 64);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  const unsigned idesc = make_idesc_tf32(TC_M, TC_N);

  const int64_t r0 = s * rows_per_split;
  const int64_t r1 = min(n, r0 + rows_per_split);
  const int nsteps = static_cast<int>((r1 - r0 + TC_KS - 1) / TC_KS);
  // this thread's slice of the accumulators: lane quarter (warp & 3), column half (warp >> 2)
  const int row_q = (warp & 3) * 32, col_h = (warp >> 2) * 32;
  const unsigned tslice = tmem + (static_cast<unsigned>(row_q) << 16) + col_h;
  float acc_h[32], acc_l[32], run[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc_h[c] = acc_l[c] = run[c] = 0.f;
  unsigned phase = 0u;
  bool ok = true;

  for (int t = 0; t < nsteps; ++t) {
    const int64_t rb = r0 + static_cast<int64_t>(t) * TC_KS;
    // X tile: 32 rows x 128 columns, one float4 per thread per pass
    for (int q = tid; q < TC_KS * (TC_M / 4); q += TC_THREADS) {
      const int k = q / (TC_M / 4), c4 = (q % (TC_M / 4)) * 4;
      const int64_t r = rb + k;
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (r < r1) {
        const float* src = X + r * ldx + i0 + c4;
        if (i0 + c4 + 3 < na) {
          const float4 f = *reinterpret_cast<const float4*>(src);
          v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = (i0 + c4 + u < na) ? src[u] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float h, l;
        split_tf32(v[u], h, l);
        const int o = kmajor_off(c4 + u, k);
        *reinterpret_cast<float*>(Ahi + o) = h;
        *reinterpret_cast<float*>(Alo + o) = l;
      }
    }
    // Y tile: 32 rows x 64 columns
    for (int q = tid; q < TC_KS * (TC_N / 4); q += TC_THREADS) {
      const int k = q / (TC_N / 4), c4 = (q % (TC_N / 4)) * 4;
      const int64_t r = rb + k;
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (r < r1) {
        const float* src = Y + r * ldy + j0 + c4;
        if (j0 + c4 + 3 < nb) {
          const float4 f = *reinterpret_cast<const float4*>(src);
          v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = (j0 + c4 + u < nb) ? src[u] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float h, l;
        split_tf32(v[u], h, l);
        const int o = kmajor_off(c4 + u, k);
        *reinterpret_cast<float*>(Bhi + o) = h;
        *reinterpret_cast<float*>(Blo + o) = l;
      }
    }
    // generic-proxy writes -> visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
      for (int kk = 0; kk < TC_KS / 8; ++kk) {
        const unsigned off = kk * 256;  // two core matrices of 128 bytes per MMA K = 8
        const unsigned long long dah = make_sdesc(ah + off, 128, 1024), dal = make_sdesc(al + off, 128, 1024);
        const unsigned long long dbh = make_sdesc(bh + off, 128, 1024), dbl = make_sdesc(bl + off, 128, 1024);
        // the leading products of each K slice into their own fresh accumulator, the two
        // cross products of the whole step into one more
        mma_tf32(tmem + kk * TC_N, dah, dbh, idesc, 0u);
        mma_tf32(tmem + 4 * TC_N, dah, dbl, idesc, kk > 0 ? 1u : 0u);
        mma_tf32(tmem + 4 * TC_N, dal, dbh, idesc, 1u);
      }
      mma_commit(bar);
    }
    ok = mbar_wait(bar, phase) && ok;
    phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float v[32], w[32];
    tmem_ld32(tslice, v);
#pragma unroll
    for (int a = 1; a <= 4; ++a) {
      tmem_ld32(tslice + a * TC_N, w);
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = __fadd_rn(v[c], w[c]);
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) run[c] = __fadd_rn(run[c], v[c]);
    if ((t % TC_FOLD) == TC_FOLD - 1 || t == nsteps - 1) {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        df_acc(acc_h[c], acc_l[c], run[c]);
        run[c] = 0.f;
      }
    }
    // every thread has read tensor memory and shared memory before they are overwritten
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok && lane == 0) atomicExch(err, 1);
  if (ok) {
    const int i = i0 + row_q + lane;
    if (i < na) {
      double* P = part + static_cast<size_t>(s) * na * nb + static_cast<size_t>(i) * nb;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int j = j0 + col_h + c;
        if (j < nb) P[j] = static_cast<double>(acc_h[c]) + static_cast<double>(acc_l[c]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace

int gram_tc_rows_align() { return TC_KS * TC_FOLD; }
int gram_tc_tile_m() { return TC_M; }
int gram_tc_tile_n() { return TC_N; }

bool gram_tc_supported(int64_t n, int64_t ldx, int64_t ldy, const void* X, const void* Y) {
  // 16-byte rows for the float4 staging loads
  return n > 0 && ldx % 4 == 0 && ldy % 4 == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0 &&
         (reinterpret_cast<uintptr_t>(Y) % 16) == 0;
}

arb_status gram_tc_launch(arb_ctx ctx, int64_t n, const float* X, int64_t ldx, int32_t na, const float* Y,
                          int64_t ldy, int32_t nb, int symmetric, double* part, int64_t nsplit, int64_t rows,
                          int* err_dev) {
  // a constant: concurrent contexts set the same value
  ARB_CUDA(ctx, cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  dim3 grid(static_cast<unsigned>((na + TC_M - 1) / TC_M), static_cast<unsigned>((nb + TC_N - 1) / TC_N),
            static_cast<unsigned>(nsplit));
  gram_tc_kernel<<<grid, TC_THREADS, TC_SMEM, ctx->stream>>>(n, X, ldx, na, Y, ldy, nb, rows, symmetric, part,
                                                              err_dev);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

}  // namespace arb
