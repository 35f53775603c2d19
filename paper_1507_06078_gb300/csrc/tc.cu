// Tensor-core (tcgen05) Gram products of FP32 blocks: part[s] = X^T Y over the rows of
// split s, the FP32 phase's Gram products (inner stop rule eq. inn-stop, orth(Z) and
// H = U^T A U of Algorithm 1).
//
// Split-TF32 ("3xTF32"): every FP32 operand x is cut into hi = x rounded to the nearest
// TF32 number and lo = the remainder x - hi rounded to TF32 (x = hi + lo to 2^-23), and
// x*y is formed as hi*hi + hi*lo + lo*hi by tcgen05.mma.kind::tf32 products.  The tensor
// core's FP32 accumulation in tensor memory does not round to nearest, and accumulating
// long runs there biases sums of squares by ~1e-6 relative (measured), so within every
// 32-row step each 16-row half gets its own fresh accumulator for hi*hi (two MMAs) and the
// cross terms (2^-11 smaller) share a third: the step's partial sums are read back, added
// in registers in FP32 (round to nearest) and folded every 256 rows into double-float sums.
//
// CTA tile: 128 columns of X (the MMA's M, tensor-memory lanes) x 64 columns of Y (N,
// tensor-memory columns), rows of the split in steps of 32.  Operands are staged by all
// 256 threads into shared memory in the canonical K-major layout without swizzling (core
// matrices of 8 rows x 16 bytes; LBO = 128 bytes between the two core matrices of one MMA's
// K = 8, SBO = 1024 bytes between 8-row groups).  Two shared-memory stages and two
// tensor-memory buffers form a software pipeline; one elected thread issues the MMAs and
// commits them to the buffer's mbarrier.  Every wait on an mbarrier is bounded; a wait that
// gives up sets the error word and the CTA stops issuing work.
#include <algorithm>

#include "arb_internal.h"

namespace arb {
namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;          // columns of X per CTA (MMA M)
constexpr int TC_N = 64;           // columns of Y per CTA (MMA N)
constexpr int TC_KS = 32;          // rows per pipeline step
constexpr int TC_FOLD = 8;         // steps (256 rows) per fold of the FP32 run sums into double-float
constexpr int TC_TMEM_COLS = 512;  // two buffers of 3 accumulators (2 leading-product slices, 1 cross) x 64 columns
constexpr int TC_A_BYTES = TC_M * TC_KS * 4;   // one operand copy (hi or lo) of the X tile
constexpr int TC_B_BYTES = TC_N * TC_KS * 4;
constexpr int TC_STAGE = 2 * TC_A_BYTES + 2 * TC_B_BYTES;  // hi, lo of both
constexpr int TC_NR = 4;                                   // raw (FP32) stages of rows in flight
// raw rows padded by 32 bytes so that a warp reading 8 columns x 4 rows hits 32 banks
constexpr int TC_RSA = TC_M + 8, TC_RSB = TC_N + 8;        // raw row strides (floats)
constexpr int TC_RAW_A = TC_KS * TC_RSA * 4;
constexpr int TC_RAW = TC_RAW_A + TC_KS * TC_RSB * 4;
constexpr int TC_SMEM = TC_NR * TC_RAW + 2 * TC_STAGE + 1024;  // raw ring, operand stages, barriers
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

__device__ __forceinline__ void mbar_expect_tx(void* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bulk copy (TMA, untiled) of `bytes` (a multiple of 16) from 16-byte aligned global memory
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, void* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Warp 0: request step u's rows into raw stage `raw` (row k of the X tile at k * TC_RSA
// floats, of the Y tile at TC_RAW_A + k * TC_RSB floats): one bulk copy per row and operand, issued by
// lane k, the columns of the tile rounded up to whole 16-byte groups (within the leading
// dimension).  Lane 0 posts the expected byte count first.
__device__ __forceinline__ void request_step(unsigned char* raw, void* bar, const float* X, int64_t ldx, int na,
                                             const float* Y, int64_t ldy, int nb, int64_t rb, int64_t r1, int i0,
                                             int j0, int lane) {
  const int ca = min(TC_M, na - i0), cb = min(TC_N, nb - j0);
  const unsigned sa = static_cast<unsigned>((ca + 3) / 4 * 16), sb = static_cast<unsigned>((cb + 3) / 4 * 16);
  const int rows = static_cast<int>(max(static_cast<int64_t>(0), min(static_cast<int64_t>(TC_KS), r1 - rb)));
  if (lane == 0) mbar_expect_tx(bar, static_cast<unsigned>(rows) * (sa + sb));
  __syncwarp();
  if (lane < rows) {
    bulk_g2s(raw + lane * (TC_RSA * 4), X + (rb + lane) * ldx + i0, sa, bar);
    bulk_g2s(raw + TC_RAW_A + lane * (TC_RSB * 4), Y + (rb + lane) * ldy + j0, sb, bar);
  }
}

// all threads: raw stage -> split-TF32 operand stage (K-major core-matrix layout); entries
// outside the rows or columns of the product are zero.  A warp converts one core-matrix
// group of 8 columns x 4 rows at a time, lane = 4 * column + row, so both its shared-memory
// reads (padded raw rows) and its writes (128 contiguous bytes) are free of bank conflicts.
__device__ __forceinline__ void split_step(const unsigned char* raw, unsigned char* stage, int rows, int ca, int cb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cl = lane >> 2, kl = lane & 3;
  unsigned char* Ahi = stage;
  unsigned char* Alo = Ahi + TC_A_BYTES;
  unsigned char* Bhi = Alo + TC_A_BYTES;
  unsigned char* Blo = Bhi + TC_B_BYTES;
  const float* ra = reinterpret_cast<const float*>(raw);
  const float* rbv = reinterpret_cast<const float*>(raw + TC_RAW_A);
  constexpr int KG = TC_KS / 4;
#pragma unroll 4
  for (int blk = warp; blk < (TC_M / 8) * KG; blk += TC_THREADS / 32) {
    const int c = (blk / KG) * 8 + cl, k = (blk % KG) * 4 + kl;
    const float x = (k < rows && c < ca) ? ra[k * TC_RSA + c] : 0.f;
    float h, l;
    split_tf32(x, h, l);
    const int o = kmajor_off(c, k);
    *reinterpret_cast<float*>(Ahi + o) = h;
    *reinterpret_cast<float*>(Alo + o) = l;
  }
#pragma unroll 4
  for (int blk = warp; blk < (TC_N / 8) * KG; blk += TC_THREADS / 32) {
    const int c = (blk / KG) * 8 + cl, k = (blk % KG) * 4 + kl;
    const float x = (k < rows && c < cb) ? rbv[k * TC_RSB + c] : 0.f;
    float h, l;
    split_tf32(x, h, l);
    const int o = kmajor_off(c, k);
    *reinterpret_cast<float*>(Bhi + o) = h;
    *reinterpret_cast<float*>(Blo + o) = l;
  }
}

// the MMAs of one step into tensor-memory buffer `dbase`: leading products of K rows 0-15
// into slice 0, of rows 16-31 into slice 1 (each slice two MMAs, fresh every step), all
// cross products into slice 2.  d[0..3]: descriptors of the stage's A hi, A lo, B hi, B lo
// at K = 0; the start-address field (bits 0-13, 16-byte units) advances by 16 per MMA K = 8.
__device__ __forceinline__ void issue_step(const unsigned long long (&d)[4], unsigned dbase, unsigned idesc) {
#pragma unroll
  for (int kk = 0; kk < TC_KS / 8; ++kk) {
    const unsigned long long o = 16ull * kk;
    mma_tf32(dbase + (kk >> 1) * TC_N, d[0] + o, d[2] + o, idesc, (kk & 1) ? 1u : 0u);
    mma_tf32(dbase + 2 * TC_N, d[0] + o, d[3] + o, idesc, kk > 0 ? 1u : 0u);
    mma_tf32(dbase + 2 * TC_N, d[1] + o, d[2] + o, idesc, 1u);
  }
}

// Pipeline over the 32-row steps, one CTA per SM: bulk copies keep TC_NR steps of raw rows
// in flight; at step t the threads split step t into operand stage t%2, thread 0 issues
// step t's MMAs into tensor-memory buffer t%2, warp 1 requests step t+TC_NR, and the
// threads add up buffer (t-1)%2 while those MMAs run.
__global__ void __launch_bounds__(TC_THREADS, 1)
gram_tc_kernel(int64_t n, const float* __restrict__ X, int64_t ldx, int na, const float* __restrict__ Y,
               int64_t ldy, int nb, int64_t rows_per_split, int symmetric, double* __restrict__ part,
               int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ti = blockIdx.x, tj = blockIdx.y, s = blockIdx.z;
  const int i0 = ti * TC_M, j0 = tj * TC_N;
  // symmetric products need every entry with i <= j: skip tiles entirely below the diagonal
  if (symmetric && j0 + TC_N - 1 < i0) return;
  unsigned char* raw = smem;                                   // TC_NR raw stages
  unsigned char* opnd = smem + TC_NR * TC_RAW;                 // 2 operand stages
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(opnd + 2 * TC_STAGE);
  unsigned long long* bar_raw = bars;                          // [TC_NR] rows landed
  unsigned long long* bar_mma = bars + TC_NR;                  // [2] MMAs of a buffer done
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + TC_NR + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < TC_NR + 2; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  const unsigned idesc = make_idesc_tf32(TC_M, TC_N);
  const unsigned dbuf[2] = {tmem, tmem + 3 * TC_N};
  unsigned long long sd[2][4];  // operand descriptors of the two stages (K = 0)
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const unsigned base = smem_u32(opnd + b * TC_STAGE);
    sd[b][0] = make_sdesc(base, 128, 1024);
    sd[b][1] = make_sdesc(base + TC_A_BYTES, 128, 1024);
    sd[b][2] = make_sdesc(base + 2 * TC_A_BYTES, 128, 1024);
    sd[b][3] = make_sdesc(base + 2 * TC_A_BYTES + TC_B_BYTES, 128, 1024);
  }

  const int64_t r0 = s * rows_per_split;
  const int64_t r1 = min(n, r0 + rows_per_split);
  const int nsteps = static_cast<int>((r1 - r0 + TC_KS - 1) / TC_KS);
  const int ca = min(TC_M, na - i0), cb = min(TC_N, nb - j0);
  // this thread's slice of the accumulators: lane quarter (warp & 3), column half (warp >> 2)
  const int row_q = (warp & 3) * 32, col_h = (warp >> 2) * 32;
  const unsigned tlane = (static_cast<unsigned>(row_q) << 16) + col_h;
  float acc_h[32], acc_l[32], run[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc_h[c] = acc_l[c] = run[c] = 0.f;
  unsigned ph_raw = 0u;   // bit q: parity to wait for on raw stage q
  unsigned ph_mma = 0u;   // bit b: parity to wait for on buffer b
  unsigned pend_raw = 0u, pend_mma = 0u;
  bool ok = true;

  if (warp == 0)
    for (int u = 0; u < TC_NR && u < nsteps; ++u)
      request_step(raw + u * TC_RAW, &bar_raw[u], X, ldx, na, Y, ldy, nb, r0 + static_cast<int64_t>(u) * TC_KS, r1,
                   i0, j0, lane);
  for (int u = 0; u < TC_NR && u < nsteps; ++u) pend_raw |= 1u << u;

  // add up tensor-memory buffer b (a finished step) into the running sums
  auto drain_buffer = [&](int b, bool fold) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float v[32], w[32];
    tmem_ld32(dbuf[b] + tlane, v);
#pragma unroll
    for (int a = 1; a <= 2; ++a) {
      tmem_ld32(dbuf[b] + tlane + a * TC_N, w);
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = __fadd_rn(v[c], w[c]);
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) run[c] = __fadd_rn(run[c], v[c]);
    if (fold) {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        df_acc(acc_h[c], acc_l[c], run[c]);
        run[c] = 0.f;
      }
    }
  };

  for (int t = 0; t < nsteps; ++t) {
    const int q = t % TC_NR, b = t & 1;
    const int64_t rb = r0 + static_cast<int64_t>(t) * TC_KS;
    const int rows = static_cast<int>(min(static_cast<int64_t>(TC_KS), r1 - rb));
    // rows of step t landed; operand stage b was read by the MMAs of step t-2, done
    ok = mbar_wait(&bar_raw[q], (ph_raw >> q) & 1u) && ok;
    ph_raw ^= 1u << q;
    pend_raw &= ~(1u << q);
    split_step(raw + q * TC_RAW, opnd + b * TC_STAGE, rows, ca, cb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue_step(sd[b], dbuf[b], idesc);
      mma_commit(&bar_mma[b]);
    }
    if (warp == 1 && t + TC_NR < nsteps)
      request_step(raw + q * TC_RAW, &bar_raw[q], X, ldx, na, Y, ldy, nb, r0 + static_cast<int64_t>(t + TC_NR) * TC_KS,
                   r1, i0, j0, lane);
    pend_mma |= 1u << b;
    if (t + TC_NR < nsteps) pend_raw |= 1u << q;
    if (t >= 1) {
      const int pb = b ^ 1;
      ok = mbar_wait(&bar_mma[pb], (ph_mma >> pb) & 1u) && ok;
      ph_mma ^= 1u << pb;
      pend_mma &= ~(1u << pb);
      drain_buffer(pb, ((t - 1) % TC_FOLD) == TC_FOLD - 1);
    }
  }
  if (ok && nsteps > 0) {
    const int lb = (nsteps - 1) & 1;
    ok = mbar_wait(&bar_mma[lb], (ph_mma >> lb) & 1u);
    ph_mma ^= 1u << lb;
    pend_mma &= ~(1u << lb);
    if (ok) drain_buffer(lb, true);
  }
  // after a failed wait: let whatever is still in flight finish before the memory goes
  for (int b = 0; b < 2; ++b)
    if ((pend_mma >> b) & 1u)
      if (!mbar_wait(&bar_mma[b], (ph_mma >> b) & 1u)) ok = false;
  for (int qq = 0; qq < TC_NR; ++qq)
    if ((pend_raw >> qq) & 1u)
      if (!mbar_wait(&bar_raw[qq], (ph_raw >> qq) & 1u)) ok = false;
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

// ---------------------------------------------------------------- tall-skinny products
// Out (n x nb) = alpha In (n x na) W (na x nb) + beta Out for FP32 blocks In, Out and a
// small FP64 matrix W: the FP32 phase's Ritz rotation X = U V (Algorithm 1), SVQB's map
// Z W_r Theta_r^{-1/2} and the block projections X - Q (Q^T X).  Split-TF32 as in the Gram
// product: hi*hi + hi*lo + lo*hi, three kind::tf32 MMAs per K = 8.  The tensor-memory
// accumulation does not round to nearest (summing all of na = 720 there left errors of
// ~1e-5 |result|, biased), so every K chunk of 16 gets a fresh accumulator (six MMAs) and
// the threads add the chunk sums in FP32 registers, rounding to nearest.
//
// CTA tile: 128 rows (MMA M) x up to 256 columns of Out (MMA N, rounded up to a multiple of
// 16); K in chunks of 16 through TG_S shared-memory stages and two tensor-memory buffers
// (chunk c into buffer c & 1, drained while chunk c + 1's MMAs run).  W is packed once per
// call (tg_pack_kernel) into per-chunk images of its split, transposed tile laid out exactly
// as a stage holds it (K-major core matrices without swizzle, LBO = 128 bytes, SBO = 512
// bytes), so one 32 KB bulk copy brings a chunk; two threads per row load the row's 16
// entries of In for the next chunk while the current one is in flight, split them and write
// them in the same layout.  Thread (warp w, lane l) owns row 32 (w % 4) + l of the tile
// (the tensor-memory lane quarter its warp may read) and columns 128 (w / 4) .. +127.
constexpr int TG_THREADS = 256;
constexpr int TG_M = 128;                                    // rows per CTA (MMA M)
constexpr int TG_N = 256;                                    // columns per CTA (MMA N at most)
constexpr int TG_KS = 16;                                    // K per chunk
constexpr int TG_S = 4;                                      // stages
constexpr int TG_A_BYTES = TG_M * TG_KS * 4;                 // hi or lo of the In tile: 8 KB
constexpr int TG_B_BYTES = TG_N * TG_KS * 4;                 // hi or lo of the W tile: 16 KB
constexpr int TG_STAGE = 2 * TG_A_BYTES + 2 * TG_B_BYTES;    // 48 KB
constexpr int TG_SMEM = TG_S * TG_STAGE + 1024;              // stages, barriers
constexpr int TG_CHUNK_FLOATS = 2 * TG_B_BYTES / 4;          // one packed chunk of W (hi, lo)

// byte offset of (row, k) in a K-major no-swizzle tile with TG_KS columns of K
__host__ __device__ constexpr int tg_off(int row, int k) {
  return (row >> 3) * 512 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// img[(t * nk + c) * TG_CHUNK_FLOATS + {0, TG_B_BYTES / 4} + tg_off(j, k) / 4] = split parts of
// W[16 c + k][256 t + j] as FP32 (zero outside na x nb)
__global__ void tg_pack_kernel(const double* __restrict__ W, int64_t ldw, int na, int nb, int nk, int ntiles,
                               float* __restrict__ img) {
  const int64_t total = static_cast<int64_t>(ntiles) * nk * TG_N * TG_KS;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(e % TG_KS);
    const int j = static_cast<int>((e / TG_KS) % TG_N);
    const int64_t tc = e / (TG_KS * TG_N);  // t * nk + c
    const int c = static_cast<int>(tc % nk), t = static_cast<int>(tc / nk);
    const int kg = c * TG_KS + k, jg = t * TG_N + j;
    const float x = (kg < na && jg < nb) ? static_cast<float>(W[static_cast<int64_t>(kg) * ldw + jg]) : 0.f;
    float h, l;
    split_tf32(x, h, l);
    float* chunk = img + tc * TG_CHUNK_FLOATS;
    chunk[tg_off(j, k) / 4] = h;
    chunk[TG_B_BYTES / 4 + tg_off(j, k) / 4] = l;
  }
}

// entries k0 .. k0 + 7 of a row of In (zero past na or n), k0 = 16 c + 8 (half)
__device__ __forceinline__ void tg_load_half(const float* __restrict__ In, int64_t ldi, int64_t row, int64_t n, int na,
                                             int c, int half, float (&a)[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) a[e] = 0.f;
  if (row >= n) return;
  const int k0 = c * TG_KS + 8 * half;
  const float* p = In + row * ldi + k0;
  const int kv = na - k0;  // valid entries from k0 (may be <= 0)
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    if (4 * g + 4 <= kv) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(p + 4 * g));
      a[4 * g] = v.x;
      a[4 * g + 1] = v.y;
      a[4 * g + 2] = v.z;
      a[4 * g + 3] = v.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * g + e < kv) a[4 * g + e] = p[4 * g + e];
    }
  }
}

__global__ void __launch_bounds__(TG_THREADS, 1)
gemm_tc_kernel(int64_t n, const float* __restrict__ In, int64_t ldi, int na, const float* __restrict__ img, int nk,
               int nb, float alpha, float beta, float* __restrict__ Out, int64_t ldo, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * TG_M;
  const int t_n = blockIdx.y, j0 = t_n * TG_N;
  const int nbt = min(TG_N, nb - j0);            // columns of this tile
  const int nmma = (nbt + 15) / 16 * 16;         // the MMA's N
  unsigned long long* bar_b = reinterpret_cast<unsigned long long*>(smem + TG_S * TG_STAGE);  // [TG_S]
  unsigned long long* bar_mma = bar_b + TG_S;                                                // [TG_S]
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(bar_mma + TG_S);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < 2 * TG_S; ++q) mbar_init(&bar_b[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  const unsigned idesc = make_idesc_tf32(TG_M, nmma);
  const float* img_t = img + static_cast<size_t>(t_n) * nk * TG_CHUNK_FLOATS;
  // this thread's accumulator slice and running sums
  const int q = warp & 3, ch = warp >> 2;
  const unsigned tl = (static_cast<unsigned>(q * 32) << 16) + static_cast<unsigned>(ch * 128);
  const int ngrp = max(0, min(4, (nbt - ch * 128 + 31) / 32));  // groups of 32 columns this thread holds
  float sum[128];
#pragma unroll
  for (int e = 0; e < 128; ++e) sum[e] = 0.f;
  // row half of In this thread stages: row tid / 2, entries 8 (tid % 2) .. +7 of each chunk
  const int arow = tid >> 1, ahalf = tid & 1;

  unsigned ph_mma = 0u, pend_mma = 0u;
  unsigned ph_b = 0u, pend_b = 0u;  // bulk copies of W: thread 0's bookkeeping only
  bool ok = true;
  float a[8];
  tg_load_half(In, ldi, r0 + arow, n, na, 0, ahalf, a);

  // add chunk cc's buffer into the running sums (its MMAs are complete)
  auto drain = [&](int cc) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned base = tmem + tl + static_cast<unsigned>((cc & 1) * TG_N);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g < ngrp) {  // warp-uniform
        float v[32];
        tmem_ld32(base + 32 * g, v);
#pragma unroll
        for (int e = 0; e < 32; ++e) sum[32 * g + e] = __fadd_rn(sum[32 * g + e], v[e]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  };

  for (int c = 0; c < nk; ++c) {
    const int s = c % TG_S;
    unsigned char* st = smem + s * TG_STAGE;
    // stage s was last read by chunk c - TG_S, whose MMAs every thread waited for when it
    // drained that chunk (at iteration c - TG_S + 1 <= c - 1)
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    if (tid == 0) {
      mbar_expect_tx(&bar_b[s], 2 * TG_B_BYTES);
      bulk_g2s(st + 2 * TG_A_BYTES, img_t + static_cast<size_t>(c) * TG_CHUNK_FLOATS, 2 * TG_B_BYTES, &bar_b[s]);
      pend_b |= 1u << s;
    }
    {
      float h[8], l[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) split_tf32(a[e], h[e], l[e]);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int o = tg_off(arow, 8 * ahalf + 4 * g);
        *reinterpret_cast<float4*>(st + o) = make_float4(h[4 * g], h[4 * g + 1], h[4 * g + 2], h[4 * g + 3]);
        *reinterpret_cast<float4*>(st + TG_A_BYTES + o) =
            make_float4(l[4 * g], l[4 * g + 1], l[4 * g + 2], l[4 * g + 3]);
      }
    }
    if (c + 1 < nk) tg_load_half(In, ldi, r0 + arow, n, na, c + 1, ahalf, a);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // also: buffer c & 1 was drained (chunk c - 2) by every thread
    if (tid == 0) {
      const bool got = mbar_wait(&bar_b[s], (ph_b >> s) & 1u);
      ok = got && ok;
      if (got) {
        ph_b ^= 1u << s;
        pend_b &= ~(1u << s);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned base = smem_u32(st);
        const unsigned long long dah = make_sdesc(base, 128, 512);
        const unsigned long long dal = make_sdesc(base + TG_A_BYTES, 128, 512);
        const unsigned long long dbh = make_sdesc(base + 2 * TG_A_BYTES, 128, 512);
        const unsigned long long dbl = make_sdesc(base + 2 * TG_A_BYTES + TG_B_BYTES, 128, 512);
        const unsigned d = tmem + static_cast<unsigned>((c & 1) * TG_N);
#pragma unroll
        for (int kk = 0; kk < TG_KS / 8; ++kk) {
          const unsigned long long o = 16ull * kk;  // 256 bytes = two core matrices along K
          mma_tf32(d, dah + o, dbh + o, idesc, kk > 0 ? 1u : 0u);
          mma_tf32(d, dah + o, dbl + o, idesc, 1u);
          mma_tf32(d, dal + o, dbh + o, idesc, 1u);
        }
      }
      mma_commit(&bar_mma[s]);  // also after a failed wait: the barrier then completes at once
    }
    pend_mma |= 1u << s;
    if (c >= 1) {  // drain chunk c - 1 while chunk c's MMAs run
      const int sp = (c - 1) % TG_S;
      if (mbar_wait(&bar_mma[sp], (ph_mma >> sp) & 1u)) {
        ph_mma ^= 1u << sp;
        pend_mma &= ~(1u << sp);
        drain(c - 1);
      } else {
        ok = false;  // left pending: the clean-up below waits for it again
      }
    }
  }
  if (ok && nk > 0) {
    const int sl = (nk - 1) % TG_S;
    if (mbar_wait(&bar_mma[sl], (ph_mma >> sl) & 1u)) {
      ph_mma ^= 1u << sl;
      pend_mma &= ~(1u << sl);
      drain(nk - 1);
    } else {
      ok = false;
    }
  }
  // after a failed wait: let whatever is still in flight finish before the memory goes
  for (int s = 0; s < TG_S; ++s)
    if ((pend_mma >> s) & 1u)
      if (!mbar_wait(&bar_mma[s], (ph_mma >> s) & 1u)) ok = false;
  if (tid == 0)
    for (int s = 0; s < TG_S; ++s)
      if ((pend_b >> s) & 1u)
        if (!mbar_wait(&bar_b[s], (ph_b >> s) & 1u)) ok = false;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && tid == 0) atomicExch(err, 1);
  if (ok) {
    const int64_t row = r0 + q * 32 + lane;
    if (row < n) {
      float* o = Out + row * ldo + j0 + ch * 128;
      const int nc = min(128, nbt - ch * 128);  // columns this thread writes (<= 0: none)
#pragma unroll
      for (int g = 0; g < 32; ++g) {
        const int c4 = 4 * g;
        if (c4 + 4 <= nc) {
          float4 r = make_float4(alpha * sum[c4], alpha * sum[c4 + 1], alpha * sum[c4 + 2], alpha * sum[c4 + 3]);
          if (beta != 0.f) {
            const float4 old = *reinterpret_cast<const float4*>(o + c4);
            r.x = fmaf(beta, old.x, r.x);
            r.y = fmaf(beta, old.y, r.y);
            r.z = fmaf(beta, old.z, r.z);
            r.w = fmaf(beta, old.w, r.w);
          }
          *reinterpret_cast<float4*>(o + c4) = r;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (c4 + e < nc) o[c4 + e] = beta != 0.f ? fmaf(beta, o[c4 + e], alpha * sum[c4 + e]) : alpha * sum[c4 + e];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
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

bool gemm_tc_supported(int64_t ldi, int64_t ldo, const void* In, const void* Out) {
  return ldi % 4 == 0 && ldo % 4 == 0 && (reinterpret_cast<uintptr_t>(In) % 16) == 0 &&
         (reinterpret_cast<uintptr_t>(Out) % 16) == 0;
}

arb_status gemm_tc_launch(arb_ctx ctx, int64_t n, const float* In, int64_t ldi, int32_t na, const double* W,
                          int64_t ldw, int32_t nb, float alpha, float beta, float* Out, int64_t ldo, float* img,
                          int* err_dev) {
  const int nk = (na + TG_KS - 1) / TG_KS, ntiles = (nb + TG_N - 1) / TG_N;
  const int64_t pack = static_cast<int64_t>(ntiles) * nk * TG_N * TG_KS;
  tg_pack_kernel<<<static_cast<unsigned>(std::min<int64_t>((pack + 255) / 256, 4096)), 256, 0, ctx->stream>>>(
      W, ldw, na, nb, nk, ntiles, img);
  ARB_LAUNCHED(ctx);
  ARB_CUDA(ctx, cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TG_SMEM));
  dim3 grid(static_cast<unsigned>((n + TG_M - 1) / TG_M), static_cast<unsigned>(ntiles));
  gemm_tc_kernel<<<grid, TG_THREADS, TG_SMEM, ctx->stream>>>(n, In, ldi, na, img, nk, nb, alpha, beta, Out, ldo,
                                                              err_dev);
  ARB_LAUNCHED(ctx);
  return ARB_OK;
}

size_t gemm_tc_image_floats(int32_t na, int32_t nb) {
  return static_cast<size_t>((nb + TG_N - 1) / TG_N) * ((na + TG_KS - 1) / TG_KS) * TG_CHUNK_FLOATS;
}

}  // namespace arb
