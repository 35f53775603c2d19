// Dense symmetric eigensolver for the projected Rayleigh-Ritz matrix H = U^T A U
// (Algorithm 1, step 3) and for the small Gram matrices of orth(Z) and of the inner stop
// rule: parallel two-sided cyclic Jacobi in FP64.
//
// Ordering: the round-robin ("circle") tournament on M = m rounded up to even indices.
// Each of the M-1 rounds of a sweep pairs every index exactly once, so the M/2 plane
// rotations of a round commute and are applied together: every 2x2 block A[P, Q] (P, Q
// pairs of the round) becomes J_P^T A[P, Q] J_Q, and every pair of columns of V is
// rotated.  Blocks are disjoint, so each is updated in place by one thread, which also
// writes the mirror block so that A stays exactly symmetric.  With an odd
// m, index m is a dummy whose rotations are the identity.
//
// One cooperative launch runs all sweeps; grid-wide barriers separate the rotation and
// update phases.  The off-diagonal norm is reduced deterministically (per-block partials
// summed in block order by every thread), so all threads take the same stop decision:
// stop when off(A) <= 1e-15 ||H||_F or after 60 sweeps.  The rotation of a pair (i, j)
// with a_ij != 0 uses theta = (a_jj - a_ii)/(2 a_ij), t = sign(theta)/(|theta| +
// sqrt(theta^2+1)), c = 1/sqrt(1+t^2), s = t c, which zeroes a_ij of J^T A J.
#include <cooperative_groups.h>

#include <algorithm>

#include "arb_internal.h"

namespace cg = cooperative_groups;

namespace arb {
namespace {

constexpr int JAC_THREADS = 256;
constexpr int JAC_MAX_SWEEPS = 60;
constexpr double JAC_TOL = 1e-15;

struct JacParams {
  int m, M;
  const double* H;
  int64_t ldh;
  double* A;     // M x M work copy
  double* V;     // M x M
  double2* rot;  // M/2 rotations (c, s) of the current round
  double* red;   // 2 * gridDim.x partials
  int32_t* perm; // m: sorted position of index i
  double* w_out;
  double* V_out;
  int64_t ldv;
  int32_t* sweeps_out;
};

__device__ __forceinline__ void round_pair(int M, int r, int k, int& i, int& j) {
  // players 1..M-1 sit at positions 0..M-2 and rotate by r; player 0 is fixed
  const int L = M - 1;
  if (k == 0) {
    i = 0;
    j = (r % L) + 1;
  } else {
    i = ((k + r) % L) + 1;
    j = ((M - 1 - k + r) % L) + 1;
  }
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
}

__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(JAC_THREADS) jacobi_kernel(JacParams P) {
  cg::grid_group g = cg::this_grid();
  __shared__ double sh[JAC_THREADS];
  const int m = P.m, M = P.M, half = M / 2;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nth = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t MM = static_cast<int64_t>(M) * M;

  // A = H (zero padded), V = I, ||H||_F^2 partials
  double fro = 0.0;
  for (int64_t t = tid; t < MM; t += nth) {
    const int i = static_cast<int>(t / M), j = static_cast<int>(t % M);
    const double v = (i < m && j < m) ? P.H[static_cast<int64_t>(i) * P.ldh + j] : 0.0;
    P.A[t] = v;
    P.V[t] = (i == j) ? 1.0 : 0.0;
    fro += v * v;
  }
  {
    const double b = block_sum(fro, sh);
    if (threadIdx.x == 0) P.red[blockIdx.x] = b;
  }
  g.sync();
  double normF2 = 0.0;
  for (int b = 0; b < static_cast<int>(gridDim.x); ++b) normF2 += P.red[b];
  const double normF = sqrt(normF2);
  g.sync();

  int sweep = 0;
  for (; sweep < JAC_MAX_SWEEPS; ++sweep) {
    double off = 0.0;
    for (int64_t t = tid; t < MM; t += nth) {
      const int i = static_cast<int>(t / M), j = static_cast<int>(t % M);
      if (i != j) off += P.A[t] * P.A[t];
    }
    {
      const double b = block_sum(off, sh);
      if (threadIdx.x == 0) P.red[gridDim.x + blockIdx.x] = b;
    }
    g.sync();
    double off2 = 0.0;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) off2 += P.red[gridDim.x + b];
    if (sqrt(off2) <= JAC_TOL * normF || normF == 0.0) break;
    for (int r = 0; r < M - 1; ++r) {
      for (int64_t k = tid; k < half; k += nth) {
        int i, j;
        round_pair(M, r, static_cast<int>(k), i, j);
        double c = 1.0, s = 0.0;
        const double aij = P.A[static_cast<int64_t>(i) * M + j];
        if (j < m && aij != 0.0) {
          const double theta = (P.A[static_cast<int64_t>(j) * M + j] - P.A[static_cast<int64_t>(i) * M + i]) / (2.0 * aij);
          const double sg = theta >= 0.0 ? 1.0 : -1.0;
          const double t = sg / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        P.rot[k] = make_double2(c, s);
      }
      g.sync();
      const int64_t nblk = static_cast<int64_t>(half) * half;
      const int64_t total = nblk + static_cast<int64_t>(M) * half;
      for (int64_t it = tid; it < total; it += nth) {
        if (it < nblk) {
          const int kp = static_cast<int>(it / half), kq = static_cast<int>(it % half);
          if (kp > kq) continue;  // the mirror block is written by the (kq, kp) thread
          int i1, j1, i2, j2;
          round_pair(M, r, kp, i1, j1);
          round_pair(M, r, kq, i2, j2);
          const double2 r1 = P.rot[kp], r2 = P.rot[kq];
          double* p_a = P.A + static_cast<int64_t>(i1) * M + i2;
          double* p_b = P.A + static_cast<int64_t>(i1) * M + j2;
          double* p_c = P.A + static_cast<int64_t>(j1) * M + i2;
          double* p_d = P.A + static_cast<int64_t>(j1) * M + j2;
          const double a = *p_a, b = *p_b, cc = *p_c, d = *p_d;
          // rows: J_P^T
          const double ra0 = r1.x * a - r1.y * cc, ra1 = r1.x * b - r1.y * d;
          const double rb0 = r1.y * a + r1.x * cc, rb1 = r1.y * b + r1.x * d;
          // columns: J_Q
          double na = r2.x * ra0 - r2.y * ra1, nb = r2.y * ra0 + r2.x * ra1;
          double nc = r2.x * rb0 - r2.y * rb1, nd = r2.y * rb0 + r2.x * rb1;
          if (kp == kq && r1.y != 0.0) {
            nb = 0.0;  // the rotation annihilates the pivot entry
            nc = 0.0;
          }
          *p_a = na;
          *p_b = nb;
          *p_c = nc;
          *p_d = nd;
          if (kp != kq) {  // keep A exactly symmetric
            P.A[static_cast<int64_t>(i2) * M + i1] = na;
            P.A[static_cast<int64_t>(j2) * M + i1] = nb;
            P.A[static_cast<int64_t>(i2) * M + j1] = nc;
            P.A[static_cast<int64_t>(j2) * M + j1] = nd;
          }
        } else {
          const int64_t it2 = it - nblk;
          const int row = static_cast<int>(it2 / half), kp = static_cast<int>(it2 % half);
          int i, j;
          round_pair(M, r, kp, i, j);
          const double2 rr = P.rot[kp];
          if (rr.y != 0.0) {
            double* vi = P.V + static_cast<int64_t>(row) * M + i;
            double* vj = P.V + static_cast<int64_t>(row) * M + j;
            const double x = *vi, y = *vj;
            *vi = rr.x * x - rr.y * y;
            *vj = rr.y * x + rr.x * y;
          }
        }
      }
      g.sync();
    }
  }
  // sort eigenvalues descending (stable by index) and write outputs
  for (int64_t i = tid; i < m; i += nth) {
    const double vi = P.A[i * M + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double vj = P.A[static_cast<int64_t>(j) * M + j];
      rank += (vj > vi) || (vj == vi && j < i);
    }
    P.perm[i] = rank;
    P.w_out[rank] = vi;
  }
  g.sync();
  for (int64_t t = tid; t < static_cast<int64_t>(m) * m; t += nth) {
    const int row = static_cast<int>(t / m), i = static_cast<int>(t % m);
    P.V_out[static_cast<int64_t>(row) * P.ldv + P.perm[i]] = P.V[static_cast<int64_t>(row) * M + i];
  }
  if (tid == 0 && P.sweeps_out) *P.sweeps_out = sweep;
}

// The same method for M <= JAC_SMALL_M in one CTA: A and V live in shared memory and the
// phase barriers are __syncthreads (no grid-wide barrier latency).
constexpr int JAC_SMALL_M = 96;
constexpr int JAC_SMALL_THREADS = 512;

__global__ void __launch_bounds__(JAC_SMALL_THREADS) jacobi_small_kernel(JacParams P) {
  extern __shared__ double smem[];
  const int m = P.m, M = P.M, half = M / 2;
  double* A = smem;
  double* V = smem + M * M;
  double2* rot = reinterpret_cast<double2*>(V + M * M);
  double* red = reinterpret_cast<double*>(rot + half);  // JAC_SMALL_THREADS
  const int tid = threadIdx.x, nth = blockDim.x;
  double fro = 0.0;
  for (int t = tid; t < M * M; t += nth) {
    const int i = t / M, j = t % M;
    const double v = (i < m && j < m) ? P.H[static_cast<int64_t>(i) * P.ldh + j] : 0.0;
    A[t] = v;
    V[t] = (i == j) ? 1.0 : 0.0;
    fro += v * v;
  }
  const double normF = sqrt(block_sum(fro, red));
  int sweep = 0;
  for (; sweep < JAC_MAX_SWEEPS; ++sweep) {
    double off = 0.0;
    for (int t = tid; t < M * M; t += nth)
      if (t / M != t % M) off += A[t] * A[t];
    const double off2 = block_sum(off, red);
    if (sqrt(off2) <= JAC_TOL * normF || normF == 0.0) break;
    for (int r = 0; r < M - 1; ++r) {
      for (int k = tid; k < half; k += nth) {
        int i, j;
        round_pair(M, r, k, i, j);
        double c = 1.0, s = 0.0;
        const double aij = A[i * M + j];
        if (j < m && aij != 0.0) {
          const double theta = (A[j * M + j] - A[i * M + i]) / (2.0 * aij);
          const double sg = theta >= 0.0 ? 1.0 : -1.0;
          const double t = sg / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        rot[k] = make_double2(c, s);
      }
      __syncthreads();
      const int nblk = half * half;
      for (int it = tid; it < nblk + M * half; it += nth) {
        if (it < nblk) {
          const int kp = it / half, kq = it % half;
          if (kp > kq) continue;
          int i1, j1, i2, j2;
          round_pair(M, r, kp, i1, j1);
          round_pair(M, r, kq, i2, j2);
          const double2 r1 = rot[kp], r2 = rot[kq];
          const double a = A[i1 * M + i2], b = A[i1 * M + j2], cc = A[j1 * M + i2], d = A[j1 * M + j2];
          const double ra0 = r1.x * a - r1.y * cc, ra1 = r1.x * b - r1.y * d;
          const double rb0 = r1.y * a + r1.x * cc, rb1 = r1.y * b + r1.x * d;
          double na = r2.x * ra0 - r2.y * ra1, nb = r2.y * ra0 + r2.x * ra1;
          double nc = r2.x * rb0 - r2.y * rb1, nd = r2.y * rb0 + r2.x * rb1;
          if (kp == kq && r1.y != 0.0) {
            nb = 0.0;
            nc = 0.0;
          }
          A[i1 * M + i2] = na;
          A[i1 * M + j2] = nb;
          A[j1 * M + i2] = nc;
          A[j1 * M + j2] = nd;
          if (kp != kq) {
            A[i2 * M + i1] = na;
            A[j2 * M + i1] = nb;
            A[i2 * M + j1] = nc;
            A[j2 * M + j1] = nd;
          }
        } else {
          const int it2 = it - nblk;
          const int row = it2 / half, kp = it2 % half;
          int i, j;
          round_pair(M, r, kp, i, j);
          const double2 rr = rot[kp];
          if (rr.y != 0.0) {
            const double x = V[row * M + i], y = V[row * M + j];
            V[row * M + i] = rr.x * x - rr.y * y;
            V[row * M + j] = rr.y * x + rr.x * y;
          }
        }
      }
      __syncthreads();
    }
  }
  int* perm = reinterpret_cast<int*>(red);  // red is free now
  __syncthreads();
  for (int i = tid; i < m; i += nth) {
    const double vi = A[i * M + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double vj = A[j * M + j];
      rank += (vj > vi) || (vj == vi && j < i);
    }
    perm[i] = rank;
    P.w_out[rank] = vi;
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += nth) {
    const int row = t / m, i = t % m;
    P.V_out[static_cast<int64_t>(row) * P.ldv + perm[i]] = V[row * M + i];
  }
  if (tid == 0 && P.sweeps_out) *P.sweeps_out = sweep;
}

}  // namespace

arb_status syevj(arb_ctx ctx, int32_t m, const double* H, int64_t ldh, double* w, double* V,
                 int64_t ldv, int32_t* sweeps) {
  if (m <= 0) {
    if (sweeps) *sweeps = 0;
    return ARB_OK;
  }
  if (m > 8192) return set_error(ctx, ARB_INVALID_ARG, "syevj: matrix too large");
  const int M = (m % 2 == 0) ? m : m + 1;
  const int half = M / 2;
  if (M <= JAC_SMALL_M) {
    const size_t smem = (2 * static_cast<size_t>(M) * M + 2 * half + JAC_SMALL_THREADS) * sizeof(double);
    int32_t* sw;
    ARB_TRY(ws<int32_t>(ctx, WS_JACOBI, 4, &sw));
    ARB_CUDA(ctx, cudaFuncSetAttribute(jacobi_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem)));
    JacParams P = {};
    P.m = m;
    P.M = M;
    P.H = H;
    P.ldh = ldh;
    P.w_out = w;
    P.V_out = V;
    P.ldv = ldv;
    P.sweeps_out = sw;
    jacobi_small_kernel<<<1, JAC_SMALL_THREADS, smem, ctx->stream>>>(P);
    ARB_LAUNCHED(ctx);
    if (sweeps) ARB_TRY(d2h_sync(ctx, sweeps, sw, sizeof(int32_t)));
    return ARB_OK;
  }
  if (ctx->jacobi_max_blocks == 0) {
    int per_sm = 0;
    ARB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, JAC_THREADS, 0));
    ctx->jacobi_max_blocks = std::max(1, per_sm) * ctx->num_sms;
  }
  const int64_t work = static_cast<int64_t>(half) * half + static_cast<int64_t>(M) * half;
  int grid = static_cast<int>(std::min<int64_t>((work + JAC_THREADS * 4 - 1) / (JAC_THREADS * 4),
                                                static_cast<int64_t>(ctx->num_sms) * 2));
  grid = std::max(1, std::min(grid, ctx->jacobi_max_blocks));
  // scratch: A, V (M x M), rotations, reductions, permutation, sweep count
  const size_t mm = static_cast<size_t>(M) * M;
  double* base;
  ARB_TRY(ws<double>(ctx, WS_JACOBI, 2 * mm + 2 * half + 2 * static_cast<size_t>(grid) + m + 8, &base));
  JacParams P;
  P.m = m;
  P.M = M;
  P.H = H;
  P.ldh = ldh;
  P.A = base;
  P.V = base + mm;
  P.rot = reinterpret_cast<double2*>(base + 2 * mm);
  P.red = base + 2 * mm + 2 * half;
  P.perm = reinterpret_cast<int32_t*>(P.red + 2 * grid);
  P.w_out = w;
  P.V_out = V;
  P.ldv = ldv;
  P.sweeps_out = reinterpret_cast<int32_t*>(P.red + 2 * grid + m + 2);
  void* args[] = {&P};
  ARB_CUDA(ctx, cudaLaunchCooperativeKernel(reinterpret_cast<void*>(jacobi_kernel), dim3(grid),
                                            dim3(JAC_THREADS), args, 0, ctx->stream));
  ARB_LAUNCHED(ctx);
  if (sweeps) ARB_TRY(d2h_sync(ctx, sweeps, P.sweeps_out, sizeof(int32_t)));
  return ARB_OK;
}

}  // namespace arb
