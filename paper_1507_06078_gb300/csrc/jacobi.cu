// Dense symmetric eigensolver for the projected Rayleigh-Ritz matrix H = U^T A U
// (Algorithm 1, step 3) and for the small Gram matrices of orth(Z) and of the inner stop
// rule: parallel two-sided cyclic Jacobi in FP64.
//
// Every rotation of the (i, j) plane with a_ij != 0 uses theta = (a_jj - a_ii)/(2 a_ij),
// t = sign(theta)/(|theta| + sqrt(theta^2+1)), c = 1/sqrt(1+t^2), s = t c, which zeroes
// a_ij of J^T A J.  Rotations are scheduled by the round-robin ("circle") tournament: each
// of the N-1 rounds pairs every one of N indices exactly once, so the rotations of a round
// commute and are applied together.  Sweeps stop when off(A) <= tol ||H||_F (1e-15 for
// FP64 data; callers whose matrices carry FP32-level errors pass 1e-10) or after 60.
//
// m <= ARB_JAC_ONE_CTA_M (32; the kernel holds up to 96): one CTA holds A and V in shared
// memory and rotates single indices.
// Above: block Jacobi.  The indices are cut into NB blocks of 16 (NB even; padding
// indices have zero rows and columns, so no rotation ever couples them to real ones).  A
// round of the tournament on the NB blocks pairs blocks (I, J); for each pair the 32 x 32
// subproblem A[I+J, I+J] gets one cyclic Jacobi sweep in shared memory, accumulating the
// orthogonal Q_p (phase 1).  Then (phase 2) every block of A is transformed,
// A[P, P'] <- Q_p^T A[P, P'] Q_p', and V[:, P] <- V[:, P] Q_p.  Both phases are split over
// the CTAs of one cooperative launch with two grid barriers per round, 2 (NB - 1) per
// sweep instead of 2 (m - 1) for index-by-index rounds.  The off-diagonal norm is reduced
// deterministically (per-CTA partials summed in CTA order by every thread), so all
// threads take the same stop decision.
#include <cooperative_groups.h>

#include <algorithm>

#include "arb_internal.h"
#include "df_arith.cuh"

namespace cg = cooperative_groups;

namespace arb {
namespace {

constexpr int JAC_THREADS = 256;
constexpr int JAC_MAX_SWEEPS = 60;

struct JacParams {
  int m, M;
  const double* H;
  int64_t ldh;
  double* A;     // M x M work copy
  double* V;     // M x M
  double* red;   // 2 * gridDim.x partials
  int32_t* perm; // m: sorted position of index i
  double* w_out;
  double* V_out;
  int64_t ldv;
  int32_t* sweeps_out;
  double* Q;     // block kernel: NB/2 orthogonal 32 x 32 factors of the current round
  double tol;    // stop when off(A) <= tol ||H||_F
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

__device__ __forceinline__ double2 jacobi_rotation(double aii, double ajj, double aij) {
  if (aij == 0.0) return make_double2(1.0, 0.0);
  const double theta = (ajj - aii) / (2.0 * aij);
  const double sg = theta >= 0.0 ? 1.0 : -1.0;
  const double t = sg / (fabs(theta) + sqrt(theta * theta + 1.0));
  const double c = 1.0 / sqrt(t * t + 1.0);
  return make_double2(c, t * c);
}

constexpr int BJ_B = 16;          // index block
constexpr int BJ_S = 2 * BJ_B;    // subproblem order
constexpr int BJ_LD = BJ_S + 1;   // shared-memory row pitch (bank spread)

// global index of local index x (< 32) of block pair (I, J)
__device__ __forceinline__ int bj_index(int I, int J, int x) {
  return x < BJ_B ? I * BJ_B + x : J * BJ_B + (x - BJ_B);
}

struct BJShared {
  double S[BJ_S * BJ_LD];   // subproblem / block of A or V
  double Qa[BJ_S * BJ_LD];
  double Qb[BJ_S * BJ_LD];
  double X[BJ_S * BJ_LD];
  double2 rot[BJ_B];
  double red[JAC_THREADS];
};

// One cyclic sweep (31 rounds of 16 rotations) on the 32 x 32 matrix in sh.S, accumulating
// the rotations into sh.Qa (initially I).
__device__ void bj_inner_sweep(BJShared& sh) {
  const int tid = threadIdx.x;
  for (int r = 0; r < BJ_S - 1; ++r) {
    if (tid < BJ_B) {
      int i, j;
      round_pair(BJ_S, r, tid, i, j);
      sh.rot[tid] = jacobi_rotation(sh.S[i * BJ_LD + i], sh.S[j * BJ_LD + j], sh.S[i * BJ_LD + j]);
    }
    __syncthreads();
    constexpr int nblk = BJ_B * BJ_B;
    for (int it = tid; it < nblk + BJ_S * BJ_B; it += blockDim.x) {
      if (it < nblk) {
        const int kp = it / BJ_B, kq = it % BJ_B;
        if (kp > kq) continue;  // the (kq, kp) thread's mirror
        int i1, j1, i2, j2;
        round_pair(BJ_S, r, kp, i1, j1);
        round_pair(BJ_S, r, kq, i2, j2);
        const double2 r1 = sh.rot[kp], r2 = sh.rot[kq];
        const double a = sh.S[i1 * BJ_LD + i2], b = sh.S[i1 * BJ_LD + j2];
        const double cc = sh.S[j1 * BJ_LD + i2], d = sh.S[j1 * BJ_LD + j2];
        const double ra0 = r1.x * a - r1.y * cc, ra1 = r1.x * b - r1.y * d;
        const double rb0 = r1.y * a + r1.x * cc, rb1 = r1.y * b + r1.x * d;
        double na = r2.x * ra0 - r2.y * ra1, nb = r2.y * ra0 + r2.x * ra1;
        double nc = r2.x * rb0 - r2.y * rb1, nd = r2.y * rb0 + r2.x * rb1;
        if (kp == kq && r1.y != 0.0) {
          nb = 0.0;
          nc = 0.0;
        }
        sh.S[i1 * BJ_LD + i2] = na;
        sh.S[i1 * BJ_LD + j2] = nb;
        sh.S[j1 * BJ_LD + i2] = nc;
        sh.S[j1 * BJ_LD + j2] = nd;
        if (kp != kq) {
          sh.S[i2 * BJ_LD + i1] = na;
          sh.S[j2 * BJ_LD + i1] = nb;
          sh.S[i2 * BJ_LD + j1] = nc;
          sh.S[j2 * BJ_LD + j1] = nd;
        }
      } else {
        const int it2 = it - nblk;
        const int row = it2 / BJ_B, kp = it2 % BJ_B;
        int i, j;
        round_pair(BJ_S, r, kp, i, j);
        const double2 rr = sh.rot[kp];
        if (rr.y != 0.0) {
          const double x = sh.Qa[row * BJ_LD + i], y = sh.Qa[row * BJ_LD + j];
          sh.Qa[row * BJ_LD + i] = rr.x * x - rr.y * y;
          sh.Qa[row * BJ_LD + j] = rr.y * x + rr.x * y;
        }
      }
    }
    __syncthreads();
  }
}

// out (32 x 32, pitch BJ_LD) = L^T R (transL) or L R; 256 threads, 4 outputs each
__device__ __forceinline__ void bj_matmul(const double* L, const double* R, double* out, bool transL) {
  const int z = threadIdx.x / 8, y0 = (threadIdx.x % 8) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
  for (int x = 0; x < BJ_S; ++x) {
    const double l = transL ? L[x * BJ_LD + z] : L[z * BJ_LD + x];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = fma(l, R[x * BJ_LD + y0 + u], acc[u]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) out[z * BJ_LD + y0 + u] = acc[u];
}

__global__ void __launch_bounds__(JAC_THREADS) jacobi_block_kernel(JacParams P) {
  cg::grid_group g = cg::this_grid();
  __shared__ BJShared sh;
  const int m = P.m, M = P.M, NB = M / BJ_B, npairs = NB / 2;
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
    const double b = block_sum(fro, sh.red);
    if (threadIdx.x == 0) P.red[blockIdx.x] = b;
  }
  g.sync();
  double normF2 = 0.0;
  for (int b = 0; b < static_cast<int>(gridDim.x); ++b) normF2 += P.red[b];
  const double normF = sqrt(normF2);
  g.sync();

  const int nA = npairs * (npairs + 1) / 2;        // blocks (p <= p') of A
  const int nV = (M / BJ_S) * npairs;              // 32-row chunks of V x pairs
  int sweep = 0;
  for (; sweep < JAC_MAX_SWEEPS; ++sweep) {
    double off = 0.0;
    for (int64_t t = tid; t < MM; t += nth) {
      const int i = static_cast<int>(t / M), j = static_cast<int>(t % M);
      if (i != j) off += P.A[t] * P.A[t];
    }
    {
      const double b = block_sum(off, sh.red);
      if (threadIdx.x == 0) P.red[gridDim.x + blockIdx.x] = b;
    }
    g.sync();
    double off2 = 0.0;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) off2 += P.red[gridDim.x + b];
    if (sqrt(off2) <= P.tol * normF || normF == 0.0) break;
    for (int r = 0; r < NB - 1; ++r) {
      // phase 1: one Jacobi sweep per block-pair subproblem -> Q_p
      for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
        int I, J;
        round_pair(NB, r, p, I, J);
        for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
          const int x = t / BJ_S, y = t % BJ_S;
          sh.S[x * BJ_LD + y] = P.A[static_cast<int64_t>(bj_index(I, J, x)) * M + bj_index(I, J, y)];
          sh.Qa[x * BJ_LD + y] = (x == y) ? 1.0 : 0.0;
        }
        __syncthreads();
        bj_inner_sweep(sh);
        double* Qp = P.Q + static_cast<size_t>(p) * BJ_S * BJ_S;
        for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x)
          Qp[t] = sh.Qa[(t / BJ_S) * BJ_LD + (t % BJ_S)];
        __syncthreads();
      }
      g.sync();
      // phase 2: A[P, P'] <- Q_p^T A[P, P'] Q_p' (p <= p', mirrored) and V[:, P] <- V[:, P] Q_p
      for (int task = blockIdx.x; task < nA + nV; task += gridDim.x) {
        if (task < nA) {
          int p = 0, rem = task;
          while (rem >= npairs - p) {
            rem -= npairs - p;
            ++p;
          }
          const int pp = p + rem;
          int I1, J1, I2, J2;
          round_pair(NB, r, p, I1, J1);
          round_pair(NB, r, pp, I2, J2);
          const double* Q1 = P.Q + static_cast<size_t>(p) * BJ_S * BJ_S;
          const double* Q2 = P.Q + static_cast<size_t>(pp) * BJ_S * BJ_S;
          for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
            const int x = t / BJ_S, y = t % BJ_S;
            sh.S[x * BJ_LD + y] = P.A[static_cast<int64_t>(bj_index(I1, J1, x)) * M + bj_index(I2, J2, y)];
            sh.Qa[x * BJ_LD + y] = Q1[t];
            sh.Qb[x * BJ_LD + y] = Q2[t];
          }
          __syncthreads();
          bj_matmul(sh.Qa, sh.S, sh.X, true);   // X = Q_p^T A[P, P']
          __syncthreads();
          bj_matmul(sh.X, sh.Qb, sh.S, false);  // S = X Q_p'
          __syncthreads();
          for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
            const int z = t / BJ_S, w = t % BJ_S;
            const int64_t gz = bj_index(I1, J1, z), gw = bj_index(I2, J2, w);
            if (p != pp) {
              const double v = sh.S[z * BJ_LD + w];
              P.A[gz * M + gw] = v;
              P.A[gw * M + gz] = v;
            } else if (z <= w) {  // diagonal block: the upper triangle, mirrored (exact symmetry)
              const double v = sh.S[z * BJ_LD + w];
              P.A[gz * M + gw] = v;
              P.A[gw * M + gz] = v;
            }
          }
          __syncthreads();
        } else {
          const int t2 = task - nA;
          const int chunk = t2 / npairs, p = t2 % npairs;
          int I, J;
          round_pair(NB, r, p, I, J);
          const double* Qp = P.Q + static_cast<size_t>(p) * BJ_S * BJ_S;
          for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
            const int x = t / BJ_S, y = t % BJ_S;
            sh.S[x * BJ_LD + y] = P.V[static_cast<int64_t>(chunk * BJ_S + x) * M + bj_index(I, J, y)];
            sh.Qa[x * BJ_LD + y] = Qp[t];
          }
          __syncthreads();
          bj_matmul(sh.S, sh.Qa, sh.X, false);  // X = V[rows, P] Q_p
          __syncthreads();
          for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
            const int x = t / BJ_S, y = t % BJ_S;
            P.V[static_cast<int64_t>(chunk * BJ_S + x) * M + bj_index(I, J, y)] = sh.X[x * BJ_LD + y];
          }
          __syncthreads();
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
    if (sqrt(off2) <= P.tol * normF || normF == 0.0) break;
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

// ---------------------------------------------------------------- double-float block Jacobi
// The block method above with its arithmetic on GB300's FP32 pipe: the pair subproblems and
// their orthogonal factors are held in double-float (hi + lo FP32) in shared memory, every
// rotation update and every block product is a compensated (Dot2) sum of double-float
// products, and A and V stay FP64 in global memory (split on load, hi + lo on store).  The
// rotation angles themselves are computed in FP64 from the current entries.  Each update
// carries about 2^-44 relative error, so sweeps stop at off(A) <= max(tol, 1e-13) ||H||_F.
struct DFShared {
  float Sh[BJ_S * BJ_LD], Sl[BJ_S * BJ_LD];   // subproblem / block of A or V
  float Ah[BJ_S * BJ_LD], Al[BJ_S * BJ_LD];   // Q_p (phase 1 accumulation / phase 2 left factor)
  float Bh[BJ_S * BJ_LD], Bl[BJ_S * BJ_LD];   // Q_p' (phase 2 right factor)
  float Xh[BJ_S * BJ_LD], Xl[BJ_S * BJ_LD];   // phase 2 intermediate
  float rot[BJ_B][4];                          // c_hi, c_lo, s_hi, s_lo
  double red[JAC_THREADS];
};

// (c1 x1 + c2 x2) for two lanes at once, compensated
__device__ __forceinline__ dfp dot2_two(const dfp& c1, const dfp& x1, const dfp& c2, const dfp& x2) {
  float2 S = make_float2(0.f, 0.f), E = make_float2(0.f, 0.f);
  dot2p(S, E, c1, neg(c1), x1);
  dot2p(S, E, c2, neg(c2), x2);
  return fast_two_sum2(S, E);
}
__device__ __forceinline__ dfp bcast(float h, float l) { return dfp{make_float2(h, h), make_float2(l, l)}; }
__device__ __forceinline__ dfp pair_of(float h0, float l0, float h1, float l1) {
  return dfp{make_float2(h0, h1), make_float2(l0, l1)};
}

// one cyclic sweep on the 32 x 32 double-float matrix (Sh, Sl), accumulating into (Ah, Al)
__device__ __forceinline__ void dfj_inner_sweep(DFShared& sh) {
  const int tid = threadIdx.x;
  for (int r = 0; r < BJ_S - 1; ++r) {
    if (tid < BJ_B) {
      int i, j;
      round_pair(BJ_S, r, tid, i, j);
      const double aii = static_cast<double>(sh.Sh[i * BJ_LD + i]) + sh.Sl[i * BJ_LD + i];
      const double ajj = static_cast<double>(sh.Sh[j * BJ_LD + j]) + sh.Sl[j * BJ_LD + j];
      const double aij = static_cast<double>(sh.Sh[i * BJ_LD + j]) + sh.Sl[i * BJ_LD + j];
      const double2 cs = jacobi_rotation(aii, ajj, aij);
      split_f64(cs.x, sh.rot[tid][0], sh.rot[tid][1]);
      split_f64(cs.y, sh.rot[tid][2], sh.rot[tid][3]);
    }
    __syncthreads();
    constexpr int nblk = BJ_B * BJ_B;
    for (int it = tid; it < nblk + BJ_S * BJ_B; it += blockDim.x) {
      if (it < nblk) {
        const int kp = it / BJ_B, kq = it % BJ_B;
        if (kp > kq) continue;
        int i1, j1, i2, j2;
        round_pair(BJ_S, r, kp, i1, j1);
        round_pair(BJ_S, r, kq, i2, j2);
        const float* r1 = sh.rot[kp];
        const float* r2 = sh.rot[kq];
        const bool pivot = (kp == kq) && (r1[2] != 0.f || r1[3] != 0.f);
        // rows: (a b; cc d) -> J_P^T (a b; cc d), both columns of the pair at once
        const dfp ab = pair_of(sh.Sh[i1 * BJ_LD + i2], sh.Sl[i1 * BJ_LD + i2], sh.Sh[i1 * BJ_LD + j2],
                               sh.Sl[i1 * BJ_LD + j2]);
        const dfp cd = pair_of(sh.Sh[j1 * BJ_LD + i2], sh.Sl[j1 * BJ_LD + i2], sh.Sh[j1 * BJ_LD + j2],
                               sh.Sl[j1 * BJ_LD + j2]);
        const dfp c1 = bcast(r1[0], r1[1]), s1 = bcast(r1[2], r1[3]);
        const dfp ra = dot2_two(c1, ab, neg(s1), cd);  // (ra0, ra1) = c1 (a, b) - s1 (cc, d)
        const dfp rb = dot2_two(s1, ab, c1, cd);       // (rb0, rb1) = s1 (a, b) + c1 (cc, d)
        // columns: (x0 x1) -> (c2 x0 - s2 x1, s2 x0 + c2 x1) for x = ra and x = rb
        const dfp c2s2 = pair_of(r2[0], r2[1], r2[2], r2[3]);
        const dfp ms2c2 = dfp{make_float2(-r2[2], r2[0]), make_float2(-r2[3], r2[1])};
        const dfp ra0 = bcast(ra.hi.x, ra.lo.x), ra1 = bcast(ra.hi.y, ra.lo.y);
        const dfp rb0 = bcast(rb.hi.x, rb.lo.x), rb1 = bcast(rb.hi.y, rb.lo.y);
        const dfp nab = dot2_two(c2s2, ra0, ms2c2, ra1);  // (na, nb)
        const dfp ncd = dot2_two(c2s2, rb0, ms2c2, rb1);  // (nc, nd)
        float nbh = nab.hi.y, nbl = nab.lo.y, nch = ncd.hi.x, ncl = ncd.lo.x;
        if (pivot) nbh = nbl = nch = ncl = 0.f;  // the rotation annihilates the pivot entry
        sh.Sh[i1 * BJ_LD + i2] = nab.hi.x;
        sh.Sl[i1 * BJ_LD + i2] = nab.lo.x;
        sh.Sh[i1 * BJ_LD + j2] = nbh;
        sh.Sl[i1 * BJ_LD + j2] = nbl;
        sh.Sh[j1 * BJ_LD + i2] = nch;
        sh.Sl[j1 * BJ_LD + i2] = ncl;
        sh.Sh[j1 * BJ_LD + j2] = ncd.hi.y;
        sh.Sl[j1 * BJ_LD + j2] = ncd.lo.y;
        if (kp != kq) {
          sh.Sh[i2 * BJ_LD + i1] = nab.hi.x;
          sh.Sl[i2 * BJ_LD + i1] = nab.lo.x;
          sh.Sh[j2 * BJ_LD + i1] = nbh;
          sh.Sl[j2 * BJ_LD + i1] = nbl;
          sh.Sh[i2 * BJ_LD + j1] = nch;
          sh.Sl[i2 * BJ_LD + j1] = ncl;
          sh.Sh[j2 * BJ_LD + j1] = ncd.hi.y;
          sh.Sl[j2 * BJ_LD + j1] = ncd.lo.y;
        }
      } else {
        const int it2 = it - nblk;
        const int row = it2 / BJ_B, kp = it2 % BJ_B;
        int i, j;
        round_pair(BJ_S, r, kp, i, j);
        const float* rr = sh.rot[kp];
        if (rr[2] != 0.f || rr[3] != 0.f) {
          // (q_i, q_j) -> (c q_i - s q_j, s q_i + c q_j)
          const dfp qi = bcast(sh.Ah[row * BJ_LD + i], sh.Al[row * BJ_LD + i]);
          const dfp qj = bcast(sh.Ah[row * BJ_LD + j], sh.Al[row * BJ_LD + j]);
          const dfp cs = pair_of(rr[0], rr[1], rr[2], rr[3]);
          const dfp msc = dfp{make_float2(-rr[2], rr[0]), make_float2(-rr[3], rr[1])};
          const dfp q = dot2_two(cs, qi, msc, qj);
          sh.Ah[row * BJ_LD + i] = q.hi.x;
          sh.Al[row * BJ_LD + i] = q.lo.x;
          sh.Ah[row * BJ_LD + j] = q.hi.y;
          sh.Al[row * BJ_LD + j] = q.lo.y;
        }
      }
    }
    __syncthreads();
  }
}

// out = L^T R (transL) or L R, 32 x 32 double-float, compensated sums; 256 threads x 4
// outputs (two packed pairs)
__device__ __forceinline__ void dfj_matmul(const float* Lh, const float* Ll, const float* Rh, const float* Rl,
                                           float* Oh, float* Ol, bool transL) {
  const int z = threadIdx.x / 8, y0 = (threadIdx.x % 8) * 4;
  float2 S[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  float2 E[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll 4
  for (int x = 0; x < BJ_S; ++x) {
    const int li = transL ? x * BJ_LD + z : z * BJ_LD + x;
    const dfp l = bcast(Lh[li], Ll[li]);
    const dfp nl = neg(l);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int ri = x * BJ_LD + y0 + 2 * u;
      dot2p(S[u], E[u], l, nl, pair_of(Rh[ri], Rl[ri], Rh[ri + 1], Rl[ri + 1]));
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const dfp o = fast_two_sum2(S[u], E[u]);
    Oh[z * BJ_LD + y0 + 2 * u] = o.hi.x;
    Ol[z * BJ_LD + y0 + 2 * u] = o.lo.x;
    Oh[z * BJ_LD + y0 + 2 * u + 1] = o.hi.y;
    Ol[z * BJ_LD + y0 + 2 * u + 1] = o.lo.y;
  }
}

__global__ void __launch_bounds__(JAC_THREADS, 3) jacobi_block_df_kernel(JacParams P) {
  cg::grid_group g = cg::this_grid();
  __shared__ DFShared sh;
  const int m = P.m, M = P.M, NB = M / BJ_B, npairs = NB / 2;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nth = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t MM = static_cast<int64_t>(M) * M;
  float* Qh = reinterpret_cast<float*>(P.Q);
  float* Ql = Qh + static_cast<size_t>(npairs) * BJ_S * BJ_S;
  float* Dh = Ql + static_cast<size_t>(npairs) * BJ_S * BJ_S;  // the diagonalised pair blocks
  float* Dl = Dh + static_cast<size_t>(npairs) * BJ_S * BJ_S;

  double fro = 0.0;
  for (int64_t t = tid; t < MM; t += nth) {
    const int i = static_cast<int>(t / M), j = static_cast<int>(t % M);
    const double v = (i < m && j < m) ? P.H[static_cast<int64_t>(i) * P.ldh + j] : 0.0;
    P.A[t] = v;
    P.V[t] = (i == j) ? 1.0 : 0.0;
    fro += v * v;
  }
  {
    const double b = block_sum(fro, sh.red);
    if (threadIdx.x == 0) P.red[blockIdx.x] = b;
  }
  g.sync();
  double normF2 = 0.0;
  for (int b = 0; b < static_cast<int>(gridDim.x); ++b) normF2 += P.red[b];
  // scale by 2^-e (exact) so that ||A||_F lies in [1/2, 1): every entry then stays inside
  // FP32's range and the split keeps its low part down to 2^-75 ||A||_F
  int e2 = 0;
  const double normF = normF2 > 0.0 ? frexp(sqrt(normF2), &e2) : 0.0;
  for (int64_t t = tid; t < MM; t += nth) P.A[t] = ldexp(P.A[t], -e2);  // this thread's own entries
  g.sync();
  const double tol = fmax(P.tol, 1e-13);

  const int nA = npairs * (npairs + 1) / 2;
  const int nV = (M / BJ_S) * npairs;
  int sweep = 0;
  for (; sweep < JAC_MAX_SWEEPS; ++sweep) {
    double off = 0.0;
    for (int64_t t = tid; t < MM; t += nth) {
      const int i = static_cast<int>(t / M), j = static_cast<int>(t % M);
      if (i != j) off += P.A[t] * P.A[t];
    }
    {
      const double b = block_sum(off, sh.red);
      if (threadIdx.x == 0) P.red[gridDim.x + blockIdx.x] = b;
    }
    g.sync();
    double off2 = 0.0;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) off2 += P.red[gridDim.x + b];
    if (sqrt(off2) <= tol * normF || normF == 0.0) break;
    for (int r = 0; r < NB - 1; ++r) {
      for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
        int I, J;
        round_pair(NB, r, p, I, J);
        for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
          const int x = t / BJ_S, y = t % BJ_S;
          split_f64(P.A[static_cast<int64_t>(bj_index(I, J, x)) * M + bj_index(I, J, y)], sh.Sh[x * BJ_LD + y],
                    sh.Sl[x * BJ_LD + y]);
          sh.Ah[x * BJ_LD + y] = (x == y) ? 1.f : 0.f;
          sh.Al[x * BJ_LD + y] = 0.f;
        }
        __syncthreads();
        dfj_inner_sweep(sh);
        for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
          const size_t o = static_cast<size_t>(p) * BJ_S * BJ_S + t;
          const int si = (t / BJ_S) * BJ_LD + (t % BJ_S);
          Qh[o] = sh.Ah[si];
          Ql[o] = sh.Al[si];
          Dh[o] = sh.Sh[si];
          Dl[o] = sh.Sl[si];
        }
        __syncthreads();
      }
      g.sync();
      for (int task = blockIdx.x; task < nA + nV; task += gridDim.x) {
        if (task < nA) {
          int p = 0, rem = task;
          while (rem >= npairs - p) {
            rem -= npairs - p;
            ++p;
          }
          const int pp = p + rem;
          int I1, J1, I2, J2;
          round_pair(NB, r, p, I1, J1);
          round_pair(NB, r, pp, I2, J2);
          const size_t o1 = static_cast<size_t>(p) * BJ_S * BJ_S, o2 = static_cast<size_t>(pp) * BJ_S * BJ_S;
          if (p == pp) {
            // the pair's own block is the rotated subproblem itself: rotations act on entries
            // near convergence with errors relative to those entries, where the product
            // Q_p^T A Q_p would leave errors of 2^-48 |a_ii| in every off-diagonal entry
            for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
              const int z = t / BJ_S, w = t % BJ_S;
              if (z > w) continue;
              const int64_t gz = bj_index(I1, J1, z), gw = bj_index(I1, J1, w);
              const double v = static_cast<double>(Dh[o1 + t]) + Dl[o1 + t];
              P.A[gz * M + gw] = v;
              P.A[gw * M + gz] = v;
            }
            continue;
          }
          for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
            const int x = t / BJ_S, y = t % BJ_S;
            split_f64(P.A[static_cast<int64_t>(bj_index(I1, J1, x)) * M + bj_index(I2, J2, y)],
                      sh.Sh[x * BJ_LD + y], sh.Sl[x * BJ_LD + y]);
            sh.Ah[x * BJ_LD + y] = Qh[o1 + t];
            sh.Al[x * BJ_LD + y] = Ql[o1 + t];
            sh.Bh[x * BJ_LD + y] = Qh[o2 + t];
            sh.Bl[x * BJ_LD + y] = Ql[o2 + t];
          }
          __syncthreads();
          dfj_matmul(sh.Ah, sh.Al, sh.Sh, sh.Sl, sh.Xh, sh.Xl, true);   // X = Q_p^T A[P, P']
          __syncthreads();
          dfj_matmul(sh.Xh, sh.Xl, sh.Bh, sh.Bl, sh.Sh, sh.Sl, false);  // S = X Q_p'
          __syncthreads();
          for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
            const int z = t / BJ_S, w = t % BJ_S;
            const int64_t gz = bj_index(I1, J1, z), gw = bj_index(I2, J2, w);
            const double v = static_cast<double>(sh.Sh[z * BJ_LD + w]) + sh.Sl[z * BJ_LD + w];
            P.A[gz * M + gw] = v;
            P.A[gw * M + gz] = v;
          }
          __syncthreads();
        } else {
          const int t2 = task - nA;
          const int chunk = t2 / npairs, p = t2 % npairs;
          int I, J;
          round_pair(NB, r, p, I, J);
          const size_t o1 = static_cast<size_t>(p) * BJ_S * BJ_S;
          for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
            const int x = t / BJ_S, y = t % BJ_S;
            split_f64(P.V[static_cast<int64_t>(chunk * BJ_S + x) * M + bj_index(I, J, y)], sh.Sh[x * BJ_LD + y],
                      sh.Sl[x * BJ_LD + y]);
            sh.Ah[x * BJ_LD + y] = Qh[o1 + t];
            sh.Al[x * BJ_LD + y] = Ql[o1 + t];
          }
          __syncthreads();
          dfj_matmul(sh.Sh, sh.Sl, sh.Ah, sh.Al, sh.Xh, sh.Xl, false);  // X = V[rows, P] Q_p
          __syncthreads();
          for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) {
            const int x = t / BJ_S, y = t % BJ_S;
            P.V[static_cast<int64_t>(chunk * BJ_S + x) * M + bj_index(I, J, y)] =
                static_cast<double>(sh.Xh[x * BJ_LD + y]) + sh.Xl[x * BJ_LD + y];
          }
          __syncthreads();
        }
      }
      g.sync();
    }
  }
  for (int64_t i = tid; i < m; i += nth) {
    const double vi = P.A[i * M + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double vj = P.A[static_cast<int64_t>(j) * M + j];
      rank += (vj > vi) || (vj == vi && j < i);
    }
    P.perm[i] = rank;
    P.w_out[rank] = ldexp(vi, e2);
  }
  g.sync();
  for (int64_t t = tid; t < static_cast<int64_t>(m) * m; t += nth) {
    const int row = static_cast<int>(t / m), i = static_cast<int>(t % m);
    P.V_out[static_cast<int64_t>(row) * P.ldv + P.perm[i]] = P.V[static_cast<int64_t>(row) * M + i];
  }
  if (tid == 0 && P.sweeps_out) *P.sweeps_out = sweep;
}

}  // namespace

// orders up to this take the one-CTA kernel; above, the cooperative block kernel.  One SM's
// FP64 pipe bounds the one-CTA kernel (2.2 ms at order 60 on GB300), so from order 33 the
// block kernel's few CTAs (or its double-float form) win: the 64^2 solve took 29.8 ms
// instead of 35.3 ms in FP64 and 24.7 ms instead of 31.0 ms in mixed precision
#ifndef ARB_JAC_ONE_CTA_M
#define ARB_JAC_ONE_CTA_M 32
#endif
static_assert(ARB_JAC_ONE_CTA_M <= JAC_SMALL_M, "the one-CTA kernel holds at most JAC_SMALL_M");

arb_status syevj(arb_ctx ctx, int32_t m, const double* H, int64_t ldh, double* w, double* V,
                 int64_t ldv, int32_t* sweeps, double tol, bool df) {
  if (m <= 0) {
    if (sweeps) *sweeps = 0;
    return ARB_OK;
  }
  if (m > 8192) return set_error(ctx, ARB_INVALID_ARG, "syevj: matrix too large");
  const int M = (m % 2 == 0) ? m : m + 1;
  const int half = M / 2;
  if (M <= ARB_JAC_ONE_CTA_M) {
    const size_t smem = (2 * static_cast<size_t>(M) * M + 2 * half + JAC_SMALL_THREADS) * sizeof(double);
    int32_t* sw;
    ARB_TRY(ws<int32_t>(ctx, WS_JACOBI, 4, &sw));
    // the limit is a property of the kernel shared by all host threads: always set it to
    // the largest size any call uses, so concurrent solves of different orders cannot
    // lower it between another thread's set and launch
    constexpr size_t smem_max =
        (2 * static_cast<size_t>(JAC_SMALL_M) * JAC_SMALL_M + JAC_SMALL_M + JAC_SMALL_THREADS) * sizeof(double);
    ARB_CUDA(ctx, cudaFuncSetAttribute(jacobi_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem_max)));
    JacParams P = {};
    P.tol = tol;
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
  void* kern = df ? reinterpret_cast<void*>(jacobi_block_df_kernel) : reinterpret_cast<void*>(jacobi_block_kernel);
  int& max_blocks = df ? ctx->jacobi_max_blocks_df : ctx->jacobi_max_blocks;
  if (max_blocks == 0) {
    int per_sm = 0;
    ARB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, JAC_THREADS, 0));
    max_blocks = std::max(1, per_sm) * ctx->num_sms;
  }
  const int NB = ((m + BJ_B - 1) / BJ_B + 1) / 2 * 2;  // index blocks, even
  const int MB = NB * BJ_B;
  const int npairs = NB / 2;
  const int tasks = npairs * (npairs + 1) / 2 + (MB / BJ_S) * npairs;
  int grid = std::max(1, std::min(tasks, max_blocks / std::max(1, ctx->coop_share)));
  // scratch: A, V (MB x MB), Q factors, reductions, permutation, sweep count
  const size_t mm = static_cast<size_t>(MB) * MB;
  const size_t qsz = static_cast<size_t>(npairs) * BJ_S * BJ_S * (df ? 2 : 1);
  double* base;
  ARB_TRY(ws<double>(ctx, WS_JACOBI, 2 * mm + qsz + 2 * static_cast<size_t>(grid) + m + 8, &base));
  JacParams P = {};
  P.tol = tol;
  P.m = m;
  P.M = MB;
  P.H = H;
  P.ldh = ldh;
  P.A = base;
  P.V = base + mm;
  P.Q = base + 2 * mm;
  P.red = base + 2 * mm + qsz;
  P.perm = reinterpret_cast<int32_t*>(P.red + 2 * grid);
  P.w_out = w;
  P.V_out = V;
  P.ldv = ldv;
  P.sweeps_out = reinterpret_cast<int32_t*>(P.red + 2 * grid + m + 2);
  void* args[] = {&P};
  ARB_CUDA(ctx, cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(JAC_THREADS), args, 0, ctx->stream));
  ARB_LAUNCHED(ctx);
  if (sweeps) ARB_TRY(d2h_sync(ctx, sweeps, P.sweeps_out, sizeof(int32_t)));
  return ARB_OK;
}

}  // namespace arb
