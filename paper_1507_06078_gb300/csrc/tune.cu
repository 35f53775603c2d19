// Autotuner of the fused block SpMM for one matrix, by measurement on the device.
//
// The hot path's dominant work is the filter's fused SpMM passes (Algorithm 7 / eq. rhod).
// Two settings decide how a pass maps onto the GPU and the best choice depends on the
// matrix and the block width: the row layout (CSR, or SELL-C-sigma with a chunk C and
// sorting window sigma, Kreutzer et al.) and the vector width per lane, which fixes the
// column slice a warp covers per row (32 x width columns).  The tuner times one FP32
// filter-like pass (gather + X and Z streams + output, as in the Clenshaw recurrence) for
// every candidate and keeps the fastest with the matrix.
#include <algorithm>
#include <vector>

#include "arb_internal.h"

namespace arb {
namespace {

__global__ void tune_fill_kernel(int64_t count, float* __restrict__ x) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < count) x[t] = 1.0f + 1e-3f * static_cast<float>(t % 1000);
}

}  // namespace
}  // namespace arb

using namespace arb;

extern "C" arb_status arb_matrix_autotune(arb_ctx ctx, arb_mat mat, int32_t ncols, int32_t* choice, double* ms_out) {
  if (!ctx || !mat || ncols <= 0 || ncols > 4096 || mat->device != ctx->device)
    return set_error(ctx, ARB_INVALID_ARG, "autotune: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  ARB_TRY(ensure_val32(ctx, mat));
  const int64_t n = mat->n;
  const int64_t ld = (ncols + 3) / 4 * 4;
  float* buf;
  ARB_TRY(ws<float>(ctx, WS_TALL0, static_cast<size_t>(4) * n * ld, &buf));
  float *Y = buf, *X = buf + n * ld, *Z = buf + 2 * n * ld, *O = buf + 3 * n * ld;
  {
    const int64_t cnt = 3 * n * ld;
    tune_fill_kernel<<<static_cast<int>((cnt + 255) / 256), 256, 0, ctx->stream>>>(cnt, buf);
    ARB_LAUNCHED(ctx);
  }
  double* coef;
  ARB_TRY(ws<double>(ctx, WS_VEC2, 3 * static_cast<size_t>(ncols), &coef));
  ARB_TRY(fill(ctx, coef, 3 * static_cast<int64_t>(ncols), 0.5));
  SpmmArgs<float> a;
  a.A = mat;
  a.ncols = ncols;
  a.Yin = Y;
  a.ldy = ld;
  a.alpha = -0.25;
  a.beta = 0.5;
  a.sy = coef;
  a.X = X;
  a.ldx = ld;
  a.sx = coef + ncols;
  a.Z = Z;
  a.ldz = ld;
  a.sz = coef + 2 * ncols;
  a.out = O;
  a.ldo = ld;
  struct Cand {
    int C, sigma, vec;
  };
  const int row_max = mat->max_row_nnz;
  std::vector<Cand> cands;
  for (int vec : {4, 2, 1})
    for (const auto& lay : {std::pair<int, int>{0, 0}, {8, 256}, {32, 1024}}) {
      if (lay.first > 0 && n < 4 * lay.first) continue;  // SELL needs a few chunks to matter
      cands.push_back({lay.first, lay.second, vec});
    }
  (void)row_max;
  cudaEvent_t e0, e1;
  ARB_CUDA(ctx, cudaEventCreate(&e0));
  ARB_CUDA(ctx, cudaEventCreate(&e1));
  double best = 1e300;
  Cand pick{0, 0, 0};
  arb_status st = ARB_OK;
  int cur_C = -1;
  for (const Cand& c : cands) {
    if (c.C != cur_C) {
      st = arb_matrix_set_sell(ctx, mat, c.C, c.sigma);
      if (st != ARB_OK) break;
      cur_C = c.C;
    }
    mat->tune_vec = c.vec;
    st = spmm_fused<float>(ctx, a);  // warm-up (kernel attributes, workspaces)
    if (st != ARB_OK) break;
    float best_c = 1e30f;
    for (int r = 0; r < 3 && st == ARB_OK; ++r) {
      cudaEventRecord(e0, ctx->stream);
      st = spmm_fused<float>(ctx, a);
      cudaEventRecord(e1, ctx->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = set_error(ctx, ARB_CUDA_ERROR, "autotune: timing failed");
        break;
      }
      float msr = 0.f;
      cudaEventElapsedTime(&msr, e0, e1);
      best_c = std::min(best_c, msr);
    }
    if (st != ARB_OK) break;
    if (best_c < best) {
      best = best_c;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ARB_OK) {
    mat->tune_vec = 0;
    arb_matrix_set_sell(ctx, mat, 0, 0);
    return st;
  }
  ARB_TRY(arb_matrix_set_sell(ctx, mat, pick.C, pick.sigma));
  mat->tune_vec = pick.vec;
  mat->tuned = true;
  if (choice) {
    choice[0] = pick.C;
    choice[1] = pick.vec;
  }
  if (ms_out) *ms_out = best;
  return ARB_OK;
}
