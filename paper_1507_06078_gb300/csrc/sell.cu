// SELL-C-sigma storage of the matrix (Kreutzer, Hager, Wellein, Fehske & Bishop, SIAM J. Sci.
// Comput. 36(5), 2014) for the block SpMM of the filter: the rows are sorted by decreasing
// nonzero count within windows of sigma consecutive rows, the sorted rows are cut into
// chunks of C, and each chunk is stored column-major with the width of its longest row
// (slot scptr[c] + j C + r holds nonzero j of the chunk's row r).  The SpMM kernels walk
// the rows in sorted order - neighbouring warps of a CTA then get rows of similar length,
// which matters for power-law degree distributions - and read and write the original
// block rows through the permutation, so results match the CSR kernels.
#include <algorithm>
#include <numeric>
#include <vector>

#include "arb_internal.h"
#include "df_arith.cuh"

namespace arb {
namespace {

struct SellLayout {
  std::vector<int32_t> perm, len;
  std::vector<int64_t> cptr;
  int64_t slots = 0;
};

// Rows sorted by decreasing length within each window of sigma rows (ties: lower index
// first), chunk widths and slot offsets.
SellLayout sell_layout(int64_t n, const int32_t* rowptr, int32_t C, int32_t sigma) {
  SellLayout L;
  L.perm.resize(n);
  std::iota(L.perm.begin(), L.perm.end(), 0);
  for (int64_t w0 = 0; w0 < n; w0 += sigma) {
    const int64_t w1 = std::min<int64_t>(n, w0 + sigma);
    std::stable_sort(L.perm.begin() + w0, L.perm.begin() + w1, [&](int32_t a, int32_t b) {
      return rowptr[a + 1] - rowptr[a] > rowptr[b + 1] - rowptr[b];
    });
  }
  L.len.resize(n);
  for (int64_t i = 0; i < n; ++i) L.len[i] = rowptr[L.perm[i] + 1] - rowptr[L.perm[i]];
  const int64_t nchunks = (n + C - 1) / C;
  L.cptr.assign(nchunks + 1, 0);
  for (int64_t c = 0; c < nchunks; ++c) {
    int32_t width = 0;
    for (int64_t i = c * C; i < std::min<int64_t>(n, (c + 1) * C); ++i) width = std::max(width, L.len[i]);
    L.cptr[c + 1] = L.cptr[c] + static_cast<int64_t>(width) * C;
  }
  L.slots = L.cptr[nchunks];
  return L;
}

// src[s] = the CSR index of the nonzero in slot s, -1 for padding
void sell_sources(const SellLayout& L, int64_t n, const int32_t* rowptr, int32_t C, int64_t* src) {
  std::fill(src, src + L.slots, int64_t(-1));
  for (int64_t i = 0; i < n; ++i) {
    const int64_t base = L.cptr[i / C] + i % C;
    const int64_t b = rowptr[L.perm[i]];
    for (int32_t j = 0; j < L.len[i]; ++j) src[base + static_cast<int64_t>(j) * C] = b + j;
  }
}

bool valid_rowptr(int64_t n, const int32_t* rowptr) {
  if (rowptr[0] != 0) return false;
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return false;
  return true;
}

// dst[s] = src[map[s]] (0 where map[s] < 0), and the FP32 / double-float copies
__global__ void sell_gather_kernel(int64_t slots, const int64_t* __restrict__ map, const int32_t* __restrict__ col,
                                   const double* __restrict__ val, int32_t* __restrict__ scol,
                                   double* __restrict__ sval, float* __restrict__ sval32, df2* __restrict__ svaldf) {
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < slots;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t e = map[s];
    const double v = e >= 0 ? val[e] : 0.0;
    scol[s] = e >= 0 ? col[e] : 0;
    sval[s] = v;
    sval32[s] = static_cast<float>(v);
    svaldf[s] = df_from(v);
  }
}

void free_sell(arb_mat m) {
  cudaFree(m->sell_perm);
  cudaFree(m->sell_len);
  cudaFree(m->sell_cptr);
  cudaFree(m->sell_col);
  cudaFree(m->sell_val);
  cudaFree(m->sell_val32);
  cudaFree(m->sell_valdf);
  m->sell_perm = m->sell_len = nullptr;
  m->sell_cptr = nullptr;
  m->sell_col = nullptr;
  m->sell_val = nullptr;
  m->sell_val32 = nullptr;
  m->sell_valdf = nullptr;
  m->sell_C = m->sell_sigma = 0;
  m->sell_slots = 0;
}

}  // namespace

void matrix_free_sell(arb_mat m) { free_sell(m); }

}  // namespace arb

using namespace arb;

extern "C" arb_status arb_sell_layout(int64_t n, const int32_t* rowptr, int32_t C, int32_t sigma, int32_t* perm,
                                      int32_t* len, int64_t* cptr, int64_t* src, int64_t src_capacity,
                                      int64_t* slots) {
  if (n < 0 || !rowptr || C < 1 || sigma < 1 || !slots || (n > 0 && (!perm || !len || !cptr)))
    return ARB_INVALID_ARG;
  if (!valid_rowptr(n, rowptr)) return ARB_INVALID_ARG;
  const SellLayout L = sell_layout(n, rowptr, C, sigma);
  *slots = L.slots;
  std::copy(L.perm.begin(), L.perm.end(), perm);
  std::copy(L.len.begin(), L.len.end(), len);
  std::copy(L.cptr.begin(), L.cptr.end(), cptr);
  if (src) {
    if (src_capacity < L.slots) return ARB_INVALID_ARG;
    sell_sources(L, n, rowptr, C, src);
  }
  return ARB_OK;
}

extern "C" arb_status arb_matrix_set_sell(arb_ctx ctx, arb_mat mat, int32_t C, int32_t sigma) {
  if (!ctx || !mat || C < 0 || (C > 0 && sigma < 1) || C > 1024)
    return set_error(ctx, ARB_INVALID_ARG, "matrix_set_sell: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  std::lock_guard<std::mutex> lock(mat->mu);
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  free_sell(mat);
  if (C == 0) return ARB_OK;
  const int64_t n = mat->n;
  std::vector<int32_t> rp(n + 1);
  ARB_CUDA(ctx, cudaMemcpy(rp.data(), mat->rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  const SellLayout L = sell_layout(n, rp.data(), C, sigma);
  std::vector<int64_t> src(std::max<int64_t>(L.slots, 1));
  sell_sources(L, n, rp.data(), C, src.data());
  const int64_t slots = std::max<int64_t>(L.slots, 1);
  int64_t* dsrc = nullptr;
  auto fail = [&](cudaError_t e, const char* what) {
    cudaFree(dsrc);
    free_sell(mat);
    return cuda_error(ctx, e, what, __FILE__, __LINE__);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&mat->sell_perm, std::max<int64_t>(n, 1) * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&mat->sell_len, std::max<int64_t>(n, 1) * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&mat->sell_cptr, L.cptr.size() * sizeof(int64_t))) != cudaSuccess ||
      (e = cudaMalloc(&mat->sell_col, slots * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&mat->sell_val, slots * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&mat->sell_val32, slots * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&mat->sell_valdf, slots * sizeof(df2))) != cudaSuccess ||
      (e = cudaMalloc(&dsrc, slots * sizeof(int64_t))) != cudaSuccess)
    return fail(e, "matrix_set_sell: allocation");
  if (n > 0) {
    if ((e = cudaMemcpy(mat->sell_perm, L.perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(mat->sell_len, L.len.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(e, "matrix_set_sell: upload");
  }
  if ((e = cudaMemcpy(mat->sell_cptr, L.cptr.data(), L.cptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(dsrc, src.data(), slots * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e, "matrix_set_sell: upload");
  if (L.slots > 0) {
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((L.slots + 255) / 256, 65535));
    sell_gather_kernel<<<blocks, 256, 0, ctx->stream>>>(L.slots, dsrc, mat->col, mat->val, mat->sell_col,
                                                        mat->sell_val, mat->sell_val32, mat->sell_valdf);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "matrix_set_sell: gather");
    ctx->launches++;
  }
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(e, "matrix_set_sell: gather");
  cudaFree(dsrc);
  mat->sell_slots = L.slots;
  mat->sell_sigma = sigma;
  mat->sell_C = C;  // last: the SpMM kernels take the SELL arrays from now on
  return ARB_OK;
}

extern "C" arb_status arb_matrix_sell_info(arb_mat mat, int32_t* C, int32_t* sigma, int64_t* slots) {
  if (!mat || !C || !sigma || !slots) return ARB_INVALID_ARG;
  *C = mat->sell_C;
  *sigma = mat->sell_sigma;
  *slots = mat->sell_slots;
  return ARB_OK;
}
