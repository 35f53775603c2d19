// C ABI of the library: contexts, matrices, the step entry points and the Algorithm 8
// driver (ARRABIT with the multi-power inner solver).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <type_traits>
#include <condition_variable>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arb_internal.h"

namespace arb {

arb_status set_error(arb_ctx ctx, arb_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

arb_status cuda_error(arb_ctx ctx, cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  if (ctx) ctx->last_error = buf;
  return e == cudaErrorMemoryAllocation ? ARB_OUT_OF_MEMORY : ARB_CUDA_ERROR;
}

arb_status ws_get(arb_ctx ctx, int slot, size_t bytes, void** out) {
  if (slot < 0 || slot >= WS_NUM_SLOTS) return set_error(ctx, ARB_INVALID_ARG, "bad workspace slot");
  if (ctx->ws_bytes[slot] < bytes) {
    if (ctx->ws[slot]) {
      if (ctx->stream_ordered) {
        ARB_CUDA(ctx, cudaFreeAsync(ctx->ws[slot], ctx->stream));
      } else {
        ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ARB_CUDA(ctx, cudaFree(ctx->ws[slot]));
      }
      ctx->ws[slot] = nullptr;
      ctx->ws_bytes[slot] = 0;
    }
    void* p = nullptr;
    if (ctx->stream_ordered) {
      ARB_CUDA(ctx, cudaMallocAsync(&p, bytes, ctx->stream));
    } else {
      ARB_CUDA(ctx, cudaMalloc(&p, bytes));
    }
    ctx->ws[slot] = p;
    ctx->ws_bytes[slot] = bytes;
  }
  *out = ctx->ws[slot];
  return ARB_OK;
}

arb_status ws_release_all(arb_ctx ctx) {
  for (int i = 0; i < WS_NUM_SLOTS; ++i) {
    if (!ctx->ws[i]) continue;
    if (ctx->stream_ordered) {
      ARB_CUDA(ctx, cudaFreeAsync(ctx->ws[i], ctx->stream));
    } else {
      ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      ARB_CUDA(ctx, cudaFree(ctx->ws[i]));
    }
    ctx->ws[i] = nullptr;
    ctx->ws_bytes[i] = 0;
  }
  return ARB_OK;
}

arb_status host_stage(arb_ctx ctx, size_t bytes, void** out) {
  if (ctx->host_pinned_bytes < bytes) {
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    ctx->host_pinned = nullptr;
    ctx->host_pinned_bytes = 0;
    ARB_CUDA(ctx, cudaMallocHost(&ctx->host_pinned, bytes));
    ctx->host_pinned_bytes = bytes;
  }
  *out = ctx->host_pinned;
  return ARB_OK;
}

arb_status device_error_word(arb_ctx ctx, int32_t** out) {
  if (!ctx->err_dev) {
    ARB_CUDA(ctx, cudaMalloc(&ctx->err_dev, 4 * sizeof(int32_t)));
    ARB_CUDA(ctx, cudaMemsetAsync(ctx->err_dev, 0, 4 * sizeof(int32_t), ctx->stream));
  }
  *out = ctx->err_dev;
  return ARB_OK;
}

// The read-back also fetches the device error word: a pipelined kernel whose bounded wait
// gave up since the last synchronisation turns this call into ARB_CUDA_ERROR.
arb_status d2h_sync(arb_ctx ctx, void* host, const void* dev, size_t bytes) {
  void* st;
  const size_t off = (bytes + 15) / 16 * 16;
  ARB_TRY(host_stage(ctx, std::max<size_t>(off + 16, 4096), &st));
  ARB_CUDA(ctx, cudaMemcpyAsync(st, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  int32_t* herr = reinterpret_cast<int32_t*>(static_cast<char*>(st) + off);
  *herr = 0;
  if (ctx->err_dev) ARB_CUDA(ctx, cudaMemcpyAsync(herr, ctx->err_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(host, st, bytes);
  if (*herr != 0) {
    ARB_CUDA(ctx, cudaMemsetAsync(ctx->err_dev, 0, sizeof(int32_t), ctx->stream));
    return set_error(ctx, ARB_CUDA_ERROR, "a pipelined kernel's bounded wait gave up (results of the call are void)");
  }
  return ARB_OK;
}

static arb_status h2d(arb_ctx ctx, void* dev, const void* host, size_t bytes) {
  if (bytes == 0) return ARB_OK;
  void* st;
  ARB_TRY(host_stage(ctx, std::max<size_t>(bytes, 4096), &st));
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // staging area may still be in use
  memcpy(st, host, bytes);
  ARB_CUDA(ctx, cudaMemcpyAsync(dev, st, bytes, cudaMemcpyHostToDevice, ctx->stream));
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ARB_OK;
}

// Chebyshev coefficients of the degree-d interpolant of f_d(t) = max(0,t)^(10 d) at the
// points x_j = cos(j pi/d), j = 0..d (the second-kind points of Section 5):
// c_k = (2/d) sum''_j f(x_j) cos(j k pi/d), with the j = 0, d terms and c_0, c_d halved.
static void interpolant_coefficients(int d, double* c) {
  const double pi = 3.14159265358979323846;
  std::vector<double> f(d + 1);
  for (int j = 0; j <= d; ++j) {
    const double x = std::cos(j * pi / d);
    f[j] = x > 0.0 ? std::pow(x, 10.0 * d) : 0.0;
  }
  for (int k = 0; k <= d; ++k) {
    double s = 0.0;
    for (int j = 0; j <= d; ++j) {
      const double w = (j == 0 || j == d) ? 0.5 : 1.0;
      s += w * f[j] * std::cos(static_cast<double>(j) * k * pi / d);
    }
    c[k] = 2.0 * s / d;
  }
  c[0] *= 0.5;
  c[d] *= 0.5;
}

}  // namespace arb

using namespace arb;

// =====================================================================================
// contexts and matrices
// =====================================================================================
extern "C" arb_status arb_ctx_create(arb_ctx* out, int device, void* cuda_stream) {
  if (!out) return ARB_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return ARB_CUDA_ERROR;
  arb_ctx ctx = new arb_ctx_s();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return ARB_CUDA_ERROR;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return ARB_CUDA_ERROR;
  }
  ctx->num_sms = prop.multiProcessorCount;
  // NULL is the legacy default stream, as everywhere in CUDA
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->own_stream = false;
  *out = ctx;
  return ARB_OK;
}

extern "C" arb_status arb_ctx_set_dense_df(arb_ctx ctx, int enable) {
  if (!ctx) return ARB_INVALID_ARG;
  ctx->dense_df = enable != 0;
  return ARB_OK;
}

extern "C" arb_status arb_ctx_destroy(arb_ctx ctx) {
  if (!ctx) return ARB_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < WS_NUM_SLOTS; ++i)
    if (ctx->ws[i]) {
      if (ctx->stream_ordered) cudaFreeAsync(ctx->ws[i], ctx->stream);
      else cudaFree(ctx->ws[i]);
    }
  cudaStreamSynchronize(ctx->stream);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  if (ctx->err_dev) cudaFree(ctx->err_dev);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return ARB_OK;
}

extern "C" const char* arb_last_error(arb_ctx ctx) {
  return ctx ? ctx->last_error.c_str() : "no context";
}

extern "C" const char* arb_status_string(arb_status s) {
  switch (s) {
    case ARB_OK: return "ok";
    case ARB_NOT_CONVERGED: return "not converged";
    case ARB_INVALID_ARG: return "invalid argument";
    case ARB_OUT_OF_MEMORY: return "out of device memory";
    case ARB_NOT_SYMMETRIC: return "matrix not symmetric";
    case ARB_BREAKDOWN: return "iterate lost numerical rank";
    case ARB_CUDA_ERROR: return "CUDA error";
    case ARB_TIMEOUT: return "timeout";
    case ARB_REJECTED: return "rejected";
  }
  return "unknown status";
}

extern "C" int64_t arb_kernel_launches(arb_ctx ctx) { return ctx ? ctx->launches : 0; }

extern "C" void arb_options_default(arb_options* o, int32_t k) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->p = k + static_cast<int32_t>(std::lround(0.1 * k));
  o->q = 1;
  o->degree = 3;
  o->maxit = 30;
  o->maxit1 = 10;
  o->maxit2 = 5;
  o->inner_fixed = 0;
  o->filter = ARB_FILTER_CHEBINTERP;
  o->precision = ARB_FP64;
  o->tol1 = 0.0;
  o->shift_sigma = std::numeric_limits<double>::quiet_NaN();
  o->seed = 20150722ull;
}

// idx_on_device: rowptr/col are device pointers; val_on_device: val is
static arb_status create_csr(arb_ctx ctx, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                             const double* val, int idx_on_device, int val_on_device, arb_mat* out) {
  const int ptr_on_device = idx_on_device;
  if (!ctx || !out || n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val)))
    return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: bad arguments");
  if (n > INT32_MAX || nnz > INT32_MAX)
    return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: int32 index range exceeded");
  *out = nullptr;
  int32_t max_row = -1;
  if (!ptr_on_device) {
    max_row = 0;
    for (int64_t i = 0; i < n; ++i) max_row = std::max<int32_t>(max_row, rowptr[i + 1] - rowptr[i]);
    if (rowptr[0] != 0 || rowptr[n] != nnz)
      return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: rowptr must start at 0 and end at nnz");
    for (int64_t i = 0; i < n; ++i)
      if (rowptr[i + 1] < rowptr[i]) return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: rowptr decreasing");
    for (int64_t e = 0; e < nnz; ++e)
      if (col[e] < 0 || col[e] >= n) return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: column out of range");
  }
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  if (ptr_on_device) {  // the longest row selects the short-row SpMM: read the row pointers once
    std::vector<int32_t> hrp(static_cast<size_t>(n) + 1);
    ARB_CUDA(ctx, cudaMemcpy(hrp.data(), rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    max_row = 0;
    for (int64_t i = 0; i < n; ++i) max_row = std::max<int32_t>(max_row, hrp[i + 1] - hrp[i]);
  }
  arb_mat m = new arb_mat_s();
  m->ctx = ctx;
  m->device = ctx->device;
  m->max_row_nnz = max_row;
  m->n = n;
  m->nnz = nnz;
  const cudaMemcpyKind kind = ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind vkind = val_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMalloc(&m->rowptr, (n + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->col, std::max<int64_t>(nnz, 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->val, std::max<int64_t>(nnz, 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->rowptr, rowptr, (n + 1) * sizeof(int32_t), kind, ctx->stream);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(m->col, col, nnz * sizeof(int32_t), kind, ctx->stream);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(m->val, val, nnz * sizeof(double), vkind, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaFree(m->rowptr);
    cudaFree(m->col);
    cudaFree(m->val);
    delete m;
    return cuda_error(ctx, e, "matrix upload", __FILE__, __LINE__);
  }
  *out = m;
  return ARB_OK;
}

extern "C" arb_status arb_matrix_create_csr(arb_ctx ctx, int64_t n, int64_t nnz, const int32_t* rowptr,
                                            const int32_t* col, const double* val, int ptr_on_device,
                                            arb_mat* out) {
  return create_csr(ctx, n, nnz, rowptr, col, val, ptr_on_device, ptr_on_device, out);
}

extern "C" arb_status arb_matrix_create_csr_f32(arb_ctx ctx, int64_t n, int64_t nnz, const int32_t* rowptr,
                                                const int32_t* col, const float* val, int ptr_on_device,
                                                arb_mat* out) {
  if (!ctx || !out || (nnz > 0 && !val)) return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr_f32: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  // widen on the device: the values go up once as FP32 and are kept in both precisions
  float* v32 = nullptr;
  double* v64 = nullptr;
  ARB_CUDA(ctx, cudaMalloc(&v32, std::max<int64_t>(nnz, 1) * sizeof(float)));
  cudaError_t e = cudaMalloc(&v64, std::max<int64_t>(nnz, 1) * sizeof(double));
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(v32, val, nnz * sizeof(float), ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e != cudaSuccess) {
    cudaFree(v32);
    cudaFree(v64);
    return cuda_error(ctx, e, "matrix_create_csr_f32 upload", __FILE__, __LINE__);
  }
  arb_status st = ARB_OK;
  if (nnz > 0) st = copy_block<float, double>(ctx, nnz, v32, 1, 1, v64, 1);
  if (st == ARB_OK) st = create_csr(ctx, n, nnz, rowptr, col, v64, ptr_on_device, 1, out);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(v64);
  if (st != ARB_OK) {
    cudaFree(v32);
    return st;
  }
  (*out)->val32 = v32;
  return ARB_OK;
}

extern "C" arb_status arb_csr_check_symmetric(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                                              const double* val, double rel_tol) {
  if (n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val)) || !(rel_tol >= 0.0)) return ARB_INVALID_ARG;
  if (rowptr[0] != 0 || rowptr[n] != nnz) return ARB_INVALID_ARG;
  // (row, col) -> value for every stored entry, duplicates summed; then a_ij vs a_ji
  std::vector<std::pair<int64_t, double>> e(static_cast<size_t>(nnz));
  double amax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return ARB_INVALID_ARG;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= n) return ARB_INVALID_ARG;
      e[k] = {i * n + col[k], val[k]};
      amax = std::max(amax, std::fabs(val[k]));
    }
  }
  std::sort(e.begin(), e.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<std::pair<int64_t, double>> u;
  for (const auto& x : e) {
    if (!u.empty() && u.back().first == x.first) u.back().second += x.second;
    else u.push_back(x);
  }
  const double tol = rel_tol * amax;
  for (const auto& x : u) {
    const int64_t i = x.first / n, j = x.first % n;
    if (i == j) continue;
    const auto it = std::lower_bound(u.begin(), u.end(), j * n + i,
                                     [](const auto& a, int64_t key) { return a.first < key; });
    const double mirror = (it != u.end() && it->first == j * n + i) ? it->second : 0.0;
    if (std::fabs(x.second - mirror) > tol) return ARB_NOT_SYMMETRIC;
  }
  return ARB_OK;
}

extern "C" arb_status arb_matrix_destroy(arb_mat m) {
  if (!m) return ARB_INVALID_ARG;
  // the creating context may already be gone: use only what the matrix owns
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  cudaFree(m->rowptr);
  cudaFree(m->col);
  cudaFree(m->val);
  if (m->val32) cudaFree(m->val32);
  if (m->valdf) cudaFree(m->valdf);
  matrix_free_sell(m);
  matrix_free_bulk(m);
  delete m;
  return ARB_OK;
}

extern "C" arb_status arb_matrix_gershgorin(arb_ctx ctx, arb_mat mat, double* lo, double* hi) {
  if (!ctx || !mat || !lo || !hi) return set_error(ctx, ARB_INVALID_ARG, "gershgorin: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  return gershgorin(ctx, mat, lo, hi);
}

extern "C" arb_status arb_filter_coefficients(int32_t filter, int32_t degree, double* coef) {
  if (!coef || degree < 1 || degree > 60) return ARB_INVALID_ARG;
  if (filter == ARB_FILTER_CHEBINTERP) {
    interpolant_coefficients(degree, coef);
  } else if (filter == ARB_FILTER_CHEBYSHEV) {
    for (int i = 0; i <= degree; ++i) coef[i] = (i == degree) ? 1.0 : 0.0;
  } else {
    return ARB_INVALID_ARG;
  }
  return ARB_OK;
}

// =====================================================================================
// step entry points
// =====================================================================================
extern "C" arb_status arb_gaussian_block(arb_ctx ctx, int64_t n, int32_t ncols, uint64_t seed, double* X,
                                         int64_t ldx) {
  if (!ctx || n < 0 || ncols < 0 || (n > 0 && ncols > 0 && (!X || ldx < ncols)))
    return set_error(ctx, ARB_INVALID_ARG, "gaussian_block: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  if (n == 0 || ncols == 0) return ARB_OK;
  return gaussian_fill(ctx, n, ncols, seed, X, ldx);
}

extern "C" arb_status arb_filter(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, double a,
                                 double b, int32_t degree, const double* coef, const double* X,
                                 int64_t ldx, int32_t ncols, const double* xscale, double* Y, int64_t ldy,
                                 double* colss) {
  if (!ctx || !mat || !coef || !X || !Y || ncols < 0 || ldx < ncols || ldy < ncols || !(b > a))
    return set_error(ctx, ARB_INVALID_ARG, "filter: bad arguments");
  if (degree < 1 || degree > 60) return set_error(ctx, ARB_INVALID_ARG, "filter: degree must be in [1, 60]");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t n = mat->n;
  const int64_t ldw = ncols + (ncols & 1);
  double *W1, *W2;
  ARB_TRY(ws<double>(ctx, WS_FILT_W1, static_cast<size_t>(n) * ldw, &W1));
  ARB_TRY(ws<double>(ctx, WS_FILT_W2, static_cast<size_t>(n) * ldw, &W2));
  FilterPlan plan = make_filter_plan(op_scale, op_shift, a, b, degree, coef);
  return filter_apply<double>(ctx, mat, plan, X, ldx, ncols, xscale, W1, W2, ldw, Y, ldy, colss, nullptr);
}

extern "C" arb_status arb_filter_f32(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, double a,
                                     double b, int32_t degree, const double* coef, const float* X, int64_t ldx,
                                     int32_t ncols, const double* xscale, float* Y, int64_t ldy, double* colss) {
  if (!ctx || !mat || !coef || !X || !Y || ncols < 0 || ldx < ncols || ldy < ncols || !(b > a))
    return set_error(ctx, ARB_INVALID_ARG, "filter_f32: bad arguments");
  if (degree < 1 || degree > 60) return set_error(ctx, ARB_INVALID_ARG, "filter_f32: degree must be in [1, 60]");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t n = mat->n;
  const int64_t ldw = ((ncols + 3) / 4) * 4;
  float *W1, *W2;
  ARB_TRY(ws<float>(ctx, WS_F32_W1, static_cast<size_t>(n) * ldw, &W1));
  ARB_TRY(ws<float>(ctx, WS_F32_W2, static_cast<size_t>(n) * ldw, &W2));
  FilterPlan plan = make_filter_plan(op_scale, op_shift, a, b, degree, coef);
  return filter_apply<float>(ctx, mat, plan, X, ldx, ncols, xscale, W1, W2, ldw, Y, ldy, colss, nullptr);
}

extern "C" arb_status arb_filter_df(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, double a,
                                    double b, int32_t degree, const double* coef, const double* X, int64_t ldx,
                                    int32_t ncols, const double* xscale, double* Y, int64_t ldy, double* colss) {
  if (!ctx || !mat || !coef || !X || !Y || ncols < 0 || ldx < ncols || ldy < ncols || !(b > a))
    return set_error(ctx, ARB_INVALID_ARG, "filter_df: bad arguments");
  if (degree < 1 || degree > 60) return set_error(ctx, ARB_INVALID_ARG, "filter_df: degree must be in [1, 60]");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  if (ncols == 0) return ARB_OK;
  const int64_t n = mat->n;
  const int64_t ldw = ncols + (ncols & 1);  // double-float rows padded to 16 bytes
  df2 *W1, *W2, *Xd, *R = nullptr;
  ARB_TRY(ws<df2>(ctx, WS_FILT_W1, static_cast<size_t>(n) * ldw, &W1));
  ARB_TRY(ws<df2>(ctx, WS_FILT_W2, static_cast<size_t>(n) * ldw, &W2));
  ARB_TRY(ws<df2>(ctx, WS_TALL0, static_cast<size_t>(n) * ldw, &Xd));
  ARB_TRY(to_df(ctx, n, X, ldx, ncols, Xd, ldw));
  FilterPlan plan = make_filter_plan(op_scale, op_shift, a, b, degree, coef);
  ARB_TRY(filter_apply<df2>(ctx, mat, plan, Xd, ldw, ncols, xscale, W1, W2, ldw, nullptr, 0, colss, &R));
  return from_df(ctx, n, R, ldw, ncols, Y, ldy);
}

extern "C" arb_status arb_spmm(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, const double* X,
                               int64_t ldx, int32_t ncols, double* Y, int64_t ldy) {
  if (!ctx || !mat || !X || !Y || ncols < 0 || ldx < ncols || ldy < ncols)
    return set_error(ctx, ARB_INVALID_ARG, "spmm: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  SpmmArgs<double> s;
  s.A = mat;
  s.ncols = ncols;
  s.Yin = X;
  s.ldy = ldx;
  s.alpha = op_scale;
  s.beta = op_shift;
  s.out = Y;
  s.ldo = ldy;
  return spmm_fused<double>(ctx, s);
}

extern "C" arb_status arb_gram(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t na,
                               const double* Y, int64_t ldy, int32_t nb, double* C, int64_t ldc) {
  if (!ctx || n < 0 || na < 0 || nb < 0 || !C || ldc < nb || (n > 0 && (!X || !Y || ldx < na || ldy < nb)))
    return set_error(ctx, ARB_INVALID_ARG, "gram: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  if (n == 0) {
    for (int32_t i = 0; i < na; ++i) ARB_TRY(fill(ctx, C + static_cast<int64_t>(i) * ldc, nb, 0.0));
    return ARB_OK;
  }
  return gram<double>(ctx, n, X, ldx, na, Y, ldy, nb, C, ldc);
}

extern "C" arb_status arb_gram_f32(arb_ctx ctx, int64_t n, const float* X, int64_t ldx, int32_t na,
                                   const float* Y, int64_t ldy, int32_t nb, double* C, int64_t ldc) {
  if (!ctx || n < 0 || na < 0 || nb < 0 || !C || ldc < nb || (n > 0 && (!X || !Y || ldx < na || ldy < nb)))
    return set_error(ctx, ARB_INVALID_ARG, "gram_f32: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  if (n == 0) {
    for (int32_t i = 0; i < na; ++i) ARB_TRY(fill(ctx, C + static_cast<int64_t>(i) * ldc, nb, 0.0));
    return ARB_OK;
  }
  return gram<float>(ctx, n, X, ldx, na, Y, ldy, nb, C, ldc);
}

extern "C" arb_status arb_gemm_tall_f32(arb_ctx ctx, int64_t n, const float* In, int64_t ldi, int32_t na,
                                        const double* W, int64_t ldw, int32_t nb, double alpha, double beta,
                                        float* Out, int64_t ldo) {
  if (!ctx || n < 0 || na < 0 || nb < 0 || (n > 0 && nb > 0 && (!Out || ldo < nb)) ||
      (n > 0 && na > 0 && nb > 0 && (!In || !W || ldi < na || ldw < nb)))
    return set_error(ctx, ARB_INVALID_ARG, "gemm_tall_f32: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  return gemm_tall<float>(ctx, n, In, ldi, na, W, ldw, nb, alpha, beta, Out, ldo);
}

extern "C" arb_status arb_syevj(arb_ctx ctx, int32_t m, const double* H, int64_t ldh, double* w, double* V,
                                int64_t ldv, int32_t* sweeps) {
  if (!ctx || m < 0 || (m > 0 && (!H || !w || !V || ldh < m || ldv < m)))
    return set_error(ctx, ARB_INVALID_ARG, "syevj: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  return syevj(ctx, m, H, ldh, w, V, ldv, sweeps, jac_tol<double>(ctx), jac_df<double>(ctx));
}

extern "C" arb_status arb_rcond_gram(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t ncols,
                                     const double* xscale, double* rc) {
  if (!ctx || n <= 0 || !X || ncols <= 0 || ldx < ncols || !rc)
    return set_error(ctx, ARB_INVALID_ARG, "rcond_gram: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  return rcond_gram<double>(ctx, n, X, ldx, ncols, xscale, rc);
}

extern "C" arb_status arb_orth(arb_ctx ctx, int64_t n, const double* Z, int64_t ldz, int32_t m, double* U,
                               int64_t ldu, int32_t* rank) {
  if (!ctx || n <= 0 || !Z || m < 0 || ldz < m || !U || ldu < m || !rank)
    return set_error(ctx, ARB_INVALID_ARG, "orth: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  double* tmp;
  ARB_TRY(ws<double>(ctx, WS_TALL0, static_cast<size_t>(n) * std::max(m, 1), &tmp));
  return orth<double>(ctx, n, Z, ldz, m, U, ldu, tmp, std::max(m, 1), rank);
}

extern "C" arb_status arb_rayleigh_ritz(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift,
                                        int64_t n, const double* Z, int64_t ldz, int32_t m, double* Y,
                                        int64_t ldy, double* w, int32_t* rank) {
  if (!ctx || !mat || n != mat->n || !Z || m <= 0 || ldz < m || !Y || ldy < m || !w || !rank)
    return set_error(ctx, ARB_INVALID_ARG, "rayleigh_ritz: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  double *U, *AU, *tmp, *H, *V;
  ARB_TRY(ws<double>(ctx, WS_TALL0, static_cast<size_t>(n) * m, &tmp));
  ARB_TRY(ws<double>(ctx, WS_TALL1, static_cast<size_t>(n) * m, &U));
  ARB_TRY(ws<double>(ctx, WS_TALL2, static_cast<size_t>(n) * m, &AU));
  int32_t r = 0;
  ARB_TRY(orth<double>(ctx, n, Z, ldz, m, U, m, tmp, m, &r));
  *rank = r;
  if (r == 0) return ARB_OK;
  SpmmArgs<double> s;
  s.A = mat;
  s.ncols = r;
  s.Yin = U;
  s.ldy = m;
  s.alpha = op_scale;
  s.beta = op_shift;
  s.out = AU;
  s.ldo = m;
  ARB_TRY(spmm_fused<double>(ctx, s));
  ARB_TRY(ws<double>(ctx, WS_S_V, static_cast<size_t>(r) * r, &H));
  ARB_TRY(ws<double>(ctx, WS_S_VSEL, static_cast<size_t>(r) * r, &V));
  ARB_TRY(gram<double>(ctx, n, U, m, r, AU, m, r, H, r));
  ARB_TRY(symmetrize(ctx, r, H, r));
  ARB_TRY(syevj(ctx, r, H, r, w, V, r, nullptr, jac_tol<double>(ctx), jac_df<double>(ctx)));
  return gemm_tall<double>(ctx, n, U, m, r, V, r, r, 1.0, 0.0, Y, ldy);
}

extern "C" arb_status arb_arr(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, int64_t n,
                              const double* X, int64_t ldx, int32_t ncols, int32_t q, int32_t npairs,
                              double* Y, int64_t ldy, double* w, int32_t* rank) {
  if (!ctx || !mat || n != mat->n || !X || ncols <= 0 || ldx < ncols || q < 0 || npairs <= 0 || !Y ||
      ldy < npairs || !w || !rank || static_cast<int64_t>(q + 1) * ncols >= n)
    return set_error(ctx, ARB_INVALID_ARG, "arr: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t ldw = ncols + (ncols & 1);
  const int64_t mcap = static_cast<int64_t>(q + 1) * ncols;
  const int64_t ldm = mcap + (mcap & 1);
  ArrWork<double> wk;
  double* Xc;
  ARB_TRY(ws<double>(ctx, WS_TALL0, static_cast<size_t>(n) * ldw, &Xc));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_U, static_cast<size_t>(n) * ldm, &wk.U));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_AU, static_cast<size_t>(n) * ldm, &wk.AU));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_T, static_cast<size_t>(n) * ldw, &wk.T1));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_T2, static_cast<size_t>(n) * ldw, &wk.T2));
  wk.ldu = wk.ldau = ldm;
  wk.ldt = wk.ldt2 = ldw;
  ARB_TRY((copy_block<double, double>(ctx, n, X, ldx, ncols, Xc, ldw)));
  double *theta, *V;
  ARB_TRY(ws<double>(ctx, WS_S_VEC, static_cast<size_t>(mcap), &theta));
  ARB_TRY(ws<double>(ctx, WS_S_V, static_cast<size_t>(mcap) * mcap, &V));
  int32_t m = 0;
  ARB_TRY(arr_basis_and_eig<double>(ctx, mat, op_scale, op_shift, n, Xc, ldw, ncols, nullptr, 0, 0, q, wk, &m,
                                    theta, V));
  *rank = m;
  if (m < npairs) return set_error(ctx, ARB_BREAKDOWN, "arr: subspace smaller than the requested pairs");
  ARB_CUDA(ctx, cudaMemcpyAsync(w, theta, npairs * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return gemm_tall<double>(ctx, n, wk.U, ldm, m, V, m, npairs, 1.0, 0.0, Y, ldy);
}

// =====================================================================================
// Algorithm 8 driver
// =====================================================================================
namespace {

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double sec() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

arb_status upload_ints(arb_ctx ctx, int32_t* dev, const std::vector<int32_t>& h) {
  return h2d(ctx, dev, h.data(), h.size() * sizeof(int32_t));
}

// Everything of a solve that does not depend on the element type of the blocks.
struct SolveState {
  int64_t n = 0;
  int32_t k = 0, p = 0, q = 0, d = 0;
  bool smallest = false;
  double sigma = 0.0, op_scale = 1.0, op_shift = 0.0, a = 0.0, b = 0.0, tol = 0.0, tol_t = 0.0;
  arb_options o{};
  double coef[64] = {};
  int64_t mcap = 0;
  // device vectors
  double *theta = nullptr, *mu = nullptr, *sigc = nullptr, *ss = nullptr, *res = nullptr, *xs = nullptr;
  double *sgn = nullptr, *V = nullptr, *Vsel = nullptr;
  int32_t *imap = nullptr, *iidx = nullptr;
  // host mirror
  int32_t w = 0, nl = 0;
  std::vector<double> h_mu, h_res, h_sigc;
  std::vector<int32_t> h_map;
  double best = std::numeric_limits<double>::infinity();
  int best_iter = 0;
  int outer = 0;  // outer iterations done in the current phase
  // adaptive augmentation and degree (Section 5): the cap of q, the previous maxres, and
  // mu_k, mu_{k+q} of the most accurate iteration so far
  int32_t q_cap = 0;
  double maxres_prev = -1.0;
  bool have_best_mu = false;
  double mu_best_k = 0.0, mu_best_kq = 0.0;
  int stop = ARB_STOP_MAXIT;
  arb_info info{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool trace = false;  // ARB_TRACE set in the environment: one line per outer iteration on stderr
  bool df_filter = false;  // FP64 phase filters in double-float arithmetic (ARB_MIXED_DF)
  // mixed paths: an idle FP32 n x ld32 block the FP64 phase uses for FP32 Gram products of
  // its inner stop rule while the rcond threshold is >= 1e-4.  An FP32 Gram entry is good to
  // ~1e-8 of ||x_i|| ||x_j||, so its smallest eigenvalue carries errors up to ~p 1e-8: at the
  // threshold 1e-6 it cannot tell rc from 0, the inner loop then ran on past the point where
  // the block lost rank (measured on the Chung-Lu Laplacian, k = 90).
  float* x32 = nullptr;
  int64_t ld32 = 0;
};

template <typename T>
struct BlockSet {
  T *X = nullptr, *W1 = nullptr, *W2 = nullptr, *Qc = nullptr, *Xall = nullptr;
  int64_t ld = 0, ldm = 0;
  ArrWork<T> wk;
};

template <typename T>
arb_status alloc_blocks(arb_ctx ctx, const SolveState& S, BlockSet<T>& B) {
  const bool f32 = sizeof(T) == 4;
  const int vec = f32 ? 4 : 2;  // keep rows 16-byte aligned
  B.ld = ((S.p + vec - 1) / vec) * vec;
  B.ldm = ((S.mcap + vec - 1) / vec) * vec;
  const size_t blk = static_cast<size_t>(S.n) * B.ld;
  const size_t big = static_cast<size_t>(S.n) * B.ldm;
  ARB_TRY(ws<T>(ctx, f32 ? WS_F32_X : WS_SOLVER_X, blk, &B.X));
  ARB_TRY(ws<T>(ctx, f32 ? WS_F32_W1 : WS_SOLVER_W1, blk, &B.W1));
  ARB_TRY(ws<T>(ctx, f32 ? WS_F32_W2 : WS_SOLVER_W2, blk, &B.W2));
  ARB_TRY(ws<T>(ctx, f32 ? WS_F32_XALL : WS_SOLVER_XALL, blk, &B.Xall));
  if (!f32) ARB_TRY(ws<T>(ctx, WS_SOLVER_QC, blk, &B.Qc));
  ARB_TRY(ws<T>(ctx, f32 ? WS_F32_U : WS_SOLVER_U, big, &B.wk.U));
  ARB_TRY(ws<T>(ctx, f32 ? WS_F32_AU : WS_SOLVER_AU, big, &B.wk.AU));
  ARB_TRY(ws<T>(ctx, f32 ? WS_F32_T : WS_SOLVER_T, blk, &B.wk.T1));
  ARB_TRY(ws<T>(ctx, f32 ? WS_F32_T2 : WS_SOLVER_T2, blk, &B.wk.T2));
  B.wk.ldu = B.wk.ldau = B.ldm;
  B.wk.ldt = B.wk.ldt2 = B.ld;
  return ARB_OK;
}

}  // namespace

// Section 5 estimates the far end of the spectrum (the paper calls eigs); a loose bound
// widens the filter's damping interval [a, b] and slows the method down, badly for graph
// Laplacians whose Gershgorin discs reach far beyond the spectrum.  Plain Lanczos (no
// reorthogonalisation: only the extreme Ritz values are used) on A, then the extreme
// eigenvalues of the tridiagonal matrix widened by their residual bounds |beta_m y_m| and
// by 1e-3 max(1, |theta|).
arb_status arb::lanczos_bounds(arb_ctx ctx, arb_mat mat, int32_t steps, uint64_t seed, double* lo, double* hi) {
  const int64_t n = mat->n;
  steps = static_cast<int32_t>(std::min<int64_t>(steps, n));
  double* base;
  ARB_TRY(ws<double>(ctx, WS_TALL0, 3 * static_cast<size_t>(n), &base));
  double *vp = base, *v = base + n, *w = base + 2 * n;
  double* dot;
  ARB_TRY(ws<double>(ctx, WS_VEC2, 2, &dot));
  ARB_TRY(gaussian_fill<double>(ctx, n, 1, seed, v, 1));
  ARB_TRY(fill(ctx, vp, n, 0.0));
  double h = 0.0;
  ARB_TRY(gram<double>(ctx, n, v, 1, 1, v, 1, 1, dot, 1));
  ARB_TRY(d2h_sync(ctx, &h, dot, sizeof(double)));
  ARB_TRY(scale_vec(ctx, n, v, v, 1.0 / std::sqrt(h)));
  std::vector<double> al, be;
  double bprev = 0.0;
  for (int j = 0; j < steps; ++j) {
    SpmmArgs<double> sa;
    sa.A = mat;
    sa.ncols = 1;
    sa.Yin = v;
    sa.ldy = 1;
    sa.out = w;
    sa.ldo = 1;
    ARB_TRY(spmm_fused<double>(ctx, sa));
    double aj = 0.0, bj2 = 0.0;
    ARB_TRY(gram<double>(ctx, n, v, 1, 1, w, 1, 1, dot, 1));
    ARB_TRY(d2h_sync(ctx, &aj, dot, sizeof(double)));
    ARB_TRY(lin3(ctx, n, w, aj, v, bprev, vp));
    ARB_TRY(gram<double>(ctx, n, w, 1, 1, w, 1, 1, dot, 1));
    ARB_TRY(d2h_sync(ctx, &bj2, dot, sizeof(double)));
    al.push_back(aj);
    const double bj = std::sqrt(std::max(bj2, 0.0));
    be.push_back(bj);
    if (!(bj > 1e-12 * std::max(1.0, std::fabs(aj)))) break;  // invariant subspace found
    ARB_TRY(scale_vec(ctx, n, vp, v, 1.0));
    ARB_TRY(scale_vec(ctx, n, v, w, 1.0 / bj));
    bprev = bj;
  }
  const int m = static_cast<int>(al.size());
  std::vector<double> T(static_cast<size_t>(m) * m, 0.0);
  for (int i = 0; i < m; ++i) {
    T[static_cast<size_t>(i) * m + i] = al[i];
    if (i + 1 < m) T[static_cast<size_t>(i) * m + i + 1] = T[static_cast<size_t>(i + 1) * m + i] = be[i];
  }
  double *Td, *wd, *Vd;
  ARB_TRY(ws<double>(ctx, WS_SMALL0, static_cast<size_t>(m) * m, &Td));
  ARB_TRY(ws<double>(ctx, WS_SMALL2, static_cast<size_t>(m) * m, &Vd));
  ARB_TRY(ws<double>(ctx, WS_VEC1, m, &wd));
  ARB_TRY(h2d(ctx, Td, T.data(), T.size() * sizeof(double)));
  ARB_TRY(syevj(ctx, m, Td, m, wd, Vd, m, nullptr));
  std::vector<double> ev(m), V(static_cast<size_t>(m) * m);
  ARB_TRY(d2h_sync(ctx, ev.data(), wd, m * sizeof(double)));
  ARB_TRY(d2h_sync(ctx, V.data(), Vd, V.size() * sizeof(double)));
  const double bm = be[m - 1];
  const double rhi = std::fabs(bm * V[static_cast<size_t>(m - 1) * m + 0]);
  const double rlo = std::fabs(bm * V[static_cast<size_t>(m - 1) * m + (m - 1)]);
  *hi = ev[0] + rhi + 1e-3 * std::max(1.0, std::fabs(ev[0]));
  *lo = ev[m - 1] - rlo - 1e-3 * std::max(1.0, std::fabs(ev[m - 1]));
  return ARB_OK;
}

namespace {

// The augmented subspace kept fewer than p directions (orth truncated a block that lost
// numerical rank): complete the Ritz block with Gaussian columns (stream seed + outer
// iteration) orthogonalised twice against the count Ritz vectors, orthonormalised and
// orthogonalised again, with their Rayleigh quotients as Ritz values - the same completion
// the oracle makes.
template <typename T>
arb_status pad_ritz_block(arb_ctx ctx, arb_mat mat, SolveState& S, BlockSet<T>& B, int32_t count, int outer) {
  const int64_t n = S.n;
  const int32_t need = S.p - count;
  T* P = B.wk.T2;  // free after the Rayleigh-Ritz step
  ARB_TRY(gaussian_fill<T>(ctx, n, need, S.o.seed + 1000003ull * static_cast<uint64_t>(S.info.outer_iters + outer),
                           P, B.ld));
  for (int pass = 0; pass < 2; ++pass) ARB_TRY(project_out<T>(ctx, n, B.Xall, B.ld, count, P, B.ld, need));
  int32_t r = 0;
  ARB_TRY(orth<T>(ctx, n, P, B.ld, need, B.wk.T1, B.ld, B.wk.U, B.ldm, &r));
  if (r < need) return set_error(ctx, ARB_BREAKDOWN, "solve: padding columns lost rank");
  for (int pass = 0; pass < 2; ++pass) ARB_TRY(project_out<T>(ctx, n, B.Xall, B.ld, count, B.wk.T1, B.ld, need));
  ARB_TRY((copy_block<T, T>(ctx, n, B.wk.T1, B.ld, need, B.Xall + count, B.ld)));
  // Rayleigh quotients x^T B x / x^T x of the padding columns
  SpmmArgs<T> sa;
  sa.A = mat;
  sa.ncols = need;
  sa.Yin = B.Xall + count;
  sa.ldy = B.ld;
  sa.alpha = S.op_scale;
  sa.beta = S.op_shift;
  sa.colred = S.ss;
  sa.dot_with_yin = true;
  ARB_TRY(spmm_fused<T>(ctx, sa));
  std::vector<double> xbx(need), xx(need), mu(need);
  ARB_TRY(d2h_sync(ctx, xbx.data(), S.ss, need * sizeof(double)));
  sa.alpha = 0.0;  // out = x: the column sums of squares are x^T x
  sa.beta = 1.0;
  sa.dot_with_yin = false;
  ARB_TRY(spmm_fused<T>(ctx, sa));
  ARB_TRY(d2h_sync(ctx, xx.data(), S.ss, need * sizeof(double)));
  for (int c = 0; c < need; ++c) mu[c] = xx[c] > 0.0 ? xbx[c] / xx[c] : 0.0;
  ARB_TRY(h2d(ctx, S.mu + count, mu.data(), need * sizeof(double)));
  S.info.spmm_cols += need;
  return ARB_OK;
}

// The polynomial degree rule of Section 5 (eqs. hat-d and degree): the smallest d >= 3 with
// rho_d(mu_kq) / rho_d(mu_k) < 0.9, capped at d_max, rho_d the filter Algorithm 8 applies
// (psi_d on the map of [0, b - a] onto [-1, 1], evaluated by the three-term recurrence).
int next_degree(int filter, double mu_k, double mu_kq, double a, double b, int d_max) {
  auto psi = [&](int d, double mu) {
    double c[64];
    arb_filter_coefficients(filter, d, c);
    const double t = 2.0 * (mu - a) / (b - a) - 1.0;
    double tp = 1.0, tc = t, sum = c[0] + c[1] * t;
    for (int j = 2; j <= d; ++j) {
      const double tn = 2.0 * t * tc - tp;
      sum += c[j] * tn;
      tp = tc;
      tc = tn;
    }
    return sum;
  };
  for (int d = 3; d <= d_max; ++d) {
    const double rk = psi(d, mu_k), rkq = psi(d, mu_kq);
    if (rk > 0.0 && std::isfinite(rk) && std::isfinite(rkq) && rkq / rk < 0.9) return d;
  }
  return d_max;
}

// One Gauss-Newton inner step (Algorithm 8's GN branch, Algorithm 4 with the accelerator):
// Y = X (X^T X)^{-1}, Z = poly(B - aI, Y, 0, b - a, Gamma_d), X <- Z - X (Y^T Z - I) / 2.
// (X^T X)^{-1} through an FP64 Cholesky factorisation; *ok = false (X unchanged) when X^T X
// is not numerically positive definite.
template <typename T>
arb_status gn_step(arb_ctx ctx, arb_mat mat, SolveState& S, BlockSet<T>& B, const FilterPlan& plan, bool* ok) {
  const int64_t n = S.n;
  const int32_t w = S.w;
  const size_t ww = static_cast<size_t>(w) * w;
  double *G, *R, *Rinv, *Ginv;
  int32_t* status;
  ARB_TRY(ws<double>(ctx, WS_SMALL0, ww, &G));
  ARB_TRY(ws<double>(ctx, WS_CHOL_R, ww, &R));
  ARB_TRY(ws<double>(ctx, WS_CHOL_RINV, ww, &Rinv));
  ARB_TRY(ws<double>(ctx, WS_SMALL1, ww, &Ginv));
  ARB_TRY(ws<int32_t>(ctx, WS_CHOL_STATUS, 4, &status));
  ARB_TRY(gram<T>(ctx, n, B.X, B.ld, w, B.X, B.ld, w, G, w));
  ARB_TRY(spd_inverse(ctx, w, G, w, R, Rinv, Ginv, status));
  int32_t st[2] = {0, 0};
  ARB_TRY(d2h_sync(ctx, st, status, sizeof(st)));
  *ok = st[0] == 0;
  if (!*ok) return ARB_OK;
  T* Y = B.wk.T2;  // free during the inner loop
  ARB_TRY(gemm_tall<T>(ctx, n, B.X, B.ld, w, Ginv, w, w, 1.0, 0.0, Y, B.ld));
  T* Z = nullptr;
  bool filtered = false;
  if constexpr (std::is_same<T, double>::value) {
    if (S.df_filter) {
      df2* Yd = reinterpret_cast<df2*>(B.wk.T1);
      df2* Rd = nullptr;
      ARB_TRY(to_df(ctx, n, Y, B.ld, w, Yd, B.ld));
      ARB_TRY(filter_apply<df2>(ctx, mat, plan, Yd, B.ld, w, nullptr, reinterpret_cast<df2*>(B.W1),
                                reinterpret_cast<df2*>(B.W2), B.ld, nullptr, 0, nullptr, &Rd));
      ARB_TRY(from_df(ctx, n, Rd, B.ld, w, B.wk.T1, B.ld));  // Yd is no longer needed
      Z = B.wk.T1;
      filtered = true;
    }
  }
  if (!filtered) ARB_TRY(filter_apply<T>(ctx, mat, plan, Y, B.ld, w, nullptr, B.W1, B.W2, B.ld, nullptr, 0, nullptr, &Z));
  double* M = G;  // Y^T Z - I
  ARB_TRY(gram<T>(ctx, n, Y, B.ld, w, Z, B.ld, w, M, w));
  ARB_TRY(add_diagonal(ctx, w, M, w, -1.0));
  ARB_TRY(gemm_tall<T>(ctx, n, B.X, B.ld, w, M, w, w, -0.5, 1.0, Z, B.ld));
  // X <- Z: exchange the buffers (all are n x ld blocks of the solve)
  if (Z == B.W1) std::swap(B.X, B.W1);
  else if (Z == B.W2) std::swap(B.X, B.W2);
  else std::swap(B.X, B.wk.T1);
  return ARB_OK;
}

// One phase of Algorithm 8 with blocks of type T (the FP32 phase or the FP64 phase of a
// solve), run until the outer stop rule holds for `tol_phase` (or a stall / maxit /
// all-locked stop).  rc_floor bounds the inner-stop threshold from below (reading c7: 100 u
// of the filter precision); lock = false disables deflation (thresholds of eq. defl are
// below what FP32 blocks resolve).  When cont_on_tol is set, reaching tol_phase performs one
// continuation step (b and tol_t updated as in eq. contin) before the phase ends.
//
// The phase is resumable at the points the lock-step batched driver needs: the start of an
// outer iteration, every inner step (whose filter the caller may have applied for many
// instances at once), the inner stop check, and the ARR / stop-rule tail.
template <typename T>
struct Phase {
  arb_ctx ctx;
  arb_mat mat;
  SolveState* S;
  BlockSet<T>* B;
  double tol_phase = 0.0, rc_floor = 0.0;
  bool lock = true, cont_on_tol = false, stop_on_stag = false;
  int j = 0;                 // outer iteration in progress
  int i1 = 0, i2 = 0;        // inner check and step counters of the current outer iteration
  int n_checks = 0, n_steps = 0;
  double rc = 0.0, rc_thr = 0.0;
  double prev_maxres = std::numeric_limits<double>::infinity();
  bool in_inner = false;     // the inner loop of outer iteration j is running
  bool done = false;         // the phase has ended (S->stop says why)
  int nf0 = 0;

  arb_status begin() {
    S->best = std::numeric_limits<double>::infinity();
    S->best_iter = 0;
    S->outer = 0;
    S->stop = ARB_STOP_MAXIT;
    S->maxres_prev = -1.0;
    S->have_best_mu = false;
    j = 0;
    done = false;
    return ARB_OK;
  }

  // start outer iteration j + 1 (or end the phase at maxit)
  arb_status outer_begin() {
    if (j >= S->o.maxit) {
      done = true;
      return ARB_OK;
    }
    ++j;
    S->outer = j;
    S->info.outer_iters++;
    nf0 = S->info.n_filters;
    ARB_CUDA(ctx, cudaEventRecord(S->ev0, ctx->stream));
    rc = std::numeric_limits<double>::infinity();
    n_checks = S->o.inner_fixed > 0 ? 1 : S->o.maxit1;
    n_steps = S->o.inner_fixed > 0 ? S->o.inner_fixed : S->o.maxit2;
    rc_thr = std::max(S->tol_t, rc_floor);
    i1 = i2 = 0;
    in_inner = true;
    return ARB_OK;
  }

  FilterPlan plan() const { return make_filter_plan(S->op_scale, S->op_shift, S->a, S->b, S->d, S->coef); }

  // MPM steps whose filter an external batched launch performs: the filter reads X with
  // the lazy column scaling xs and writes the result, with its column sums of squares in
  // ss, to filter_out(); step_post() then takes it over as the iterate
  bool batchable() const {
    if (S->o.inner != ARB_INNER_MPM) return false;
    if constexpr (std::is_same<T, double>::value) return !S->df_filter;
    return true;
  }
  T* filter_out() const { return B->W1; }

  // one inner step, filter included
  arb_status step() {
    const int64_t n = S->n;
    const FilterPlan pl = plan();
    if (S->o.inner == ARB_INNER_GN) {
      bool ok = true;
      ARB_TRY(gn_step<T>(ctx, mat, *S, *B, pl, &ok));
      if (!ok) {  // X^T X not positive definite: the GN step is undefined, go to the ARR step
        in_inner = false;
        return ARB_OK;
      }
      if (S->nl > 0) ARB_TRY(project_out<T>(ctx, n, B->Qc, B->ld, S->nl, B->X, B->ld, S->w));
      return count_step();
    }
    bool filtered = false;
    if constexpr (std::is_same<T, double>::value) {
      if (S->df_filter) {
        // double-float filter: X rounded into T1 (free during the inner loop), the passes
        // run in W1 / W2 (same bytes per element as FP64), the result read back into X
        df2* Xd = reinterpret_cast<df2*>(B->wk.T1);
        df2* R = nullptr;
        ARB_TRY(to_df(ctx, n, B->X, B->ld, S->w, Xd, B->ld));
        ARB_TRY(filter_apply<df2>(ctx, mat, pl, Xd, B->ld, S->w, S->xs, reinterpret_cast<df2*>(B->W1),
                                  reinterpret_cast<df2*>(B->W2), B->ld, nullptr, 0, S->ss, &R));
        ARB_TRY(from_df(ctx, n, R, B->ld, S->w, B->X, B->ld));
        filtered = true;
      }
    }
    if (!filtered) {
      T* result = nullptr;
      ARB_TRY(filter_apply<T>(ctx, mat, pl, B->X, B->ld, S->w, S->xs, B->W1, B->W2, B->ld, nullptr, 0, S->ss, &result));
      if (result == B->W1) std::swap(B->X, B->W1);
      else std::swap(B->X, B->W2);
    }
    return normalise_project_count();
  }

  // after an external filter wrote the filtered block into filter_out() (and its column
  // sums of squares into S->ss): it becomes the iterate
  arb_status step_post_external() {
    std::swap(B->X, B->W1);
    return normalise_project_count();
  }

  arb_status normalise_project_count() {
    ARB_TRY(inv_sqrt(ctx, S->w, S->ss, S->xs));  // column normalisation, applied lazily
    if (S->nl > 0) ARB_TRY(project_out<T>(ctx, S->n, B->Qc, B->ld, S->nl, B->X, B->ld, S->w));
    return count_step();
  }

  arb_status count_step() {
    S->info.n_filters++;
    S->info.spmm_cols += static_cast<int64_t>(S->d) * S->w;
    ++i2;
    return ARB_OK;
  }

  bool step_due() const { return in_inner && i2 < n_steps; }

  // after n_steps steps: the inner stop rule (eq. inn-stop), or the end of a fixed schedule
  arb_status check() {
    i2 = 0;
    ++i1;
    if (S->o.inner_fixed > 0) {
      in_inner = false;
      return ARB_OK;
    }
    const int64_t n = S->n;
    const double rcp = rc;
    bool done_rc = false;
    if constexpr (std::is_same<T, double>::value) {
      if (S->x32 && rc_thr >= 1e-4) {
        ARB_TRY((copy_block<double, float>(ctx, n, B->X, B->ld, S->w, S->x32, S->ld32)));
        ARB_TRY(rcond_gram<float>(ctx, n, S->x32, S->ld32, S->w, S->xs, &rc));
        done_rc = true;
      }
    }
    if (!done_rc) ARB_TRY(rcond_gram<T>(ctx, n, B->X, B->ld, S->w, S->xs, &rc));
    if (S->trace) fprintf(stderr, "[arb] %s check %d: rc %.3e (threshold %.1e)\n", sizeof(T) == 4 ? "fp32" : "fp64", i1, rc, rc_thr);
    if (rc <= rc_thr || rc / rcp > 0.99 || i1 >= n_checks) in_inner = false;
    return ARB_OK;
  }

  // augmentation + projection + RR, residuals, stop rules, continuation, deflation and the
  // adaptive rules of the outer iteration j
  arb_status outer_tail() {
    arb_status st = outer_tail_impl();
    if (st != ARB_OK) done = true;
    return st;
  }

  arb_status outer_tail_impl() {
    SolveState& Sr = *S;
    BlockSet<T>& Br = *B;
    const int64_t n = Sr.n;
    const int32_t p = Sr.p, k = Sr.k;
    float ms = 0.f;
    ARB_CUDA(ctx, cudaEventRecord(Sr.ev1, ctx->stream));
    ARB_CUDA(ctx, cudaEventSynchronize(Sr.ev1));
    ARB_CUDA(ctx, cudaEventElapsedTime(&ms, Sr.ev0, Sr.ev1));
    Sr.info.t_filter += ms * 1e-3;
    // ---------------- augmentation + projection + RR (Algorithm 5 inside Algorithm 8)
    ARB_CUDA(ctx, cudaEventRecord(Sr.ev0, ctx->stream));
    int32_t m = 0;
    ARB_TRY(arr_basis_and_eig<T>(ctx, mat, Sr.op_scale, Sr.op_shift, n, Br.X, Br.ld, Sr.w, Br.Qc, Br.ld, Sr.nl, Sr.q,
                                 Br.wk, &m, Sr.theta, Sr.V));
    Sr.info.last_rank = m;
    Sr.info.spmm_cols += m;
    // the p leading pairs of (Q_c, Sigma_c) and (U V, theta)
    ARB_TRY(select_top(ctx, Sr.sigc, Sr.nl, Sr.theta, m, p, Sr.imap, Sr.mu));
    ARB_TRY(d2h_sync(ctx, Sr.h_map.data(), Sr.imap, p * sizeof(int32_t)));
    int32_t count = 0;  // Ritz pairs available (the rest of the block is padded below)
    while (count < p && Sr.h_map[count] >= 0) ++count;
    // mu_{k+q} is an estimate of lambda_{k+q} only when it is a Ritz value: after padding
    // (a Rayleigh quotient of a random column) b keeps its previous value
    const bool b_ok = (count == p);
    if (count == 0) return set_error(ctx, ARB_BREAKDOWN, "solve: no Ritz pairs");
    std::vector<int32_t> newcols, src(count);
    for (int s = 0; s < count; ++s) {
      if (Sr.h_map[s] < Sr.nl) {
        src[s] = -Sr.h_map[s] - 1;  // locked column
      } else {
        src[s] = static_cast<int32_t>(newcols.size());
        newcols.push_back(Sr.h_map[s] - Sr.nl);
      }
    }
    const int32_t pn = static_cast<int32_t>(newcols.size());
    if (pn > 0) {
      ARB_TRY(upload_ints(ctx, Sr.iidx, newcols));
      ARB_TRY(gather_cols<double>(ctx, m, Sr.V, m, Sr.iidx, pn, Sr.Vsel, pn));  // V: m x m, ld m
      ARB_TRY(gemm_tall<T>(ctx, n, Br.wk.U, Br.ldm, m, Sr.Vsel, pn, pn, 1.0, 0.0, Br.wk.T1, Br.ld));
    }
    ARB_TRY(upload_ints(ctx, Sr.imap, src));
    ARB_TRY(gather_cols2<T>(ctx, n, Br.wk.T1, Br.ld, Br.Qc, Br.ld, Sr.imap, count, Br.Xall, Br.ld));
    if (count < p) ARB_TRY(pad_ritz_block(ctx, mat, Sr, Br, count, j));
    // residuals (eq. resi): ||B x - mu x|| with the sign folded (-B x + mu x)
    {
      SpmmArgs<T> sa;
      sa.A = mat;
      sa.ncols = p;
      sa.Yin = Br.Xall;
      sa.ldy = Br.ld;
      sa.alpha = -Sr.op_scale;
      sa.beta = -Sr.op_shift;
      sa.X = Br.Xall;
      sa.ldx = Br.ld;
      sa.sx = Sr.mu;
      sa.colred = Sr.ss;
      ARB_TRY(spmm_fused<T>(ctx, sa));
      ARB_TRY(residual_finish(ctx, p, Sr.ss, Sr.mu, Sr.smallest ? 1 : 0, Sr.sigma, Sr.res));
      Sr.info.spmm_cols += p;
    }
    ARB_TRY(d2h_sync(ctx, Sr.h_mu.data(), Sr.mu, p * sizeof(double)));
    ARB_TRY(d2h_sync(ctx, Sr.h_res.data(), Sr.res, p * sizeof(double)));
    ARB_CUDA(ctx, cudaEventRecord(Sr.ev1, ctx->stream));
    ARB_CUDA(ctx, cudaEventSynchronize(Sr.ev1));
    ARB_CUDA(ctx, cudaEventElapsedTime(&ms, Sr.ev0, Sr.ev1));
    Sr.info.t_arr += ms * 1e-3;

    // ---------------- outer stop rules, continuation, deflation (Section 5)
    double maxres = 0.0;
    int h = 0;
    for (int i = 0; i < k; ++i) {
      maxres = std::max(maxres, std::isnan(Sr.h_res[i]) ? std::numeric_limits<double>::infinity() : Sr.h_res[i]);
      h += Sr.h_res[i] < 0.1 * tol_phase;
    }
    if (Sr.trace)
      fprintf(stderr,
              "[arb] %s outer %d: filters %d (total %d) rc %.3e rank %d maxres %.3e b %.9g tol_t %.1e locked %d "
              "t_filter %.3fs t_arr %.3fs\n",
              sizeof(T) == 4 ? "fp32" : "fp64", j, Sr.info.n_filters - nf0, Sr.info.n_filters, rc,
              m, maxres, Sr.b, Sr.tol_t, Sr.nl, Sr.info.t_filter, Sr.info.t_arr);
    Sr.info.maxres = maxres;
    if (maxres < Sr.best) {
      Sr.best = maxres;
      Sr.best_iter = j;
      Sr.have_best_mu = true;
      Sr.mu_best_k = Sr.h_mu[k - 1];
      Sr.mu_best_kq = Sr.h_mu[p - 1];
    }
    if (maxres <= tol_phase) {
      Sr.stop = ARB_STOP_CONVERGED;
      if (cont_on_tol && tol_phase > Sr.tol) {
        if (b_ok) Sr.b = Sr.h_mu[p - 1];
        if (!(Sr.b > Sr.a)) Sr.b = Sr.a + 1e-3 * std::max(1.0, std::fabs(Sr.a));
      }
      done = true;
      return ARB_OK;
    }
    // mixed path: the FP32 iterate has reached its accuracy floor when an outer iteration
    // no longer halves maxres; hand over to FP64 with the best interval estimate
    if (stop_on_stag && j >= 2 && maxres > 0.5 * prev_maxres) {
      Sr.stop = ARB_STOP_STALLED;
      if (b_ok) Sr.b = Sr.h_mu[p - 1];
      if (!(Sr.b > Sr.a)) Sr.b = Sr.a + 1e-3 * std::max(1.0, std::fabs(Sr.a));
      done = true;
      return ARB_OK;
    }
    prev_maxres = maxres;
    if (maxres < (1.0 + 9.0 * h / k) * tol_phase) {
      Sr.stop = ARB_STOP_NEAR_TOL;
      done = true;
      return ARB_OK;
    }
    if (j - Sr.best_iter >= 3) {
      Sr.stop = ARB_STOP_STALLED;
      done = true;
      return ARB_OK;
    }
    if (maxres <= Sr.tol_t) {  // continuation, eq. contin
      Sr.tol_t = std::max(1e-2 * Sr.tol_t, Sr.tol);
      if (b_ok) Sr.b = Sr.h_mu[p - 1];
    } else if (Sr.o.b_update == 1) {  // Section 5: a better estimate of lambda_{k+q} after each ARR
      if (b_ok) Sr.b = Sr.h_mu[p - 1];
    }
    if (!(Sr.b > Sr.a)) Sr.b = Sr.a + 1e-3 * std::max(1.0, std::fabs(Sr.a));
    const double thr = std::max(1e-14, Sr.tol_t * Sr.tol_t);  // eq. defl
    std::vector<int32_t> lock_idx, free_idx;
    Sr.h_sigc.clear();
    for (int s = 0; s < p; ++s) {
      if (lock && s < k && Sr.h_res[s] <= thr) {
        lock_idx.push_back(s);
        Sr.h_sigc.push_back(Sr.h_mu[s]);
      } else {
        free_idx.push_back(s);
      }
    }
    Sr.nl = static_cast<int32_t>(lock_idx.size());
    Sr.info.max_locked = std::max(Sr.info.max_locked, Sr.nl);
    Sr.w = p - Sr.nl;
    if (Sr.w == 0) {
      Sr.stop = ARB_STOP_ALL_LOCKED;
      done = true;
      return ARB_OK;
    }
    if (Sr.nl > 0) {
      ARB_TRY(upload_ints(ctx, Sr.iidx, lock_idx));
      ARB_TRY(gather_cols<T>(ctx, n, Br.Xall, Br.ld, Sr.iidx, Sr.nl, Br.Qc, Br.ld));
      ARB_TRY(h2d(ctx, Sr.sigc, Sr.h_sigc.data(), Sr.nl * sizeof(double)));
    }
    ARB_TRY(upload_ints(ctx, Sr.iidx, free_idx));
    ARB_TRY(gather_cols<T>(ctx, n, Br.Xall, Br.ld, Sr.iidx, Sr.w, Br.X, Br.ld));
    ARB_TRY(fill(ctx, Sr.xs, Sr.w, 1.0));
    // augmentation blocks (eq. block): little decay of the relevant Ritz values of B - aI
    // (the operator the inner solver works on) and a disappointing residual decrease
    if ((Sr.o.adapt & ARB_ADAPT_Q) && Sr.maxres_prev > 0.0 && Sr.q < Sr.q_cap) {
      const double ratio = (Sr.h_mu[p - 1] - Sr.a) / (Sr.h_mu[k - 1] - Sr.a);
      if (ratio > 0.95 && maxres / Sr.maxres_prev > 0.1) Sr.q++;
    }
    Sr.maxres_prev = maxres;
    // polynomial degree (eqs. hat-d, degree) from the most accurate Ritz values so far
    if ((Sr.o.adapt & ARB_ADAPT_DEGREE) && Sr.have_best_mu) {
      const int d = next_degree(Sr.o.filter, Sr.mu_best_k, Sr.mu_best_kq, Sr.a, Sr.b, Sr.o.d_max > 0 ? Sr.o.d_max : 15);
      if (d != Sr.d) {
        Sr.d = d;
        if (arb_filter_coefficients(Sr.o.filter, Sr.d, Sr.coef) != ARB_OK)
          return set_error(ctx, ARB_INVALID_ARG, "solve: bad filter kind");
      }
    }
    return ARB_OK;
  }
};

template <typename T>
arb_status run_outer(arb_ctx ctx, arb_mat mat, SolveState& S, BlockSet<T>& B, double tol_phase, double rc_floor,
                     bool lock, bool continue_on_phase_tol, bool stop_on_stagnation = false) {
  Phase<T> ph;
  ph.ctx = ctx;
  ph.mat = mat;
  ph.S = &S;
  ph.B = &B;
  ph.tol_phase = tol_phase;
  ph.rc_floor = rc_floor;
  ph.lock = lock;
  ph.cont_on_tol = continue_on_phase_tol;
  ph.stop_on_stag = stop_on_stagnation;
  ARB_TRY(ph.begin());
  for (;;) {
    ARB_TRY(ph.outer_begin());
    if (ph.done) break;
    while (ph.in_inner) {
      while (ph.step_due()) ARB_TRY(ph.step());
      if (ph.in_inner) ARB_TRY(ph.check());
    }
    ARB_TRY(ph.outer_tail());
    if (ph.done) break;
  }
  return ARB_OK;
}

// One arb_solve: set-up (spectrum bounds, workspaces, start block, first b), the phases of
// Algorithm 8 (an FP32 phase and an FP64 refinement on the mixed paths, one FP64 phase
// otherwise) and the outputs.  solve_impl runs the phases back to back; the lock-step
// batched driver advances the phases of many solves together.
struct Solve {
  arb_ctx ctx = nullptr;
  arb_mat mat = nullptr;
  Timer total;
  SolveState S;
  BlockSet<double> D;
  BlockSet<float> F;
  bool mixed = false;
  double lo_A = 0.0, hi_A = 0.0;
  double tol_phase32 = 0.0, tol_t64 = 0.0;
  int stage = 0;  // 0: FP32 phase, 1: FP64 phase, 2: phases over
  Phase<float> p32;
  Phase<double> p64;
  bool dense_set = false, dense_saved = false;

  ~Solve() {
    if (S.ev0) cudaEventDestroy(S.ev0);
    if (S.ev1) cudaEventDestroy(S.ev1);
    if (dense_set) ctx->dense_df = dense_saved;
  }

  arb_status setup(int32_t k, arb_which which, double tol, const arb_options& o, const double* x0, int x0_on_device,
                   double* evecs, int64_t ldq) {
    S.o = o;
    S.n = mat->n;
    S.k = k;
    S.p = o.p > 0 ? o.p : k + static_cast<int32_t>(std::lround(0.1 * k));
    S.q = o.q;
    S.d = o.degree;
    S.tol = tol;
    const int64_t n = S.n;
    const int32_t p = S.p;
    if (k <= 0 || k > p || S.q < 0 || S.d < 1 || S.d > 60 || o.maxit < 1 || o.maxit1 < 1 || o.maxit2 < 1 ||
        static_cast<int64_t>(S.q + 1) * p >= n || !(tol > 0.0))
      return set_error(ctx, ARB_INVALID_ARG, "solve: need 0 < k <= p, (q+1) p < n, 1 <= degree <= 60, tol > 0");
    if (o.precision != ARB_FP64 && o.precision != ARB_MIXED && o.precision != ARB_MIXED_DF)
      return set_error(ctx, ARB_INVALID_ARG, "solve: unknown precision");
    if (o.b_update != 0 && o.b_update != 1) return set_error(ctx, ARB_INVALID_ARG, "solve: b_update must be 0 or 1");
    if (o.inner != ARB_INNER_MPM && o.inner != ARB_INNER_GN) return set_error(ctx, ARB_INVALID_ARG, "solve: bad inner solver");
    if ((o.adapt & ~(ARB_ADAPT_Q | ARB_ADAPT_DEGREE)) != 0 || o.q_max < 0 || o.d_max < 0 || o.d_max > 60)
      return set_error(ctx, ARB_INVALID_ARG, "solve: bad adaptation options");
    if (which != ARB_LARGEST && which != ARB_SMALLEST) return set_error(ctx, ARB_INVALID_ARG, "solve: bad which");
    if (evecs && ldq < n) return set_error(ctx, ARB_INVALID_ARG, "solve: ldq < n");
    S.smallest = (which == ARB_SMALLEST);
    mixed = (o.precision == ARB_MIXED || o.precision == ARB_MIXED_DF);
    S.df_filter = (o.precision == ARB_MIXED_DF);
    S.trace = getenv("ARB_TRACE") != nullptr;

    // operator B = op_scale A + op_shift I whose largest eigenpairs are wanted; the far end
    // of A's spectrum from the tighter of Gershgorin's bound and a Lanczos estimate
    double glo, ghi, llo, lhi;
    ARB_TRY(gershgorin(ctx, mat, &glo, &ghi));
    ARB_TRY(lanczos_bounds(ctx, mat, 32, o.seed + 0x9E3779B97F4A7C15ull, &llo, &lhi));
    hi_A = std::min(ghi, lhi);
    lo_A = std::max(glo, llo);
    if (S.smallest) {
      S.sigma = std::isnan(o.shift_sigma) ? hi_A : o.shift_sigma;
      S.op_scale = -1.0;
      S.op_shift = S.sigma;
      S.a = S.sigma - hi_A;  // lower bound of sigma I - A
    } else {
      S.a = lo_A;
    }

    // device buffers (room for the largest q the adaptation may reach, (q+1) p < n)
    S.q_cap = S.q;
    if (o.adapt & ARB_ADAPT_Q) {
      const int64_t fit = (n - 1) / p - 1;
      S.q_cap = static_cast<int32_t>(std::max<int64_t>(S.q, std::min<int64_t>(o.q_max > 0 ? o.q_max : 3, fit)));
    }
    S.mcap = static_cast<int64_t>(S.q_cap + 1) * p;
    ARB_TRY(alloc_blocks<double>(ctx, S, D));
    if (mixed) {
      ARB_TRY(alloc_blocks<float>(ctx, S, F));
      ARB_TRY(ensure_val32(ctx, mat));
      if (S.df_filter) ARB_TRY(ensure_valdf(ctx, mat));
    }
    ARB_TRY(ws<double>(ctx, WS_S_V, static_cast<size_t>(S.mcap) * S.mcap, &S.V));
    ARB_TRY(ws<double>(ctx, WS_S_VSEL, static_cast<size_t>(S.mcap) * p, &S.Vsel));
    double* vec;
    ARB_TRY(ws<double>(ctx, WS_S_VEC, static_cast<size_t>(S.mcap) + 8 * static_cast<size_t>(p) + 64, &vec));
    S.theta = vec;
    S.mu = S.theta + S.mcap;
    S.sigc = S.mu + p;
    S.ss = S.sigc + p;
    S.res = S.ss + p;
    S.xs = S.res + p;
    S.imap = reinterpret_cast<int32_t*>(S.xs + p);
    S.iidx = S.imap + p + (p & 1);
    S.sgn = reinterpret_cast<double*>(S.iidx + p + (p & 1));
    S.h_mu.resize(p);
    S.h_res.resize(p);
    S.h_map.resize(p);

    // start block X0 (Algorithm 8: i.i.d. Gaussian n x (k+q)), held in the FP64 iterate
    if (x0) {
      ARB_CUDA(ctx, cudaMemcpy2DAsync(D.X, D.ld * sizeof(double), x0, p * sizeof(double), p * sizeof(double), n,
                                      x0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                      ctx->stream));
    } else {
      ARB_TRY(gaussian_fill(ctx, n, p, o.seed, D.X, D.ld));
    }

    // b: smallest Ritz value of orth(X0) (Section 5, "Estimation of lambda_n and lambda_{k+q}");
    // an estimate, so the mixed paths take it from FP32 blocks
    auto initial_b = [&](auto& Bk) -> arb_status {
      using E = typename std::remove_reference<decltype(*Bk.X)>::type;
      int32_t r = 0;
      ARB_TRY(orth<E>(ctx, n, Bk.X, Bk.ld, p, Bk.wk.U, Bk.ldm, Bk.wk.T1, Bk.ld, &r));
      if (r == 0) return set_error(ctx, ARB_BREAKDOWN, "solve: start block has no numerical rank");
      SpmmArgs<E> sa;
      sa.A = mat;
      sa.ncols = r;
      sa.Yin = Bk.wk.U;
      sa.ldy = Bk.ldm;
      sa.alpha = S.op_scale;
      sa.beta = S.op_shift;
      sa.out = Bk.wk.AU;
      sa.ldo = Bk.ldm;
      ARB_TRY(spmm_fused<E>(ctx, sa));
      double* H;
      ARB_TRY(ws<double>(ctx, WS_SMALL0, static_cast<size_t>(r) * r, &H));
      ARB_TRY(gram<E>(ctx, n, Bk.wk.U, Bk.ldm, r, Bk.wk.AU, Bk.ldm, r, H, r));
      ARB_TRY(symmetrize(ctx, r, H, r));
      ARB_TRY(syevj(ctx, r, H, r, S.theta, S.V, r, nullptr, jac_tol<E>(ctx), jac_df<E>(ctx)));
      ARB_TRY(d2h_sync(ctx, &S.b, S.theta + (r - 1), sizeof(double)));
      S.info.spmm_cols += r;
      return ARB_OK;
    };
    if (mixed) {
      ARB_TRY((copy_block<double, float>(ctx, n, D.X, D.ld, p, F.X, F.ld)));
      ARB_TRY(initial_b(F));
      S.x32 = F.wk.T2;
      S.ld32 = F.ld;
    } else {
      ARB_TRY(initial_b(D));
    }
    S.info.a = S.a;
    S.info.b0 = S.b;
    S.info.sigma = S.sigma;
    if (!(S.b > S.a)) S.b = S.a + 1e-3 * std::max(1.0, std::fabs(S.a));

    if (arb_filter_coefficients(o.filter, S.d, S.coef) != ARB_OK)
      return set_error(ctx, ARB_INVALID_ARG, "solve: bad filter kind");
    const double tol1 = o.tol1 > 0.0 ? o.tol1 : (tol <= 1e-8 ? std::max(1e-6, tol) : tol);
    S.tol_t = std::max(tol1, tol);
    S.w = p;
    S.nl = 0;
    ARB_TRY(fill(ctx, S.xs, S.w, 1.0));
    ARB_CUDA(ctx, cudaEventCreate(&S.ev0));
    ARB_CUDA(ctx, cudaEventCreate(&S.ev1));

    return ARB_OK;
  }

  // the first phase: FP32 on the mixed paths (reading c7: inner-stop threshold >= 100 u32;
  // the FP32 residual floor ~ 32 u32 ||B||, ||B|| bounded by the spectrum estimates, ends it,
  // as do tol_switch and an outer iteration that fails to halve maxres), else FP64
  arb_status start() {
    if (mixed) {
      const double normB = std::max(std::fabs(S.sigma - lo_A), std::fabs(S.sigma - hi_A));
      const double floor32 = 32.0 * 5.96e-8 * (S.smallest ? normB : std::max(std::fabs(lo_A), std::fabs(hi_A)));
      const double sw = std::max(S.o.tol_switch > 0.0 ? S.o.tol_switch : 1e-5, floor32);
      tol_phase32 = std::max(sw, S.tol);
      tol_t64 = S.tol_t;  // the FP64 phase starts the paper's continuation at tol_1
      S.tol_t = std::max(S.tol_t, tol_phase32);
      init_phase(p32, F, tol_phase32, 100.0 * 5.96e-8, false, true, true);
      stage = 0;
      return p32.begin();
    }
    init_phase(p64, D, S.tol, 0.0, true, false, false);
    stage = 1;
    return p64.begin();
  }

  template <typename T>
  void init_phase(Phase<T>& ph, BlockSet<T>& B, double tol_phase, double rc_floor, bool lock, bool cont, bool stag) {
    ph.ctx = ctx;
    ph.mat = mat;
    ph.S = &S;
    ph.B = &B;
    ph.tol_phase = tol_phase;
    ph.rc_floor = rc_floor;
    ph.lock = lock;
    ph.cont_on_tol = cont;
    ph.stop_on_stag = stag;
  }

  // the current phase has ended: from the FP32 phase to the FP64 refinement (Algorithm 8
  // continued in FP64 from the FP32 Ritz block), or the end of the phases
  arb_status phase_ended() {
    const int64_t n = S.n;
    const int32_t p = S.p;
    if (stage == 0) {
      S.info.outer_iters_fp32 = S.info.outer_iters;
      S.tol_t = tol_t64;
      const bool done32 = (S.stop == ARB_STOP_CONVERGED || S.stop == ARB_STOP_NEAR_TOL) && tol_phase32 <= S.tol;
      // If the FP32 phase made no usable progress - its block lost rank (the filter's
      // dynamic range outran FP32 before the inner stop rule could see it, e.g. an isolated
      // extreme eigenvalue and a crude first b) or maxres stayed above 1e-2 - the refinement
      // starts over from X0 with the first interval estimate, as the FP64 method would.
      const bool fp32_failed = !(S.info.maxres <= 1e-2) || S.info.last_rank < p;
      if (fp32_failed) {
        S.b = S.info.b0;
        if (!(S.b > S.a)) S.b = S.a + 1e-3 * std::max(1.0, std::fabs(S.a));
        S.tol_t = tol_t64;
      } else {
        ARB_TRY((copy_block<float, double>(ctx, n, F.Xall, F.ld, p, D.Xall, D.ld)));
      }
      if (!done32 || fp32_failed) {
        // D.X still holds X0 (the FP32 phase ran on its own blocks)
        if (!fp32_failed) ARB_TRY((copy_block<double, double>(ctx, n, D.Xall, D.ld, p, D.X, D.ld)));
        S.w = p;
        S.nl = 0;
        ARB_TRY(fill(ctx, S.xs, S.w, 1.0));
        // ARB_MIXED_DF: the refinement's dense products in double-float arithmetic too
        if (S.df_filter) {
          dense_set = true;
          dense_saved = ctx->dense_df;
          ctx->dense_df = true;
        }
        init_phase(p64, D, S.tol, 0.0, true, false, false);
        stage = 1;
        return p64.begin();
      }
      stage = 2;
      return ARB_OK;
    }
    if (dense_set) {
      ctx->dense_df = dense_saved;
      dense_set = false;
    }
    stage = 2;
    return ARB_OK;
  }

  // every phase to its end, back to back
  arb_status run() {
    ARB_TRY(start());
    while (stage < 2) {
      if (stage == 0) ARB_TRY(run_phase(p32));
      else ARB_TRY(run_phase(p64));
      ARB_TRY(phase_ended());
    }
    return ARB_OK;
  }

  template <typename T>
  static arb_status run_phase(Phase<T>& ph) {
    for (;;) {
      ARB_TRY(ph.outer_begin());
      if (ph.done) return ARB_OK;
      while (ph.in_inner) {
        while (ph.step_due()) ARB_TRY(ph.step());
        if (ph.in_inner) ARB_TRY(ph.check());
      }
      ARB_TRY(ph.outer_tail());
      if (ph.done) return ARB_OK;
    }
  }

  // outputs: Rayleigh quotients on A, order, sign, column-major copy
  arb_status finish(double* evals, double* evecs, int64_t ldq, int evecs_on_device, arb_info* info_out) {
    const int64_t n = S.n;
    const int32_t p = S.p, k = S.k;
    S.info.stop_reason = S.stop;
    S.info.b_final = S.b;
    S.info.n_locked = S.nl;
    S.info.final_q = S.q;
    S.info.final_d = S.d;

    // ---------------- outputs: Rayleigh quotients on A, order, sign, column-major copy
    {
      SpmmArgs<double> sa;
      sa.A = mat;
      sa.ncols = k;
      sa.Yin = D.Xall;
      sa.ldy = D.ld;
      sa.alpha = 1.0;
      sa.beta = 0.0;
      sa.colred = S.ss;
      sa.dot_with_yin = true;
      ARB_TRY(spmm_fused<double>(ctx, sa));
      S.info.spmm_cols += k;
    }
    std::vector<double> rq(k);
    ARB_TRY(d2h_sync(ctx, rq.data(), S.ss, k * sizeof(double)));
    std::vector<int32_t> perm(k);
    for (int i = 0; i < k; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(),
                     [&](int x, int y) { return S.smallest ? rq[x] < rq[y] : rq[x] > rq[y]; });
    if (evals)
      for (int i = 0; i < k; ++i) evals[i] = rq[perm[i]];
    if (evecs) {
      ARB_TRY(column_signs(ctx, n, D.Xall, D.ld, p, S.sgn));
      std::vector<double> hs(p);
      ARB_TRY(d2h_sync(ctx, hs.data(), S.sgn, p * sizeof(double)));
      std::vector<double> sgn_perm(k);
      for (int i = 0; i < k; ++i) sgn_perm[i] = hs[perm[i]];
      ARB_TRY(upload_ints(ctx, S.iidx, perm));
      ARB_TRY(h2d(ctx, S.res, sgn_perm.data(), k * sizeof(double)));
      if (evecs_on_device) {
        ARB_TRY(write_colmajor(ctx, n, D.Xall, D.ld, S.iidx, S.res, k, evecs, ldq));
      } else {
        // stage through a device block (W1 is free now), then one strided copy to the host
        ARB_TRY(write_colmajor(ctx, n, D.Xall, D.ld, S.iidx, S.res, k, D.W1, n));
        ARB_CUDA(ctx, cudaMemcpy2DAsync(evecs, ldq * sizeof(double), D.W1, n * sizeof(double), n * sizeof(double), k,
                                        cudaMemcpyDeviceToHost, ctx->stream));
      }
    }
    ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    S.info.t_total = total.sec();
    if (info_out) *info_out = S.info;
    const bool ok = (S.stop == ARB_STOP_CONVERGED || S.stop == ARB_STOP_NEAR_TOL);
    return ok ? ARB_OK : ARB_NOT_CONVERGED;
  }
};

arb_status solve_impl(arb_ctx ctx, arb_mat mat, int32_t k, arb_which which, double tol, const arb_options& o,
                      const double* x0, int x0_on_device, double* evals, double* evecs, int64_t ldq,
                      int evecs_on_device, arb_info* info_out) {
  Solve sv;
  sv.ctx = ctx;
  sv.mat = mat;
  ARB_TRY(sv.setup(k, which, tol, o, x0, x0_on_device, evecs, ldq));
  ARB_TRY(sv.run());
  return sv.finish(evals, evecs, ldq, evecs_on_device, info_out);
}

// ---------------------------------------------------------------- lock-step batched driver
// A context of the lock-step driver: the caller's device, its own stream and workspaces.
// A context of the lock-step driver: the caller's device, a stream of its own (or the given
// one) and workspaces of its own.  coop_share: the cooperative launches of this many such
// contexts may run at once (each grid takes 1/coop_share of the device).
arb_ctx make_sub_context(arb_ctx parent, cudaStream_t stream, int coop_share) {
  arb_ctx c = new arb_ctx_s();
  c->device = parent->device;
  c->num_sms = parent->num_sms;
  c->coop_share = std::max(1, coop_share);
  if (stream) {
    c->stream = stream;
    c->own_stream = false;
  } else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) == cudaSuccess) {
    c->own_stream = true;
  } else {
    delete c;
    return nullptr;
  }
  if (cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return nullptr;
  }
  return c;
}

void drop_sub_context(arb_ctx c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int i = 0; i < WS_NUM_SLOTS; ++i)
    if (c->ws[i]) cudaFree(c->ws[i]);
  if (c->host_pinned) cudaFreeHost(c->host_pinned);
  if (c->err_dev) cudaFree(c->err_dev);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

// host threads of the lock-step driver's worker pool (each instance's checks and ARR tails
// run on one of them, on the instance's own stream); 256 diffusion instances: 15.9 solves/s
// with 16, 15.6 with 32, 15.3 with 64 - a round waits for its slowest tail either way
#ifndef ARB_LOCKSTEP_WORKERS
#define ARB_LOCKSTEP_WORKERS 16
#endif

// A fixed pool of host threads running one parallel loop at a time: run(count, f) calls
// f(i) for i < count, spread over the workers, and returns when all calls have returned.
class WorkerPool {
 public:
  explicit WorkerPool(int n) {
    for (int t = 0; t < n; ++t) threads_.emplace_back([this] { work(); });
  }
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> l(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }
  void run(int count, const std::function<void(int)>& f) {
    if (count <= 0) return;
    std::unique_lock<std::mutex> l(mu_);
    f_ = &f;
    count_ = count;
    next_ = 0;
    left_ = count;
    ++gen_;
    cv_.notify_all();
    done_.wait(l, [this] { return left_ == 0; });
    f_ = nullptr;
  }

 private:
  void work() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> l(mu_);
    for (;;) {
      cv_.wait(l, [&] { return stop_ || gen_ != seen; });
      if (stop_) return;
      seen = gen_;
      while (next_ < count_) {
        const int i = next_++;
        const std::function<void(int)>* f = f_;
        l.unlock();
        (*f)(i);
        l.lock();
        if (--left_ == 0) done_.notify_all();
      }
    }
  }
  std::vector<std::thread> threads_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* f_ = nullptr;
  int count_ = 0, next_ = 0, left_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

// What the driver needs of the current phase of a solve, whatever its element type.
struct PhaseView {
  Solve* sv;
  template <typename F>
  auto with(F&& f) -> decltype(f(sv->p64)) {
    if (sv->stage == 0) return f(sv->p32);
    return f(sv->p64);
  }
};

// The filter job of the current inner step of an instance (its batched form).
template <typename T>
arb_filter_job job_of(const Phase<T>& ph) {
  const SolveState& S = *ph.S;
  arb_filter_job J{};
  J.mat = ph.mat;
  J.op_scale = S.op_scale;
  J.op_shift = S.op_shift;
  J.a = S.a;
  J.b = S.b;
  J.degree = S.d;
  J.fp32 = sizeof(T) == 4 ? 1 : 0;
  J.coef = S.coef;
  J.X = ph.B->X;
  J.ldx = ph.B->ld;
  J.ncols = S.w;
  J.xscale = S.xs;
  J.Y = ph.filter_out();
  J.ldy = ph.B->ld;
  J.colss = S.ss;
  return J;
}

// key of a round's captured graph: everything the recorded kernels bake in
std::string round_key(const BatchPlan& plan) {
  std::string key;
  auto put = [&](const void* p, size_t b) { key.append(static_cast<const char*>(p), b); };
  put(&plan.dj, sizeof(plan.dj));
  put(&plan.dp, sizeof(plan.dp));
  put(&plan.dmax, sizeof(plan.dmax));
  for (const auto& c : plan.cls) {
    put(&c.first, sizeof(c.first));
    put(&c.count, sizeof(c.count));
    put(&c.grid, sizeof(c.grid));
    put(&c.doff, sizeof(c.doff));
    put(&c.dcs, sizeof(c.dcs));
    put(&c.tickets, sizeof(c.tickets));
  }
  return key;
}

int64_t round_kernels(const BatchPlan& plan) {
  int64_t k = 0;
  for (const auto& c : plan.cls) k += c.count > 0 ? 1 : 0;
  return k;
}

}  // namespace

extern "C" arb_status arb_solve_lockstep(arb_ctx ctx, int32_t nb, const arb_mat* mats, const int32_t* k,
                                         const arb_which* which, const double* tol, const arb_options* opts,
                                         const double* const* x0, double* const* evals, double* const* evecs,
                                         const int64_t* ldq, arb_info* info, int32_t flags, arb_batch_stats* stats) {
  if (!ctx || nb < 0 || (nb > 0 && (!mats || !k || !which || !tol || !evals)) || (flags & ~3) != 0)
    return set_error(ctx, ARB_INVALID_ARG, "solve_lockstep: bad arguments");
  Timer total;
  arb_batch_stats bs{};
  if (nb == 0) {
    if (stats) *stats = bs;
    return ARB_OK;
  }
  for (int32_t i = 0; i < nb; ++i)
    if (!mats[i] || mats[i]->device != ctx->device)
      return set_error(ctx, ARB_INVALID_ARG, "solve_lockstep: matrix missing or on another device");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t stream = nullptr;
  ARB_CUDA(ctx, cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
  cudaEvent_t order = nullptr, kev0 = nullptr, kev1 = nullptr;
  cudaEventCreateWithFlags(&order, cudaEventDisableTiming);
  cudaEventCreate(&kev0);
  cudaEventCreate(&kev1);
  cudaEventRecord(order, ctx->stream);  // the caller's earlier work first
  cudaStreamWaitEvent(stream, order, 0);
  // the instances' per-instance work (inner stop checks, ARR tails, steps that do not join
  // the batch) runs on a pool of host threads, each instance on a stream of its own; their
  // cooperative launches (block Jacobi) share the device among the workers
  const int workers = std::max(1, std::min<int>(nb, ARB_LOCKSTEP_WORKERS));
  arb_ctx bctx = make_sub_context(ctx, stream, 1);  // the batched filter's workspaces and stream
  std::vector<arb_ctx> subs(nb, nullptr);
  std::vector<std::unique_ptr<Solve>> sv(nb);
  std::vector<arb_status> st(nb, ARB_OK);
  std::vector<bool> live(nb, false), in_outer(nb, false);
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
  };
  std::unordered_map<std::string, Graph> graphs;
  std::unordered_map<std::string, int> seen;
  bool graphs_ok = (flags & ARB_BATCH_GRAPHS) != 0;
  arb_status fatal = ARB_OK;
  auto cleanup = [&]() {
    for (auto& g : graphs)
      if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    sv.clear();
    for (arb_ctx c : subs) drop_sub_context(c);
    drop_sub_context(bctx);
    cudaStreamSynchronize(stream);
    cudaEventRecord(order, stream);  // the caller's later work after ours (the instances' streams are drained)
    cudaStreamWaitEvent(ctx->stream, order, 0);
    cudaEventDestroy(order);
    cudaEventDestroy(kev0);
    cudaEventDestroy(kev1);
    cudaStreamDestroy(stream);
  };
  // autotuned SpMM settings per distinct matrix (width of its first problem)
  if (flags & ARB_BATCH_AUTOTUNE) {
    for (int32_t i = 0; i < nb && fatal == ARB_OK; ++i) {
      if (mats[i]->tuned) continue;
      arb_options o;
      if (opts) o = opts[i];
      else arb_options_default(&o, k[i]);
      const int32_t p = o.p > 0 ? o.p : k[i] + static_cast<int32_t>(std::lround(0.1 * k[i]));
      fatal = arb_matrix_autotune(bctx, mats[i], p, nullptr, nullptr);
    }
    if (fatal != ARB_OK) {
      set_error(ctx, fatal, std::string("solve_lockstep: autotune: ") + bctx->last_error);
      cleanup();
      return fatal;
    }
  }
  // set-up and first phase of every instance
  for (int32_t i = 0; i < nb; ++i) {
    subs[i] = make_sub_context(ctx, nullptr, workers);
    if (!subs[i]) {
      st[i] = set_error(ctx, ARB_CUDA_ERROR, "solve_lockstep: stream creation");
      continue;
    }
    cudaStreamWaitEvent(subs[i]->stream, order, 0);
    sv[i].reset(new Solve());
    sv[i]->ctx = subs[i];
    sv[i]->mat = mats[i];
    arb_options o;
    if (opts) o = opts[i];
    else arb_options_default(&o, k[i]);
    st[i] = sv[i]->setup(k[i], which[i], tol[i], o, x0 ? x0[i] : nullptr, 0, evecs ? evecs[i] : nullptr,
                         ldq ? ldq[i] : mats[i]->n);
    if (st[i] == ARB_OK) st[i] = sv[i]->start();
    live[i] = st[i] == ARB_OK;
  }
  WorkerPool pool(workers);
  // the lock-step loop
  for (;;) {
    // phase transitions and the start of outer iterations
    bool any = false;
    for (int32_t i = 0; i < nb; ++i) {
      while (live[i] && !in_outer[i]) {
        Solve& s = *sv[i];
        if (s.stage >= 2) {
          live[i] = false;
          break;
        }
        PhaseView pv{&s};
        const bool ended = pv.with([](auto& ph) { return ph.done; });
        if (ended) {
          st[i] = s.phase_ended();
          if (st[i] != ARB_OK) live[i] = false;
          continue;
        }
        st[i] = pv.with([](auto& ph) { return ph.outer_begin(); });
        if (st[i] != ARB_OK) {
          live[i] = false;
          break;
        }
        if (!pv.with([](auto& ph) { return ph.done; })) in_outer[i] = true;
      }
      any = any || live[i];
    }
    if (!any) break;
    // one inner step of every instance whose inner loop runs: the batchable ones together,
    // the others alone on the worker pool
    std::vector<arb_filter_job> jobs;
    std::vector<int32_t> who, alone;
    for (int32_t i = 0; i < nb; ++i) {
      if (!live[i] || !in_outer[i]) continue;
      PhaseView pv{sv[i].get()};
      if (!pv.with([](auto& ph) { return ph.step_due(); })) continue;
      if (pv.with([](auto& ph) { return ph.batchable(); })) {
        jobs.push_back(pv.with([](auto& ph) { return job_of(ph); }));
        who.push_back(i);
      } else {
        alone.push_back(i);
      }
    }
    Timer t_single;
    pool.run(static_cast<int>(alone.size()), [&](int t) {
      const int32_t i = alone[t];
      PhaseView pv{sv[i].get()};
      st[i] = pv.with([](auto& ph) { return ph.step(); });
    });
    for (int32_t i : alone) {
      bs.single_steps++;
      if (st[i] != ARB_OK) live[i] = false;
    }
    bs.t_single += t_single.sec();
    if (!jobs.empty()) {
      Timer t_batch;
      // the batch reads the instances' blocks: their streams' work first
      for (int32_t i : who) {
        cudaEventRecord(subs[i]->ev_join, subs[i]->stream);
        cudaStreamWaitEvent(stream, subs[i]->ev_join, 0);
      }
      BatchPlan plan;
      Timer t_prep;
      fatal = filter_batched_prepare(bctx, static_cast<int32_t>(jobs.size()), jobs.data(), &plan);
      if (fatal != ARB_OK) break;
      bs.t_prepare += t_prep.sec();
      cudaEventRecord(kev0, stream);
      bool ran = false;
      if (graphs_ok) {
        const std::string key = round_key(plan);
        auto g = graphs.find(key);
        if (g != graphs.end()) {
          if (cudaGraphLaunch(g->second.exec, stream) == cudaSuccess) {
            bctx->launches += g->second.kernels;
            bs.graph_launches++;
            ran = true;
          } else {
            cudaGetLastError();
            graphs_ok = false;
          }
        } else if (++seen[key] >= 2) {
          // the second occurrence of this round shape: its workspaces exist, capture it
          cudaGraph_t graph = nullptr;
          bool captured = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
          arb_status ls = ARB_OK;
          if (captured) {
            const int64_t l0 = bctx->launches;
            ls = filter_batched_launch(bctx, plan);
            bctx->launches = l0;
            captured = cudaStreamEndCapture(stream, &graph) == cudaSuccess && ls == ARB_OK && graph;
          }
          Graph gx;
          if (captured && cudaGraphInstantiate(&gx.exec, graph, 0) == cudaSuccess &&
              cudaGraphLaunch(gx.exec, stream) == cudaSuccess) {
            gx.kernels = round_kernels(plan);
            bctx->launches += gx.kernels;
            graphs[key] = gx;
            bs.graphs_captured++;
            bs.graph_launches++;
            ran = true;
          } else {
            // capture is not available here: run the rounds directly from now on
            if (gx.exec) cudaGraphExecDestroy(gx.exec);
            cudaGetLastError();
            graphs_ok = false;
          }
          if (graph) cudaGraphDestroy(graph);
        }
      }
      if (!ran) {
        fatal = filter_batched_launch(bctx, plan);
        if (fatal != ARB_OK) break;
      }
      bs.batched_launches++;
      bs.batched_jobs += static_cast<int64_t>(jobs.size());
      cudaEventRecord(kev1, stream);
      // and the instances' next work reads its results; the batch ends before the workers'
      // cooperative launches start, so those never share the device with it
      cudaEventRecord(bctx->ev_join, stream);
      for (int32_t i : who) {
        cudaStreamWaitEvent(subs[i]->stream, bctx->ev_join, 0);
        PhaseView pv{sv[i].get()};
        st[i] = pv.with([](auto& ph) { return ph.step_post_external(); });
        if (st[i] != ARB_OK) live[i] = false;
      }
      if (cudaStreamSynchronize(stream) != cudaSuccess) {
        fatal = cuda_error(bctx, cudaGetLastError(), "batched filter", __FILE__, __LINE__);
        break;
      }
      bs.t_batched += t_batch.sec();
      float kms = 0.f;
      if (cudaEventElapsedTime(&kms, kev0, kev1) == cudaSuccess) bs.t_batch_kernel += kms * 1e-3;
    }
    bs.rounds++;
    // inner stop checks, then the ARR tails of the instances whose inner loop has ended,
    // on the worker pool
    std::vector<int32_t> busy;
    for (int32_t i = 0; i < nb; ++i)
      if (live[i] && in_outer[i]) busy.push_back(i);
    std::vector<char> tail_done(nb, 0);
    Timer t_checks;
    pool.run(static_cast<int>(busy.size()), [&](int t) {
      const int32_t i = busy[t];
      PhaseView pv{sv[i].get()};
      const bool due = pv.with([](auto& ph) { return ph.in_inner && !ph.step_due(); });
      if (due) {
        st[i] = pv.with([](auto& ph) { return ph.check(); });
        if (st[i] != ARB_OK) return;
      }
      if (!pv.with([](auto& ph) { return ph.in_inner; })) {
        st[i] = pv.with([](auto& ph) { return ph.outer_tail(); });
        tail_done[i] = 1;
      }
    });
    bs.t_checks += t_checks.sec();
    for (int32_t i : busy) {
      if (tail_done[i]) in_outer[i] = false;
      if (st[i] != ARB_OK) live[i] = false;
    }
  }
  if (fatal != ARB_OK) {
    set_error(ctx, fatal, std::string("solve_lockstep: batched filter: ") + bctx->last_error);
    ctx->launches += bctx->launches;
    cleanup();
    return fatal;
  }
  // outputs
  pool.run(nb, [&](int i) {
    if (st[i] == ARB_OK)
      st[i] = sv[i]->finish(evals[i], evecs ? evecs[i] : nullptr, ldq ? ldq[i] : mats[i]->n, 0,
                            info ? &info[i] : nullptr);
  });
  arb_status worst = ARB_OK;
  for (int32_t i = 0; i < nb; ++i) {
    if (st[i] != ARB_OK && subs[i]) {
      set_error(ctx, st[i], std::string("solve_lockstep: instance ") + std::to_string(i) + ": " + subs[i]->last_error);
    }
    if (st[i] != ARB_OK && (worst == ARB_OK || (worst == ARB_NOT_CONVERGED && st[i] < 0))) worst = st[i];
    if (subs[i]) ctx->launches += subs[i]->launches;
  }
  ctx->launches += bctx->launches;
  bs.t_total = total.sec();
  if (stats) *stats = bs;
  cleanup();
  return worst;
}

namespace {

}  // namespace

size_t arb::solve_footprint(int64_t n, int64_t nnz, int32_t p, int32_t q, int32_t precision) {
  const bool mixed = (precision == ARB_MIXED || precision == ARB_MIXED_DF);
  const int64_t ld = p + (p & 1), ldm = static_cast<int64_t>(q + 1) * p + (((q + 1) * p) & 1);
  const int64_t mcap = static_cast<int64_t>(q + 1) * p;
  size_t b = static_cast<size_t>(n) * (7 * ld + 2 * ldm) * sizeof(double);
  if (mixed) {
    const int64_t l4 = (p + 3) / 4 * 4, m4 = (mcap + 3) / 4 * 4;
    b += static_cast<size_t>(n) * (6 * l4 + 2 * m4) * sizeof(float) + static_cast<size_t>(nnz) * sizeof(float);
  }
  if (precision == ARB_MIXED_DF) b += static_cast<size_t>(nnz) * 2 * sizeof(float);  // double-float values of A
  // small dense state (H, eigenvectors, Gram matrices, Jacobi copies), split-K and column
  // reduction partial sums: bounded by a few m x m matrices plus one slab of partials
  b += static_cast<size_t>(8 * mcap * mcap + 2048 * mcap) * sizeof(double) + (64u << 20);
  return b;
}

extern "C" arb_status arb_solve(arb_ctx ctx, arb_mat mat, int32_t k, arb_which which, double tol,
                                const arb_options* opts, const double* x0, int x0_on_device, double* evals,
                                double* evecs, int64_t ldq, int evecs_on_device, arb_info* info) {
  return arb::solve_on(ctx, mat, k, which, tol, opts, x0, x0_on_device, evals, evecs, ldq, evecs_on_device, info);
}

arb_status arb::solve_on(arb_ctx ctx, arb_mat mat, int32_t k, arb_which which, double tol, const arb_options* opts,
                         const double* x0, int x0_on_device, double* evals, double* evecs, int64_t ldq,
                         int evecs_on_device, arb_info* info) {
  if (!ctx || !mat || mat->device != ctx->device)
    return set_error(ctx, ARB_INVALID_ARG, "solve: bad context or matrix (matrix on another device)");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  arb_options o;
  if (opts) {
    o = *opts;
  } else {
    arb_options_default(&o, k);
  }
  return solve_impl(ctx, mat, k, which, tol, o, x0, x0_on_device, evals, evecs, ldq, evecs_on_device, info);
}
