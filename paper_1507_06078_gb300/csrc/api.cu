// C ABI of the library: contexts, matrices, the step entry points and the Algorithm 8
// driver (ARRABIT with the multi-power inner solver).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
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
      ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      ARB_CUDA(ctx, cudaFree(ctx->ws[slot]));
      ctx->ws[slot] = nullptr;
      ctx->ws_bytes[slot] = 0;
    }
    void* p = nullptr;
    ARB_CUDA(ctx, cudaMalloc(&p, bytes));
    ctx->ws[slot] = p;
    ctx->ws_bytes[slot] = bytes;
  }
  *out = ctx->ws[slot];
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

arb_status d2h_sync(arb_ctx ctx, void* host, const void* dev, size_t bytes) {
  void* st;
  ARB_TRY(host_stage(ctx, std::max<size_t>(bytes, 4096), &st));
  ARB_CUDA(ctx, cudaMemcpyAsync(st, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(host, st, bytes);
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

extern "C" arb_status arb_ctx_destroy(arb_ctx ctx) {
  if (!ctx) return ARB_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < WS_NUM_SLOTS; ++i)
    if (ctx->ws[i]) cudaFree(ctx->ws[i]);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
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

extern "C" arb_status arb_matrix_create_csr(arb_ctx ctx, int64_t n, int64_t nnz, const int32_t* rowptr,
                                            const int32_t* col, const double* val, int ptr_on_device,
                                            arb_mat* out) {
  if (!ctx || !out || n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val)))
    return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: bad arguments");
  if (n > INT32_MAX || nnz > INT32_MAX)
    return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: int32 index range exceeded");
  *out = nullptr;
  if (!ptr_on_device) {
    if (rowptr[0] != 0 || rowptr[n] != nnz)
      return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: rowptr must start at 0 and end at nnz");
    for (int64_t i = 0; i < n; ++i)
      if (rowptr[i + 1] < rowptr[i]) return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: rowptr decreasing");
    for (int64_t e = 0; e < nnz; ++e)
      if (col[e] < 0 || col[e] >= n) return set_error(ctx, ARB_INVALID_ARG, "matrix_create_csr: column out of range");
  }
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  arb_mat m = new arb_mat_s();
  m->ctx = ctx;
  m->device = ctx->device;
  m->n = n;
  m->nnz = nnz;
  const cudaMemcpyKind kind = ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMalloc(&m->rowptr, (n + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->col, std::max<int64_t>(nnz, 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->val, std::max<int64_t>(nnz, 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->rowptr, rowptr, (n + 1) * sizeof(int32_t), kind, ctx->stream);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(m->col, col, nnz * sizeof(int32_t), kind, ctx->stream);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(m->val, val, nnz * sizeof(double), kind, ctx->stream);
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

extern "C" arb_status arb_matrix_destroy(arb_mat m) {
  if (!m) return ARB_INVALID_ARG;
  // the creating context may already be gone: use only what the matrix owns
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  cudaFree(m->rowptr);
  cudaFree(m->col);
  cudaFree(m->val);
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
  return filter_apply(ctx, mat, plan, X, ldx, ncols, xscale, W1, W2, ldw, Y, ldy, colss, nullptr);
}

extern "C" arb_status arb_spmm(arb_ctx ctx, arb_mat mat, double op_scale, double op_shift, const double* X,
                               int64_t ldx, int32_t ncols, double* Y, int64_t ldy) {
  if (!ctx || !mat || !X || !Y || ncols < 0 || ldx < ncols || ldy < ncols)
    return set_error(ctx, ARB_INVALID_ARG, "spmm: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  SpmmArgs s;
  s.A = mat;
  s.ncols = ncols;
  s.Yin = X;
  s.ldy = ldx;
  s.alpha = op_scale;
  s.beta = op_shift;
  s.out = Y;
  s.ldo = ldy;
  return spmm_fused(ctx, s);
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
  return gram(ctx, n, X, ldx, na, Y, ldy, nb, C, ldc);
}

extern "C" arb_status arb_syevj(arb_ctx ctx, int32_t m, const double* H, int64_t ldh, double* w, double* V,
                                int64_t ldv, int32_t* sweeps) {
  if (!ctx || m < 0 || (m > 0 && (!H || !w || !V || ldh < m || ldv < m)))
    return set_error(ctx, ARB_INVALID_ARG, "syevj: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  return syevj(ctx, m, H, ldh, w, V, ldv, sweeps);
}

extern "C" arb_status arb_rcond_gram(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t ncols,
                                     const double* xscale, double* rc) {
  if (!ctx || n <= 0 || !X || ncols <= 0 || ldx < ncols || !rc)
    return set_error(ctx, ARB_INVALID_ARG, "rcond_gram: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  return rcond_gram(ctx, n, X, ldx, ncols, xscale, rc);
}

extern "C" arb_status arb_orth(arb_ctx ctx, int64_t n, const double* Z, int64_t ldz, int32_t m, double* U,
                               int64_t ldu, int32_t* rank) {
  if (!ctx || n <= 0 || !Z || m < 0 || ldz < m || !U || ldu < m || !rank)
    return set_error(ctx, ARB_INVALID_ARG, "orth: bad arguments");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  double* tmp;
  ARB_TRY(ws<double>(ctx, WS_TALL0, static_cast<size_t>(n) * std::max(m, 1), &tmp));
  return orth(ctx, n, Z, ldz, m, U, ldu, tmp, std::max(m, 1), rank);
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
  ARB_TRY(orth(ctx, n, Z, ldz, m, U, m, tmp, m, &r));
  *rank = r;
  if (r == 0) return ARB_OK;
  SpmmArgs s;
  s.A = mat;
  s.ncols = r;
  s.Yin = U;
  s.ldy = m;
  s.alpha = op_scale;
  s.beta = op_shift;
  s.out = AU;
  s.ldo = m;
  ARB_TRY(spmm_fused(ctx, s));
  ARB_TRY(ws<double>(ctx, WS_S_V, static_cast<size_t>(r) * r, &H));
  ARB_TRY(ws<double>(ctx, WS_S_VSEL, static_cast<size_t>(r) * r, &V));
  ARB_TRY(gram(ctx, n, U, m, r, AU, m, r, H, r));
  ARB_TRY(symmetrize(ctx, r, H, r));
  ARB_TRY(syevj(ctx, r, H, r, w, V, r, nullptr));
  return gemm_tall(ctx, n, U, m, r, V, r, r, 1.0, 0.0, Y, ldy);
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
  ArrWork wk;
  double* Xc;
  ARB_TRY(ws<double>(ctx, WS_TALL0, static_cast<size_t>(n) * ldw, &Xc));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_U, static_cast<size_t>(n) * ldm, &wk.U));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_AU, static_cast<size_t>(n) * ldm, &wk.AU));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_T, static_cast<size_t>(n) * ldw, &wk.T));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_T2, static_cast<size_t>(n) * ldw, &wk.T2));
  wk.ldu = wk.ldau = ldm;
  wk.ldt = wk.ldt2 = ldw;
  ARB_TRY(copy_block(ctx, n, X, ldx, ncols, Xc, ldw));
  double *theta, *V;
  ARB_TRY(ws<double>(ctx, WS_S_VEC, static_cast<size_t>(mcap), &theta));
  ARB_TRY(ws<double>(ctx, WS_S_V, static_cast<size_t>(mcap) * mcap, &V));
  int32_t m = 0;
  ARB_TRY(arr_basis_and_eig(ctx, mat, op_scale, op_shift, n, Xc, ldw, ncols, nullptr, 0, 0, q, wk, &m,
                            theta, V));
  *rank = m;
  if (m < npairs) return set_error(ctx, ARB_BREAKDOWN, "arr: subspace smaller than the requested pairs");
  ARB_CUDA(ctx, cudaMemcpyAsync(w, theta, npairs * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return gemm_tall(ctx, n, wk.U, ldm, m, V, m, npairs, 1.0, 0.0, Y, ldy);
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

arb_status solve_impl(arb_ctx ctx, arb_mat mat, int32_t k, arb_which which, double tol, const arb_options& o,
                      const double* x0, int x0_on_device, double* evals, double* evecs, int64_t ldq,
                      int evecs_on_device, arb_info* info_out) {
  Timer total;
  arb_info info;
  memset(&info, 0, sizeof(info));
  const int64_t n = mat->n;
  const int32_t p = o.p > 0 ? o.p : k + static_cast<int32_t>(std::lround(0.1 * k));
  const int32_t q = o.q, d = o.degree;
  if (k <= 0 || k > p || q < 0 || d < 1 || d > 60 || o.maxit < 1 || o.maxit1 < 1 || o.maxit2 < 1 ||
      static_cast<int64_t>(q + 1) * p >= n || !(tol > 0.0))
    return set_error(ctx, ARB_INVALID_ARG, "solve: need 0 < k <= p, (q+1) p < n, 1 <= degree <= 60, tol > 0");
  if (o.precision != ARB_FP64) return set_error(ctx, ARB_INVALID_ARG, "solve: only ARB_FP64 is implemented");
  if (which != ARB_LARGEST && which != ARB_SMALLEST) return set_error(ctx, ARB_INVALID_ARG, "solve: bad which");
  if (evecs && ldq < n) return set_error(ctx, ARB_INVALID_ARG, "solve: ldq < n");
  const bool smallest = (which == ARB_SMALLEST);

  // operator B = op_scale A + op_shift I whose largest eigenpairs are wanted
  double glo, ghi;
  ARB_TRY(gershgorin(ctx, mat, &glo, &ghi));
  double sigma = 0.0, op_scale = 1.0, op_shift = 0.0, a;
  if (smallest) {
    sigma = std::isnan(o.shift_sigma) ? ghi : o.shift_sigma;
    op_scale = -1.0;
    op_shift = sigma;
    a = sigma - ghi;  // Gershgorin lower bound of sigma I - A
  } else {
    a = glo;
  }

  // device buffers
  const int64_t ld = p + (p & 1);
  const int64_t mcap = static_cast<int64_t>(q + 1) * p;
  const int64_t ldm = mcap + (mcap & 1);
  const size_t blk = static_cast<size_t>(n) * ld;
  double *bufX, *bufW1, *bufW2, *Qc, *Xall;
  ArrWork wk;
  ARB_TRY(ws<double>(ctx, WS_SOLVER_X, blk, &bufX));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_W1, blk, &bufW1));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_W2, blk, &bufW2));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_QC, blk, &Qc));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_XALL, blk, &Xall));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_U, static_cast<size_t>(n) * ldm, &wk.U));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_AU, static_cast<size_t>(n) * ldm, &wk.AU));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_T, blk, &wk.T));
  ARB_TRY(ws<double>(ctx, WS_SOLVER_T2, blk, &wk.T2));
  wk.ldu = wk.ldau = ldm;
  wk.ldt = wk.ldt2 = ld;
  double *V, *Vsel, *vec;
  ARB_TRY(ws<double>(ctx, WS_S_V, static_cast<size_t>(mcap) * mcap, &V));
  ARB_TRY(ws<double>(ctx, WS_S_VSEL, static_cast<size_t>(mcap) * p, &Vsel));
  // vec layout: theta[mcap] | mu[p] | sigc[p] | ss[p] | res[p] | xs[p] | negmu... | ints
  ARB_TRY(ws<double>(ctx, WS_S_VEC, static_cast<size_t>(mcap) + 8 * static_cast<size_t>(p) + 64, &vec));
  double* theta = vec;
  double* mu = theta + mcap;
  double* sigc = mu + p;
  double* ss = sigc + p;
  double* res = ss + p;
  double* xs = res + p;
  int32_t* imap = reinterpret_cast<int32_t*>(xs + p);       // p ints
  int32_t* iidx = imap + p + (p & 1);                          // p ints
  double* sgn = reinterpret_cast<double*>(iidx + p + (p & 1)); // p doubles

  // start block X0 (Algorithm 8: i.i.d. Gaussian n x (k+q))
  if (x0) {
    ARB_CUDA(ctx, cudaMemcpy2DAsync(bufX, ld * sizeof(double), x0, p * sizeof(double), p * sizeof(double), n,
                                    x0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    ctx->stream));
  } else {
    ARB_TRY(gaussian_fill(ctx, n, p, o.seed, bufX, ld));
  }

  // b: smallest Ritz value of orth(X0) (Section 5, "Estimation of lambda_n and lambda_{k+q}")
  double b;
  {
    int32_t r = 0;
    ARB_TRY(orth(ctx, n, bufX, ld, p, wk.U, ldm, wk.T, ld, &r));
    if (r == 0) return set_error(ctx, ARB_BREAKDOWN, "solve: start block has no numerical rank");
    SpmmArgs s;
    s.A = mat;
    s.ncols = r;
    s.Yin = wk.U;
    s.ldy = ldm;
    s.alpha = op_scale;
    s.beta = op_shift;
    s.out = wk.AU;
    s.ldo = ldm;
    ARB_TRY(spmm_fused(ctx, s));
    double* H;
    ARB_TRY(ws<double>(ctx, WS_SMALL0, static_cast<size_t>(r) * r, &H));
    ARB_TRY(gram(ctx, n, wk.U, ldm, r, wk.AU, ldm, r, H, r));
    ARB_TRY(symmetrize(ctx, r, H, r));
    ARB_TRY(syevj(ctx, r, H, r, theta, V, r, nullptr));
    ARB_TRY(d2h_sync(ctx, &b, theta + (r - 1), sizeof(double)));
    info.spmm_cols += r;
  }
  info.a = a;
  info.b0 = b;
  info.sigma = sigma;
  if (!(b > a)) b = a + 1e-3 * std::max(1.0, std::fabs(a));  // degenerate start: keep the map defined

  double coef[64];
  ARB_TRY(arb_filter_coefficients(o.filter, d, coef) == ARB_OK ? ARB_OK
                                                                 : set_error(ctx, ARB_INVALID_ARG, "bad filter"));
  const double tol1 = o.tol1 > 0.0 ? o.tol1 : (tol <= 1e-8 ? std::max(1e-6, tol) : tol);
  double tol_t = std::max(tol1, tol);

  double* X = bufX;
  double* W1 = bufW1;
  double* W2 = bufW2;
  int32_t w = p, nl = 0;
  std::vector<double> h_sigc;  // locked Ritz values (host mirror)
  ARB_TRY(fill(ctx, xs, w, 1.0));
  double best = std::numeric_limits<double>::infinity();
  int best_iter = 0;
  int stop = ARB_STOP_MAXIT;
  std::vector<double> h_mu(p), h_res(p);
  std::vector<int32_t> h_map(p);
  int j = 0;
  cudaEvent_t ev0, ev1;
  ARB_CUDA(ctx, cudaEventCreate(&ev0));
  ARB_CUDA(ctx, cudaEventCreate(&ev1));
  for (j = 1; j <= o.maxit; ++j) {
    // ---------------- inner loop: multi-power steps (Algorithm 8, MPM branch)
    ARB_CUDA(ctx, cudaEventRecord(ev0, ctx->stream));
    double rc = std::numeric_limits<double>::infinity();
    const int n_outer_checks = o.inner_fixed > 0 ? 1 : o.maxit1;
    const int n_steps = o.inner_fixed > 0 ? o.inner_fixed : o.maxit2;
    for (int i1 = 0; i1 < n_outer_checks; ++i1) {
      for (int i2 = 0; i2 < n_steps; ++i2) {
        const FilterPlan plan = make_filter_plan(op_scale, op_shift, a, b, d, coef);
        double* result = nullptr;
        ARB_TRY(filter_apply(ctx, mat, plan, X, ld, w, xs, W1, W2, ld, nullptr, 0, ss, &result));
        // the result lives in W1 or W2: rotate the three buffers
        if (result == W1) std::swap(X, W1);
        else std::swap(X, W2);
        ARB_TRY(inv_sqrt(ctx, w, ss, xs));  // column normalisation, applied lazily
        if (nl > 0) ARB_TRY(project_out(ctx, n, Qc, ld, nl, X, ld, w));
        info.n_filters++;
        info.spmm_cols += static_cast<int64_t>(d) * w;
      }
      if (o.inner_fixed > 0) break;
      const double rcp = rc;
      ARB_TRY(rcond_gram(ctx, n, X, ld, w, xs, &rc));
      if (rc <= tol_t || rc / rcp > 0.99) break;  // eq. inn-stop
    }
    ARB_CUDA(ctx, cudaEventRecord(ev1, ctx->stream));
    ARB_CUDA(ctx, cudaEventSynchronize(ev1));
    float ms = 0.f;
    ARB_CUDA(ctx, cudaEventElapsedTime(&ms, ev0, ev1));
    info.t_filter += ms * 1e-3;

    // ---------------- augmentation + projection + RR (Algorithm 5 inside Algorithm 8)
    ARB_CUDA(ctx, cudaEventRecord(ev0, ctx->stream));
    int32_t m = 0;
    ARB_TRY(arr_basis_and_eig(ctx, mat, op_scale, op_shift, n, X, ld, w, Qc, ld, nl, q, wk, &m, theta, V));
    info.last_rank = m;
    info.spmm_cols += m;
    // the p leading pairs of (Q_c, Sigma_c) and (U V, theta)
    ARB_TRY(select_top(ctx, sigc, nl, theta, m, p, imap, mu));
    ARB_TRY(d2h_sync(ctx, h_map.data(), imap, p * sizeof(int32_t)));
    for (int s = 0; s < p; ++s)
      if (h_map[s] < 0) return set_error(ctx, ARB_BREAKDOWN, "solve: fewer Ritz pairs than the block width");
    std::vector<int32_t> newcols, src(p);
    for (int s = 0; s < p; ++s) {
      if (h_map[s] < nl) {
        src[s] = -h_map[s] - 1;  // locked column
      } else {
        src[s] = static_cast<int32_t>(newcols.size());
        newcols.push_back(h_map[s] - nl);
      }
    }
    const int32_t pn = static_cast<int32_t>(newcols.size());
    if (pn > 0) {
      ARB_TRY(upload_ints(ctx, iidx, newcols));
      // V is m x m with leading dimension m (see arr_basis_and_eig call: ldv = m)
      ARB_TRY(gather_cols(ctx, m, V, m, iidx, pn, Vsel, pn));
      ARB_TRY(gemm_tall(ctx, n, wk.U, ldm, m, Vsel, pn, pn, 1.0, 0.0, wk.T, ld));
    }
    ARB_TRY(upload_ints(ctx, imap, src));
    ARB_TRY(gather_cols2(ctx, n, wk.T, ld, Qc, ld, imap, p, Xall, ld));
    // residuals (eq. resi): ||B x - mu x|| with the sign folded (-B x + mu x)
    {
      SpmmArgs s;
      s.A = mat;
      s.ncols = p;
      s.Yin = Xall;
      s.ldy = ld;
      s.alpha = -op_scale;
      s.beta = -op_shift;
      s.X = Xall;
      s.ldx = ld;
      s.sx = mu;
      s.colred = ss;
      ARB_TRY(spmm_fused(ctx, s));
      ARB_TRY(residual_finish(ctx, p, ss, mu, smallest ? 1 : 0, sigma, res));
      info.spmm_cols += p;
    }
    ARB_TRY(d2h_sync(ctx, h_mu.data(), mu, p * sizeof(double)));
    ARB_TRY(d2h_sync(ctx, h_res.data(), res, p * sizeof(double)));
    ARB_CUDA(ctx, cudaEventRecord(ev1, ctx->stream));
    ARB_CUDA(ctx, cudaEventSynchronize(ev1));
    ARB_CUDA(ctx, cudaEventElapsedTime(&ms, ev0, ev1));
    info.t_arr += ms * 1e-3;

    // ---------------- outer stop rules, continuation, deflation (Section 5)
    double maxres = 0.0;
    int h = 0;
    for (int i = 0; i < k; ++i) {
      maxres = std::max(maxres, std::isnan(h_res[i]) ? std::numeric_limits<double>::infinity() : h_res[i]);
      h += h_res[i] < 0.1 * tol;
    }
    info.maxres = maxres;
    if (maxres < best) {
      best = maxres;
      best_iter = j;
    }
    if (maxres <= tol) {
      stop = ARB_STOP_CONVERGED;
      break;
    }
    if (maxres < (1.0 + 9.0 * h / k) * tol) {
      stop = ARB_STOP_NEAR_TOL;
      break;
    }
    if (j - best_iter >= 3) {
      stop = ARB_STOP_STALLED;
      break;
    }
    if (maxres <= tol_t) {  // continuation, eq. contin
      tol_t = std::max(1e-2 * tol_t, tol);
      b = h_mu[p - 1];
      if (!(b > a)) b = a + 1e-3 * std::max(1.0, std::fabs(a));
    }
    const double thr = std::max(1e-14, tol_t * tol_t);  // eq. defl
    std::vector<int32_t> lock_idx, free_idx;
    h_sigc.clear();
    for (int s = 0; s < p; ++s) {
      if (s < k && h_res[s] <= thr) {
        lock_idx.push_back(s);
        h_sigc.push_back(h_mu[s]);
      } else {
        free_idx.push_back(s);
      }
    }
    nl = static_cast<int32_t>(lock_idx.size());
    w = p - nl;
    if (w == 0) {
      stop = ARB_STOP_ALL_LOCKED;
      break;
    }
    if (nl > 0) {
      ARB_TRY(upload_ints(ctx, iidx, lock_idx));
      ARB_TRY(gather_cols(ctx, n, Xall, ld, iidx, nl, Qc, ld));
      ARB_TRY(h2d(ctx, sigc, h_sigc.data(), nl * sizeof(double)));
    }
    ARB_TRY(upload_ints(ctx, iidx, free_idx));
    ARB_TRY(gather_cols(ctx, n, Xall, ld, iidx, w, X, ld));
    ARB_TRY(fill(ctx, xs, w, 1.0));
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  info.outer_iters = std::min(j, o.maxit);
  info.stop_reason = stop;
  info.b_final = b;
  info.n_locked = nl;

  // ---------------- outputs: Rayleigh quotients on A, order, sign, column-major copy
  {
    SpmmArgs s;
    s.A = mat;
    s.ncols = k;
    s.Yin = Xall;
    s.ldy = ld;
    s.alpha = 1.0;
    s.beta = 0.0;
    s.colred = ss;
    s.dot_with_yin = true;
    ARB_TRY(spmm_fused(ctx, s));
    info.spmm_cols += k;
  }
  std::vector<double> rq(k);
  ARB_TRY(d2h_sync(ctx, rq.data(), ss, k * sizeof(double)));
  std::vector<int32_t> perm(k);
  for (int i = 0; i < k; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return smallest ? rq[x] < rq[y] : rq[x] > rq[y]; });
  if (evals)
    for (int i = 0; i < k; ++i) evals[i] = rq[perm[i]];
  if (evecs) {
    ARB_TRY(column_signs(ctx, n, Xall, ld, p, sgn));
    std::vector<double> hs(p);
    ARB_TRY(d2h_sync(ctx, hs.data(), sgn, p * sizeof(double)));
    std::vector<double> sgn_perm(k);
    for (int i = 0; i < k; ++i) sgn_perm[i] = hs[perm[i]];
    ARB_TRY(upload_ints(ctx, iidx, perm));
    ARB_TRY(h2d(ctx, res, sgn_perm.data(), k * sizeof(double)));
    if (evecs_on_device) {
      ARB_TRY(write_colmajor(ctx, n, Xall, ld, iidx, res, k, evecs, ldq));
    } else {
      // stage through a device block (W1 is free now), then one strided copy to the host
      ARB_TRY(write_colmajor(ctx, n, Xall, ld, iidx, res, k, W1, n));
      ARB_CUDA(ctx, cudaMemcpy2DAsync(evecs, ldq * sizeof(double), W1, n * sizeof(double), n * sizeof(double), k,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    }
  }
  ARB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  info.t_total = total.sec();
  if (info_out) *info_out = info;
  const bool ok = (stop == ARB_STOP_CONVERGED || stop == ARB_STOP_NEAR_TOL);
  return ok ? ARB_OK : ARB_NOT_CONVERGED;
}

}  // namespace

extern "C" arb_status arb_solve(arb_ctx ctx, arb_mat mat, int32_t k, arb_which which, double tol,
                                const arb_options* opts, const double* x0, int x0_on_device, double* evals,
                                double* evecs, int64_t ldq, int evecs_on_device, arb_info* info) {
  if (!ctx || !mat || mat->ctx != ctx) return set_error(ctx, ARB_INVALID_ARG, "solve: bad context or matrix");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  arb_options o;
  if (opts) {
    o = *opts;
  } else {
    arb_options_default(&o, k);
  }
  return solve_impl(ctx, mat, k, which, tol, o, x0, x0_on_device, evals, evecs, ldq, evecs_on_device, info);
}
