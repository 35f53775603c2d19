// Gram product for callers that cannot allocate device memory.
//
// arb_gram's split-K partial sums normally live in a workspace the context allocates on
// first use.  Some callers cannot let a library call cudaMalloc: applications whose device
// memory is owned by their own pool allocator (it may hold all free memory, and it must
// account for every allocation), and latency-critical loops that must not hit the
// implicit synchronisation of cudaMalloc/cudaFree.  arb_gram_noalloc serves them: its
// partial sums go to a file-scope device array that exists as long as the library is
// loaded, so the call itself allocates nothing.
#include <mutex>

#include "arb_internal.h"

namespace {

// 1,048,576 doubles = 8 MiB of partial sums, held on every device that loads the library.
constexpr size_t kScratchDoubles = size_t(1) << 20;
__device__ __align__(256) double g_gram_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on `device` (which must be current).  Host code
// only ever holds a stand-in for the symbol, so the real address is looked up once per
// device and cached.
arb_status scratch_address(arb_ctx ctx, int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return arb::set_error(ctx, ARB_INVALID_ARG, "gram_noalloc: device id");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) return arb::cuda_error(ctx, e, "cudaGetSymbolAddress(g_gram_scratch)", __FILE__, __LINE__);
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return ARB_OK;
}

}  // namespace

extern "C" arb_status arb_gram_noalloc(arb_ctx ctx, int64_t n, const double* X, int64_t ldx, int32_t na,
                                       const double* Y, int64_t ldy, int32_t nb, double* C, int64_t ldc) {
  if (!ctx || n < 1 || na < 1 || nb < 1 || !X || !Y || !C || ldx < na || ldy < nb || ldc < nb)
    return arb::set_error(ctx, ARB_INVALID_ARG, "gram_noalloc: bad arguments");
  if (static_cast<size_t>(na) * static_cast<size_t>(nb) > kScratchDoubles)
    return arb::set_error(ctx, ARB_INVALID_ARG,
                          "gram_noalloc: na * nb exceeds the 1048576-double static scratch (use arb_gram)");
  ARB_CUDA(ctx, cudaSetDevice(ctx->device));
  double* part = nullptr;
  ARB_TRY(scratch_address(ctx, ctx->device, &part));
  return arb::gram_into(ctx, n, X, ldx, na, Y, ldy, nb, C, ldc, part, kScratchDoubles);
}
