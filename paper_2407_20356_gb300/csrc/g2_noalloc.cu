// g2 over a stored two-time matrix with no device allocation at call time.
//
// Same computation and kernels as xpcs_g2 (ring-averaged g2 from the lower triangle of
// C), but the per-split partial sums live in one fixed array of this module instead of
// the context's scratch, which xpcs_g2 grows with cudaMalloc on demand.  It is meant for
// callers that must not allocate device memory while they run: a loop that has already
// handed all of its HBM to other streams under a budget, or a latency-bound loop that
// cannot take the device-wide synchronisation a cudaFree may imply.
//
// The first call on each device does the set-up (looks up the array's device address and
// loads the two kernels into the context, either of which the runtime may do by
// allocating); make that first call at start-up, before any stream capture and before
// the point from which the caller must not allocate.  Every later call on that device
// only launches two kernels.  The address found at set-up belongs to the device's primary
// context and is kept for the life of the process: a caller that resets the device
// (cudaDeviceReset) or runs the library in another context of it must not call this
// entry point afterwards.
//
// Nothing in the array has to start at zero: the first kernel writes every partial sum
// the second one reads, for every call.  The array is shared by all calls on a device,
// so two calls whose kernels can overlap (different CUDA streams, or different contexts
// on one device) race on it; calls on one CUDA stream are ordered and safe.
#include <algorithm>
#include <mutex>
#include <string>

#include "handles.h"
#include "internal.h"

using namespace xpcs;

namespace {

constexpr size_t kCellBytes = sizeof(double) + sizeof(long long);  // one partial sum + its count
constexpr size_t kScratchBytes = (size_t)XPCS_G2_NOALLOC_MAX_CELLS * kCellBytes;
constexpr int kMaxDevices = 64;

}  // namespace

// The fixed scratch: [splits][n_q][T] f64 partial sums, then [splits][n_q][T] i64 counts.
static __device__ __align__(256) unsigned char g2_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_setup_mu;
void* g_scratch[kMaxDevices] = {};

// Once per device, with that device current: address of the array, kernels loaded.
xpcs_status setup(xpcs_ctx* ctx, void** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return fail(ctx, XPCS_EINVAL, "xpcs_g2_noalloc: device index " + std::to_string(ctx->device) + " above " +
                                      std::to_string(kMaxDevices - 1));
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch[ctx->device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g2_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(ctx, XPCS_ECUDA, std::string("xpcs_g2_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    XPCS_CUDA(ctx, preload_g2_from_C());
    g_scratch[ctx->device] = p;
  }
  *out = g_scratch[ctx->device];
  return XPCS_OK;
}

}  // namespace

extern "C" xpcs_status xpcs_g2_noalloc(xpcs_ctx* ctx, const float* C, int n_q, int64_t T, double* g2_out,
                                       int64_t* count_out) {
  if (!ctx || !C || !g2_out || n_q <= 0 || T <= 0) return fail(ctx, XPCS_EINVAL, "bad g2 args");
  if (n_q > XPCS_G2_MAX_RINGS)
    return fail(ctx, XPCS_ERANGE,
                "xpcs_g2_noalloc: n_q = " + std::to_string(n_q) + " rings exceeds the limit of " +
                    std::to_string(XPCS_G2_MAX_RINGS));
  if (T > XPCS_G2_NOALLOC_MAX_CELLS || (int64_t)n_q * T > XPCS_G2_NOALLOC_MAX_CELLS)
    return fail(ctx, XPCS_ERANGE,
                "xpcs_g2_noalloc: n_q * T = " + std::to_string((int64_t)n_q * T) + " exceeds its fixed scratch of " +
                    std::to_string((int64_t)XPCS_G2_NOALLOC_MAX_CELLS) + " ring-lag cells; use xpcs_g2");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  void* base = nullptr;
  XPCS_TRY(setup(ctx, &base));
  const int64_t cells = (int64_t)n_q * T;
  // row splits as in xpcs_g2, capped by what the array holds
  int64_t splits = g2_from_C_splits(T, n_q, ctx->num_sms);
  splits = std::min<int64_t>(splits, XPCS_G2_NOALLOC_MAX_CELLS / cells);
  double* part = static_cast<double*>(base);
  long long* cpart = reinterpret_cast<long long*>(static_cast<char*>(base) + (size_t)splits * cells * sizeof(double));
  XPCS_LAUNCH(ctx, "g2_from_C", 1, launch_g2_from_C(C, n_q, T, part, (int)splits, cpart, ctx->stream));
  XPCS_LAUNCH(ctx, "g2_from_C_reduce", 1, launch_g2_from_C_reduce(part, cpart, n_q, T, (int)splits, g2_out,
                                         reinterpret_cast<long long*>(count_out), ctx->stream));
  return finish(ctx);
}
