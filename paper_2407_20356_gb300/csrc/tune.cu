// Autotuner of the two-time calls (compressed and raw).
//
// The two-time kernel has two run-time choices for a workload shape: the length of a work
// item (tiles along one tile diagonal whose diagonal sums meet once: 1, 2, 4, 8, 16 or 32; it
// trades load balance across the SMs against the number of partial-sum slots and per-item
// overheads) and its schedule: single tiles, or tile pairs (one N = 256 MMA for tiles
// (I, J) and (I, J + 1)).  The autotuner times every candidate on the caller's own inputs and outputs
// (CUDA events on the context's stream, after one untimed run per candidate that builds
// its work items), keeps the fastest in the context's table for the shape (rings, tiles,
// operand format, raw or compressed, whether C is stored), and finally runs it, so the
// outputs are those of the chosen configuration.  Later two-time calls of that shape use
// it.  A candidate replaces the default configuration only when it is at least 3 % faster,
// so timing noise does not flip the choice.
#include <functional>
#include <string>

#include "handles.h"
#include "internal.h"

using namespace xpcs;

namespace {

xpcs_status tune_shape(xpcs_ctx* ctx, uint64_t key, std::pair<int, int> dflt, int reps,
                       const std::function<xpcs_status()>& call, int* tiles_out, int* sched_out, double* ms_out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  XPCS_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, XPCS_ECUDA, "autotune: event creation failed");
  }
  const bool async = ctx->async, prof = ctx->prof;
  ctx->async = true;  // back-to-back calls; the events bound the timed runs
  ctx->prof = false;
  std::pair<int, int> best = dflt;
  double best_ms = 1e300, dflt_ms = 1e300;
  xpcs_status st = XPCS_OK;
  const int tiles[6] = {1, 2, 4, 8, 16, 32};
  for (int sched = 0; sched < 2 && st == XPCS_OK; ++sched) {
    for (int ti = 0; ti < 6 && st == XPCS_OK; ++ti) {
      ctx->tune_forced = true;
      ctx->tune_force = {tiles[ti], sched};
      st = call();  // untimed: builds the work items
      if (st != XPCS_OK) break;
      cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < reps && st == XPCS_OK; ++r) st = call();
      cudaEventRecord(e1, ctx->stream);
      if (st != XPCS_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = fail(ctx, XPCS_ECUDA, "autotune: event wait failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ctx->tune_force == dflt) dflt_ms = ms / reps;
      if (ms / reps < best_ms) {
        best_ms = ms / reps;
        best = ctx->tune_force;
      }
    }
  }
  ctx->tune_forced = false;
  if (st == XPCS_OK && best != dflt && best_ms > 0.97 * dflt_ms) {  // not clearly faster than the default
    best = dflt;
    best_ms = dflt_ms;
  }
  if (st == XPCS_OK) {
    ctx->gram_tune[key] = best;
    st = call();  // outputs of the chosen configuration
  }
  if (st == XPCS_OK) st = xpcs_synchronize(ctx);
  ctx->async = async;
  ctx->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != XPCS_OK) return st;
  if (tiles_out) *tiles_out = best.first;
  if (sched_out) *sched_out = best.second;
  if (ms_out) *ms_out = best_ms;
  return XPCS_OK;
}

}  // namespace

extern "C" xpcs_status xpcs_autotune_twotime(xpcs_ctx* ctx, const xpcs_basis* B, const float* A, int64_t T,
                                             xpcs_precision prec, float* C_out, double* g2_out, int64_t* count_out,
                                             int reps, int* tiles_out, int* sched_out, double* ms_out) {
  if (!ctx || !B || !A || T <= 0 || B->ctx != ctx || (int)prec < 0 || (int)prec > 2 || reps < 1 || reps > 100)
    return fail(ctx, XPCS_EINVAL, "bad autotune_twotime args");
  if (ctx->capturing) return fail(ctx, XPCS_EINVAL, "autotuning cannot run during a capture");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int n_q = B->rings->n_q;
  const int nT = (int)((T + TILE - 1) / TILE);
  const bool split = prec == XPCS_PREC_BF16X3;
  const uint64_t key = gram_tune_key(n_q, nT, prec == XPCS_PREC_FP16 ? 0 : 1, split ? 1 : 0, 0, C_out != nullptr);
  const bool merge = C_out == nullptr && g2_out != nullptr;
  return tune_shape(ctx, key, gram_default_compressed(merge), reps,
                    [&] { return xpcs_twotime(ctx, B, A, T, prec, C_out, g2_out, count_out); }, tiles_out,
                    sched_out, ms_out);
}

extern "C" xpcs_status xpcs_autotune_twotime_raw(xpcs_ctx* ctx, const xpcs_rings* R, const void* X,
                                                 xpcs_dtype dtype, int64_t T, float* C_out, int64_t* N_out,
                                                 double* g2_out, int64_t* count_out, int reps, int* tiles_out,
                                                 int* sched_out, double* ms_out) {
  if (!ctx || !R || !X || T <= 0 || R->ctx != ctx || reps < 1 || reps > 100)
    return fail(ctx, XPCS_EINVAL, "bad autotune_twotime_raw args");
  if (ctx->capturing) return fail(ctx, XPCS_EINVAL, "autotuning cannot run during a capture");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int nT = (int)((T + TILE - 1) / TILE);
  const uint64_t key = gram_tune_key(R->n_q, nT, 1, 0, 1, C_out || N_out);
  return tune_shape(ctx, key, gram_default_raw(R->n_q, nT), reps,
                    [&] { return xpcs_twotime_raw(ctx, R, X, dtype, T, C_out, N_out, g2_out, count_out); },
                    tiles_out, sched_out, ms_out);
}
