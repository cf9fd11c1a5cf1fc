// Failure-detection self test: a bounded device wait that nothing satisfies.
//
// Every wait of the library's kernels on an mbarrier is bounded by the globaltimer; when
// the limit passes, the waiting thread records XPCS_DEV_TIMEOUT in the context's status
// word and the kernel unwinds, so the host sees XPCS_ETIMEOUT and the context stays
// usable.  This entry point runs that path on purpose, with a wait on an mbarrier no
// thread ever arrives on, so that a test can check the detection end to end: either with
// its own limit, or through the library's bounded wait with the context's limit
// (xpcs_set_timeout).
#include "common.cuh"
#include "handles.h"
#include "internal.h"

using namespace xpcs;

namespace {

__global__ void selftest_wait_kernel(uint32_t* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(&bar, 0)) {  // phase 0 never completes: no thread arrives
      if (globaltimer() - t0 > limit_ns) {
        set_status(status, XPCS_DEV_TIMEOUT);
        break;
      }
    }
  }
}

// The same wait through the library's own bounded wait (mbar_wait), with the limit the
// context's kernels use.
__global__ void selftest_ctx_wait_kernel(uint32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, status);  // records XPCS_DEV_TIMEOUT at the limit
}

}  // namespace

extern "C" xpcs_status xpcs_selftest_timeout(xpcs_ctx* ctx, int limit_ms) {
  if (!ctx || limit_ms < 0 || limit_ms > 1000) return fail(ctx, XPCS_EINVAL, "selftest limit must be 0..1000 ms");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  if (limit_ms == 0) {
    if (ctx->wait_ns > 10000000000ull)
      return fail(ctx, XPCS_EINVAL, "selftest with the context's limit needs a limit of at most 10 s");
    XPCS_LAUNCH(ctx, "selftest_wait", 1,
                (selftest_ctx_wait_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_status), cudaGetLastError()));
  } else {
    XPCS_LAUNCH(ctx, "selftest_wait", 1,
                (selftest_wait_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_status,
                                                                 (unsigned long long)limit_ms * 1000000ull),
                 cudaGetLastError()));
  }
  return finish(ctx);
}

extern "C" xpcs_status xpcs_set_timeout(xpcs_ctx* ctx, int timeout_ms) {
  if (!ctx) return XPCS_EINVAL;
  if (timeout_ms < 0 || timeout_ms > 600000) return fail(ctx, XPCS_EINVAL, "timeout_ms must be 0..600000");
  if (ctx->capturing) return fail(ctx, XPCS_EBUSY, "the wait limit cannot change during a capture");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const uint64_t ns = (uint64_t)timeout_ms * 1000000ull;
  // ordered after the work already queued on the context's stream; the copy is from a
  // host value, so wait for it before returning
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  XPCS_CUDA(ctx, cudaMemcpy(ctx->d_status + 2, &ns, sizeof(ns), cudaMemcpyHostToDevice));
  ctx->wait_ns = ns;
  return XPCS_OK;
}

extern "C" int xpcs_get_timeout(const xpcs_ctx* ctx) {
  if (!ctx) return -1;
  return (int)((ctx->wait_ns ? ctx->wait_ns : XPCS_WAIT_NS) / 1000000ull);
}
