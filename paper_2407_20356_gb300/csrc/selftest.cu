// Failure-detection self test: a bounded device wait that nothing satisfies.
//
// Every wait of the library's kernels on an mbarrier is bounded by the globaltimer; when
// the limit passes, the waiting thread records XPCS_DEV_TIMEOUT in the context's status
// word and the kernel unwinds, so the host sees XPCS_ETIMEOUT and the context stays
// usable.  This entry point runs that path on purpose, with a wait on an mbarrier no
// thread ever arrives on, so that a test can check the detection end to end.
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

}  // namespace

extern "C" xpcs_status xpcs_selftest_timeout(xpcs_ctx* ctx, int limit_ms) {
  if (!ctx || limit_ms < 1 || limit_ms > 1000) return fail(ctx, XPCS_EINVAL, "selftest limit must be 1..1000 ms");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  XPCS_LAUNCH(ctx, "selftest_wait", 1,
              (selftest_wait_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_status, (unsigned long long)limit_ms * 1000000ull),
               cudaGetLastError()));
  return finish(ctx);
}
