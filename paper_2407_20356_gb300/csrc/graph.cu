// CUDA-graph capture of library calls on a context's stream.
//
// xpcs_capture_begin puts the context's stream into capture mode (thread-local), so the
// following library calls on that context are recorded instead of run; xpcs_capture_end
// instantiates them as one graph, which xpcs_graph_launch replays with a single launch on
// the context's stream.  During the capture the context runs asynchronously (no
// synchronisation is allowed while capturing) and its profiling must be off.  The graph
// refers to the buffers the captured calls used (the caller's and the context's scratch),
// so while a graph exists the context refuses anything that would move or rewrite them:
// scratch growth, work items of another shape, first-use basis copies (XPCS_EBUSY).  Run
// each call once, at its largest size, before capturing it.
#include <string>

#include "handles.h"
#include "internal.h"

using namespace xpcs;

struct xpcs_graph {
  xpcs_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;  // kernels of the library in the graph
};

extern "C" xpcs_status xpcs_capture_begin(xpcs_ctx* ctx) {
  if (!ctx) return XPCS_EINVAL;
  if (ctx->capturing) return fail(ctx, XPCS_EINVAL, "capture already in progress");
  if (ctx->prof) return fail(ctx, XPCS_EINVAL, "turn profiling off before capturing");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  XPCS_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  ctx->capturing = true;
  ctx->async_before_capture = ctx->async;
  ctx->async = true;
  ctx->launches_at_capture = ctx->launches;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_capture_end(xpcs_ctx* ctx, xpcs_graph** out) {
  if (!ctx || !out) return XPCS_EINVAL;
  *out = nullptr;
  if (!ctx->capturing) return fail(ctx, XPCS_EINVAL, "no capture in progress");
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  ctx->capturing = false;
  ctx->async = ctx->async_before_capture;
  const uint64_t kernels = ctx->launches - ctx->launches_at_capture;
  ctx->launches = ctx->launches_at_capture;  // recorded, not run
  if (e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return fail(ctx, XPCS_ECUDA, std::string("capture failed: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t x = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
  if (ei != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(ctx, XPCS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  }
  auto* G = new xpcs_graph();
  G->ctx = ctx;
  G->graph = g;
  G->exec = x;
  G->kernels = kernels;
  ++ctx->graphs;
  *out = G;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_graph_launch(xpcs_ctx* ctx, const xpcs_graph* g) {
  if (!ctx || !g || g->ctx != ctx || ctx->capturing) return fail(ctx, XPCS_EINVAL, "bad graph_launch args");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  XPCS_CUDA(ctx, cudaGraphLaunch(g->exec, ctx->stream));
  ctx->launches += g->kernels;
  return finish(ctx);
}

extern "C" uint64_t xpcs_graph_kernels(const xpcs_graph* g) { return g ? g->kernels : 0; }

extern "C" xpcs_status xpcs_graph_destroy(xpcs_graph* g) {
  if (!g) return XPCS_EINVAL;
  xpcs_ctx* ctx = g->ctx;
  cudaStreamSynchronize(ctx->stream);  // no replay of it may still be running
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  --ctx->graphs;
  delete g;
  return XPCS_OK;
}
