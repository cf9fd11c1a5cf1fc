// C ABI of the online stream (Sec. 2.2, Fig. 1c): open, push frames, poll, read g2.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "handles.h"
#include "internal.h"

using namespace xpcs;

namespace xpcs {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace xpcs

namespace {


int kpad_of(int k) { return (k + 63) / 64 * 64; }
// ring slots: the window plus a batch, and at least 256 so that a 128-row history
// operand starting anywhere in the ring ends before the 128 mirrored rows do; whole
// 128-frame blocks, at least one more than the tile diagonals a lag < W can reach (the
// two-time kernel reads the history by blocks, the step's block among them)
int64_t ring_cap(int64_t W, int max_batch) {
  const int64_t c = std::max<int64_t>({W + max_batch, 256, 128LL * (stream_nd(W) + 1)});
  return (c + 127) / 128 * 128;
}
// frames per stream step (one launch of each stream kernel)
constexpr int STEP_MAX = 64;        // frames per step on the row update kernel (at most)
constexpr int STEP_MAX_GRAM = 128;  // frames per step on the two-time kernel (one block)
// W2 rows: the pair-ordered M-tiles of every ring group for any step size, plus one
// spare 128-row box
int64_t w2_rows(int max_batch, int n_q) {
  int mt = 0;  // the pair layouts of small and large steps differ: take the largest step need
  for (int b = 1; b <= std::min(STEP_MAX, max_batch); ++b) mt = std::max(mt, w2_mtiles(b, n_q));
  return (int64_t)((n_q + 35) / 36) * mt * 128 + 128;
}
int nblk_of(int64_t M) { return (int)((M + 4095) / 4096); }
// row pitch (elements) of the g2 sums and counts: whole 64-lag tiles
int64_t wpitch(int64_t W) { return (W + 63) / 64 * 64; }

struct Sizes {
  size_t frames, A2, Rh, vbits, g2sum, cnt, part, a, W2, g2, stage, Wg, gpart, se;
};

Sizes stream_sizes(int64_t M, int n_q, int k, int64_t W, int max_batch, int eb) {
  const int64_t cap = ring_cap(W, max_batch);
  Sizes z;
  z.frames = (size_t)max_batch * M * eb;
  z.A2 = (size_t)(cap + 128) * 2 * kpad_of(k) * 2;
  z.Rh = (size_t)(cap + 128) * stream_npad(n_q) * 4;
  z.vbits = (size_t)n_q * stream_vwords(cap) * 8;
  z.g2sum = (size_t)n_q * wpitch(W) * 8;
  z.cnt = (size_t)n_q * wpitch(W) * 8;
  // the sparse encode's slice partials, or the tensor-core encode's split-K partials of
  // one 128-frame step (at most 256 pixel splits)
  z.part = std::max((size_t)max_batch * nblk_of(M) * k * 4, (size_t)256 * 128 * k * 4);
  z.a = (size_t)max_batch * k * 4;
  z.W2 = (size_t)w2_rows(max_batch, n_q) * 2 * kpad_of(k) * 2;
  z.g2 = (size_t)n_q * W * 8;
  z.stage = (size_t)max_batch * M * eb;
  z.Wg = (size_t)n_q * 128 * 2 * kpad_of(k) * 2;
  z.gpart = (size_t)n_q * stream_nd(W) * DIAG_SLOTS * 4;
  z.se = (size_t)STEP_MAX_GRAM * 4;  // per-frame counters of the sparse encode's slice blocks
  return z;
}

void stream_free(xpcs_stream* S) {
  xpcs_ctx* ctx = S->ctx;
  if (S->stream) cudaStreamSynchronize(S->stream);
  const Sizes z = stream_sizes(S->M, S->n_q, S->k, S->W, S->max_batch, S->dtype == XPCS_U8 ? 1 : 2);
  dev_free(ctx, S->d_frames, z.frames);
  dev_free(ctx, S->d_A2, z.A2);
  dev_free(ctx, S->d_Rh, z.Rh);
  dev_free(ctx, S->d_vbits, z.vbits);
  dev_free(ctx, S->d_g2sum, z.g2sum);
  dev_free(ctx, S->d_cnt, z.cnt);
  dev_free(ctx, S->d_part, z.part);
  dev_free(ctx, S->d_a, z.a);
  dev_free(ctx, S->d_W2, z.W2);
  dev_free(ctx, S->d_Wg, z.Wg);
  dev_free(ctx, S->d_gpart, z.gpart);
  dev_free(ctx, S->d_se_done, z.se);
  if (S->h_status) cudaFreeHost(S->h_status);
  dev_free(ctx, S->d_g2, z.g2);
  dev_free(ctx, S->d_qmap, (size_t)S->M * 4);
  dev_free(ctx, S->d_Sx, (size_t)STEP_MAX_GRAM * S->n_q * 8);
  for (int i = 0; i < 2; ++i) {
    if (S->h_stage[i]) cudaFreeHost(S->h_stage[i]);
    if (S->stage_done[i]) cudaEventDestroy(S->stage_done[i]);
  }
  for (auto& t : S->tickets) {
    cudaEventDestroy(t.ev);
    if (t.stamp && !t.stamp->done_ns) delete t.stamp;  // not yet handed to `stamps`
  }
  for (auto e : S->event_pool) cudaEventDestroy(e);
  for (auto st : S->stamps) delete st;
  if (S->base_ev) cudaEventDestroy(S->base_ev);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // namespace

namespace xpcs {

size_t stream_footprint(const xpcs_basis* B, int64_t W, int max_batch, int elem_bytes) {
  const Sizes z = stream_sizes(B->M, B->n_q, B->k, W, max_batch, elem_bytes);
  size_t b = z.frames + z.A2 + z.Rh + z.vbits + z.g2sum + z.cnt + z.part + z.a + z.W2 + z.g2 + z.Wg + z.gpart + z.se;
  if (!B->d_B32) b += (size_t)B->rings->M * B->k * 4;  // f32 basis copy made on first use
  return b;
}

}  // namespace xpcs

namespace {

// Host time of the base event: record it on the idle stream and watch it complete
// (bounded to one second); completion is seen within the polling interval.
cudaError_t calibrate_clock(xpcs_stream* S) {
  cudaError_t e = cudaEventRecord(S->base_ev, S->stream);
  if (e != cudaSuccess) return e;
  const int64_t t_end = now_ns() + 1000000000ll;
  while ((e = cudaEventQuery(S->base_ev)) == cudaErrorNotReady)
    if (now_ns() > t_end) return cudaErrorNotReady;
  S->base_ns = now_ns();
  return e;
}

}  // namespace

extern "C" xpcs_status xpcs_stream_open(xpcs_ctx* ctx, const xpcs_basis* B, int64_t history, int max_batch,
                                        xpcs_dtype dtype, xpcs_stream** out) {
  return xpcs_stream_open_opts(ctx, B, history, max_batch, dtype, nullptr, out);
}

extern "C" xpcs_status xpcs_stream_open_opts(xpcs_ctx* ctx, const xpcs_basis* B, int64_t history, int max_batch,
                                             xpcs_dtype dtype, const xpcs_options* opt, xpcs_stream** out) {
  if (!ctx || !B || !out || B->ctx != ctx || history < 1 || max_batch < 1 || max_batch > 1024 || B->k > 256 ||
      (dtype != XPCS_U8 && dtype != XPCS_U16) || (opt && (opt->qmean < 0 || opt->qmean > 1)) ||
      (opt && opt->precision != XPCS_PREC_FP16 && opt->precision != XPCS_PREC_BF16X3))
    return fail(ctx, XPCS_EINVAL, "bad stream_open args");
  const bool exact = opt && opt->qmean == XPCS_QMEAN_EXACT_RAW;
  const int sp = (opt && opt->precision == XPCS_PREC_FP16) ? 1 : 0;
  *out = nullptr;
  int lt = 0, wst = 0, epi = 0;  // the largest step the row update kernel takes
  if (!row_update_config(B->rings->n_q, kpad_of(B->k), STREAM_GRAM_MIN - 1, &lt, &wst, &epi))
    return fail(ctx, XPCS_ENOTSUP, "stream: the row-update tile does not fit shared memory at this k");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int eb = dtype == XPCS_U8 ? 1 : 2;
  const size_t exact_bytes = exact ? (size_t)B->rings->M * 4 + (size_t)STEP_MAX_GRAM * B->rings->n_q * 8 : 0;
  const size_t need = stream_footprint(B, history, max_batch, eb) + exact_bytes;
  if (ctx->budget && ctx->held + need > ctx->budget)
    return fail(ctx, XPCS_EBUSY,
                "stream needs " + std::to_string(need) + " device bytes; " +
                    std::to_string(ctx->budget > ctx->held ? ctx->budget - ctx->held : 0) + " free in the budget");
  xpcs_basis* Bm = const_cast<xpcs_basis*>(B);
  if (!Bm->d_B32) {
    void* p = nullptr;
    XPCS_TRY(dev_alloc(ctx, &p, (size_t)B->rings->M * B->k * 4));
    Bm->d_B32 = static_cast<float*>(p);
    Bm->bytes += (size_t)B->rings->M * B->k * 4;
    XPCS_LAUNCH(ctx, "basis_f32", 1, launch_basis_f32(B->d_B, (long long)B->rings->M * B->k, Bm->d_B32, ctx->stream));
    XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  auto* S = new xpcs_stream();
  S->ctx = ctx;
  S->basis = B;
  S->W = history;
  S->cap = ring_cap(history, max_batch);
  S->max_batch = max_batch;
  S->dtype = dtype;
  S->M = B->M;
  S->n_q = B->n_q;
  S->k = B->k;
  S->nblk = nblk_of(B->M);
  S->sp = sp;
  const Sizes z = stream_sizes(S->M, S->n_q, S->k, history, max_batch, eb);
  xpcs_status st = XPCS_OK;
  void* p = nullptr;
#define XPCS_SALLOC(field, bytes, T)                  \
  if (st == XPCS_OK) {                                \
    st = dev_alloc(ctx, &p, (bytes));                 \
    S->field = static_cast<T>(p);                     \
  }
  XPCS_SALLOC(d_frames, z.frames, void*)
  XPCS_SALLOC(d_A2, z.A2, __nv_bfloat16*)
  XPCS_SALLOC(d_Rh, z.Rh, float*)
  XPCS_SALLOC(d_vbits, z.vbits, unsigned long long*)
  XPCS_SALLOC(d_g2sum, z.g2sum, float2*)
  XPCS_SALLOC(d_cnt, z.cnt, long long*)
  XPCS_SALLOC(d_part, z.part, float*)
  XPCS_SALLOC(d_a, z.a, float*)
  XPCS_SALLOC(d_W2, z.W2, __nv_bfloat16*)
  XPCS_SALLOC(d_g2, z.g2, double*)
  XPCS_SALLOC(d_Wg, z.Wg, __nv_bfloat16*)
  XPCS_SALLOC(d_gpart, z.gpart, float*)
  XPCS_SALLOC(d_se_done, z.se, unsigned*)
  if (exact) {
    XPCS_SALLOC(d_qmap, (size_t)B->rings->M * 4, int*)
    XPCS_SALLOC(d_Sx, (size_t)STEP_MAX_GRAM * B->rings->n_q * 8, long long*)
  }
#undef XPCS_SALLOC
  cudaError_t e = cudaSuccess;
  if (st == XPCS_OK) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && st == XPCS_OK && e == cudaSuccess; ++i) {
    e = cudaHostAlloc(&S->h_stage[i], z.stage, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->stage_done[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(S->stage_done[i], S->stream);
  }
  if (st == XPCS_OK && e == cudaSuccess && exact)  // the stream's own copy of the ring labels
    e = cudaMemcpyAsync(S->d_qmap, B->rings->d_qmap, (size_t)B->rings->M * 4, cudaMemcpyDeviceToDevice, S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(S->d_A2, 0, z.A2, S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(S->d_W2, 0, z.W2, S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(S->d_Wg, 0, z.Wg, S->stream);
  // status word, then (8 bytes on) the bounded-wait limit taken from the context
  if (st == XPCS_OK && e == cudaSuccess) e = cudaHostAlloc((void**)&S->h_status, 16, cudaHostAllocMapped);
  if (st == XPCS_OK && e == cudaSuccess) {
    *S->h_status = 0;
    *reinterpret_cast<volatile uint64_t*>(S->h_status + 2) = ctx->wait_ns;
    e = cudaHostGetDevicePointer((void**)&S->d_status, S->h_status, 0);
  }
  if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(S->d_Rh, 0, z.Rh, S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(S->d_vbits, 0, z.vbits, S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(S->d_g2sum, 0, z.g2sum, S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(S->d_cnt, 0, z.cnt, S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(S->d_se_done, 0, z.se, S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaEventCreate(&S->base_ev);
  if (st == XPCS_OK && e == cudaSuccess) e = calibrate_clock(S);
  if (st == XPCS_OK && e != cudaSuccess) st = fail(ctx, XPCS_ECUDA, std::string("stream setup: ") + cudaGetErrorString(e));
  S->kpad = kpad_of(B->k);
  if (st == XPCS_OK)
    st = make_map(ctx, &S->tmA, S->d_A2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2 * S->kpad, S->cap + 128, 64, 128,
                  CU_TENSOR_MAP_SWIZZLE_128B);
  if (st == XPCS_OK)
    st = make_map(ctx, &S->tmW, S->d_W2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2 * S->kpad,
                  w2_rows(max_batch, B->rings->n_q), 64, 128, CU_TENSOR_MAP_SWIZZLE_128B);
  if (st == XPCS_OK)
    st = make_map(ctx, &S->tmW48, S->d_W2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2 * S->kpad,
                  w2_rows(max_batch, B->rings->n_q), 64, 48, CU_TENSOR_MAP_SWIZZLE_128B);
  if (st == XPCS_OK)
    st = make_map(ctx, &S->tmWg, S->d_Wg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2 * S->kpad,
                  (uint64_t)128 * B->rings->n_q, 64, 128, CU_TENSOR_MAP_SWIZZLE_128B);
  if (st == XPCS_OK)  // ring pairs (rows past the last ring read as zeros)
    st = make_map(ctx, &S->tmWg2, S->d_Wg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2 * S->kpad,
                  (uint64_t)128 * B->rings->n_q, 64, 256, CU_TENSOR_MAP_SWIZZLE_128B);
  if (st == XPCS_OK) {
    const int npad = stream_npad(B->rings->n_q);
    st = make_map(ctx, &S->tmR, S->d_Rh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, npad, S->cap + 128,
                  std::min(36, npad), 128, CU_TENSOR_MAP_SWIZZLE_NONE);
  }
  // g2 sums and counts: W x n_q with row pitch Wp, boxes of lt lags x up to 36 rings for
  // every lag tile a step may take
  const int qg2 = std::min(36, B->rings->n_q);
  for (int i = 0; i < RT_N_LT && st == XPCS_OK; ++i) {
    // 8-byte elements (f32 pairs; the copies are bitwise)
    st = make_map(ctx, &S->tmG[i], S->d_g2sum, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, history, B->rings->n_q,
                  RT_LTS[i], qg2, CU_TENSOR_MAP_SWIZZLE_NONE, (uint64_t)wpitch(history) * 8);
    if (st == XPCS_OK)
      st = make_map(ctx, &S->tmC[i], S->d_cnt, CU_TENSOR_MAP_DATA_TYPE_INT64, 8, history, B->rings->n_q,
                    RT_LTS[i], qg2, CU_TENSOR_MAP_SWIZZLE_NONE, (uint64_t)wpitch(history) * 8);
  }
  if (st != XPCS_OK) {
    stream_free(S);
    return st;
  }
  S->bytes = need;
  *out = S;
  return XPCS_OK;
}

namespace {

cudaEvent_t take_event(xpcs_stream* S) {
  if (!S->event_pool.empty()) {
    cudaEvent_t e = S->event_pool.back();
    S->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Retire the completed batches at the front of the ticket queue: their completion time
// from the event timing, their event back to the pool.  A base older than five seconds is
// replaced by a retired event (keeps the f32 millisecond differences fine-grained).
xpcs_status retire(xpcs_stream* S) {
  while (!S->tickets.empty()) {
    xpcs_stream::Ticket& tk = S->tickets.front();
    const cudaError_t q = cudaEventQuery(tk.ev);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) return fail(S->ctx, XPCS_ECUDA, std::string("stream: ") + cudaGetErrorString(q));
    if (const uint32_t code = *static_cast<volatile uint32_t*>(S->h_status)) {
      *S->h_status = 0;
      return fail(S->ctx, code == XPCS_DEV_TIMEOUT ? XPCS_ETIMEOUT : XPCS_ECUDA,
                  "stream: a bounded device wait expired (device status " + std::to_string(code) + ")");
    }
    float ms = 0.f;
    const cudaError_t e = cudaEventElapsedTime(&ms, S->base_ev, tk.ev);
    if (e != cudaSuccess) return fail(S->ctx, XPCS_ECUDA, std::string("stream timing: ") + cudaGetErrorString(e));
    const int64_t done = S->base_ns + (int64_t)((double)ms * 1e6);
    if (tk.stamp) {
      tk.stamp->done_ns = done > 0 ? done : 1;
      S->stamps.push_back(tk.stamp);
    }
    if (done - S->base_ns > 5000000000ll) {
      S->event_pool.push_back(S->base_ev);
      S->base_ev = tk.ev;
      S->base_ns = done;
    } else {
      S->event_pool.push_back(tk.ev);
    }
    S->tickets.pop_front();
  }
  return XPCS_OK;
}

// Add the deferred pair counts still missing: the parts of the block before that are not
// done, and (all) also the latest block's.  Enqueued on the stream's CUDA stream.
cudaError_t flush_counts(xpcs_stream* S, bool all) {
  const long long vw = stream_vwords(S->cap), Wp = wpitch(S->W);
  cudaError_t e = cudaSuccess;
  if (S->cf_prev)
    e = launch_count_flush(S->d_vbits, vw, S->cap, S->n_q, S->W, Wp, S->d_cnt, (S->cf_blk - 1) * 64, S->cf_prev,
                           S->cf_done, S->stream);
  S->cf_prev = 0;
  S->cf_done = 0;
  if (all && e == cudaSuccess) {
    if (S->cf_cur)
      e = launch_count_flush(S->d_vbits, vw, S->cap, S->n_q, S->W, Wp, S->d_cnt, S->cf_blk * 64, S->cf_cur, 0ull,
                             S->stream);
    S->cf_cur = 0;
  }
  return e;
}

// Before a step that starts in count block blk: the block before the previous one gets
// its missing parts; a step in the next block makes the latest block the one whose parts
// its single-frame steps add, and a larger jump flushes both.
cudaError_t roll_counts(xpcs_stream* S, int64_t blk) {
  if (blk == S->cf_blk) return cudaSuccess;
  const bool next = blk == S->cf_blk + 1;
  const cudaError_t e = flush_counts(S, !next);
  if (next) S->cf_prev = S->cf_cur;
  S->cf_cur = 0;
  S->cf_done = 0;
  S->cf_blk = blk;
  return e;
}

// Enqueue one batch whose counts are already on the device.
xpcs_status enqueue_batch(xpcs_stream* S, const void* X, int64_t n, xpcs_stream::Stamp* stamp) {
  xpcs_ctx* ctx = S->ctx;
  const xpcs_basis* B = S->basis;
  StreamStep s{};
  s.X = X;
  s.dtype = S->dtype;
  s.vec16 = (reinterpret_cast<uintptr_t>(X) % 16 == 0) &&
            ((size_t)B->rings->M * (S->dtype == XPCS_U8 ? 1 : 2)) % 16 == 0;
  s.M = B->rings->M;
  s.k = B->k;
  s.n_q = B->rings->n_q;
  s.b = (int)n;
  s.t0 = S->frames;
  s.W = S->W;
  s.Wp = wpitch(S->W);
  s.cap = S->cap;
  s.nblk = S->nblk;
  s.B32 = B->d_B32;
  s.G32 = B->d_G32;
  s.s64 = B->d_s;
  s.Mq = B->rings->d_Mq;
  s.qmap = S->d_qmap;
  s.Sx = S->d_Sx;
  s.part = S->d_part;
  s.se_done = S->d_se_done;
  s.a = S->d_a;
  s.W2 = S->d_W2;
  s.A2 = S->d_A2;
  s.kpad = S->kpad;
  s.w2_rows = w2_rows(S->max_batch, B->rings->n_q);
  s.Rh = S->d_Rh;
  s.vbits = S->d_vbits;
  s.vwords = stream_vwords(S->cap);
  s.status = S->d_status;
  s.num_sms = ctx->num_sms;
  s.tmA = &S->tmA;
  s.tmW = &S->tmW;
  s.tmR = &S->tmR;
  s.tmG = S->tmG;
  s.tmC = S->tmC;
  s.g2sum = S->d_g2sum;
  s.cnt = S->d_cnt;
  s.Wg = S->d_Wg;
  s.gpart = S->d_gpart;
  s.nd = stream_nd(S->W);
  s.tmWg = &S->tmWg;
  s.tmWg2 = &S->tmWg2;
  s.tmW48 = &S->tmW48;
  s.sp = S->sp;
  // steps of at most STEP_MAX_GRAM frames; the batch completes with its last step
  const size_t fb = (size_t)B->rings->M * (S->dtype == XPCS_U8 ? 1 : 2);
  const size_t part_bytes =
      stream_sizes(S->M, S->n_q, S->k, S->W, S->max_batch, S->dtype == XPCS_U8 ? 1 : 2).part;
  cudaError_t e = cudaSuccess;
  for (int64_t f0 = 0; f0 < n && e == cudaSuccess; f0 += s.b) {
    s.X = static_cast<const char*>(X) + f0 * fb;
    s.vec16 = (reinterpret_cast<uintptr_t>(s.X) % 16 == 0) && fb % 16 == 0;
    s.t0 = S->frames + f0;
    // a step large enough for the two-time kernel takes up to the rest of its 128-frame
    // block; smaller ones go to the row update kernel
    const int room = 128 - (int)(s.t0 & 127);
    s.b = (int)std::min<int64_t>(STEP_MAX_GRAM, n - f0);
    if (s.b >= STREAM_GRAM_MIN) s.b = std::min(s.b, room);
    if (s.b < STREAM_GRAM_MIN) s.b = std::min(s.b, STEP_MAX);
    // steps on the two-time kernel take the tensor-core encode (frames once, the basis
    // pieces once per step) instead of gathering the nonzero pixels' f32 basis rows, unless
    // the exact ring sums of the frames are wanted (the sparse encode forms them)
    s.pre_encoded = 0;
    if (s.b >= STREAM_GRAM_MIN && !S->d_Sx && s.vec16 &&
        encode_partials(B, s.b, ctx->num_sms) * 4 <= part_bytes) {
      const xpcs_status es =
          encode_on_stream(ctx, B, s.X, (xpcs_dtype)S->dtype, s.b, s.a, s.part, S->d_status, S->stream);
      if (es != XPCS_OK) {
        delete stamp;
        return es;
      }
      s.pre_encoded = 1;
    }
    // pair counts: a single-frame step defers its own to its count block and adds part
    // (t mod 64) of the block before's; other steps count their frames themselves
    s.cf_mask = 0;
    if ((e = roll_counts(S, s.t0 >> 6)) != cudaSuccess) break;
    if (stream_step_row1(s)) {
      const int j = (int)(s.t0 & 63);
      S->cf_cur |= 1ull << j;
      const long long L = cf_part_len(S->W);
      if (S->cf_prev && !((S->cf_done >> j) & 1ull) && j * L < S->W) {
        s.cf_t0 = (S->cf_blk - 1) * 64;
        s.cf_mask = S->cf_prev;
        s.cf_tau0 = (int)(j * L);
        s.cf_tau1 = (int)std::min<long long>(S->W, (j + 1) * L);
      }
      S->cf_done |= 1ull << j;
    }
    e = launch_stream_step(s, S->stream);
    if (e == cudaSuccess) ctx->launches += s.b >= STREAM_GRAM_MIN ? 5 : 4;
  }
  if (e != cudaSuccess) {
    delete stamp;
    return fail(ctx, XPCS_ECUDA, std::string("stream step: ") + cudaGetErrorString(e));
  }
  S->frames += n;
  cudaEvent_t ev = take_event(S);
  if (!ev) {
    delete stamp;
    return fail(ctx, XPCS_ECUDA, "stream event: cudaEventCreate failed");
  }
  e = cudaEventRecord(ev, S->stream);
  if (e != cudaSuccess) {
    delete stamp;
    return fail(ctx, XPCS_ECUDA, std::string("stream event: ") + cudaGetErrorString(e));
  }
  S->tickets.push_back({(uint64_t)S->frames, ev, stamp});
  return retire(S);
}

}  // namespace

namespace xpcs {

xpcs_status stream_push_host(xpcs_stream* S, const void* frames, int64_t n, const int64_t* arrive_ns, bool block) {
  xpcs_ctx* ctx = S->ctx;
  const size_t fb = (size_t)S->basis->rings->M * (S->dtype == XPCS_U8 ? 1 : 2);
  const int i = S->stage_i;
  if (block) {
    XPCS_CUDA(ctx, cudaEventSynchronize(S->stage_done[i]));  // the staging buffer is free again
  } else {
    const cudaError_t q = cudaEventQuery(S->stage_done[i]);
    if (q == cudaErrorNotReady) return XPCS_EBUSY;
    if (q != cudaSuccess) return fail(ctx, XPCS_ECUDA, std::string("stream staging: ") + cudaGetErrorString(q));
  }
  S->stage_i ^= 1;
  auto* stamp = new xpcs_stream::Stamp();
  const int64_t t = now_ns();
  stamp->arrive_ns.resize(n);
  for (int64_t f = 0; f < n; ++f) stamp->arrive_ns[f] = arrive_ns ? arrive_ns[f] : t;
  memcpy(S->h_stage[i], frames, n * fb);
  cudaError_t e = cudaMemcpyAsync(S->d_frames, S->h_stage[i], n * fb, cudaMemcpyHostToDevice, S->stream);
  if (e == cudaSuccess) e = cudaEventRecord(S->stage_done[i], S->stream);
  if (e != cudaSuccess) {
    delete stamp;
    return fail(ctx, XPCS_ECUDA, std::string("stream copy: ") + cudaGetErrorString(e));
  }
  return enqueue_batch(S, S->d_frames, n, stamp);
}

}  // namespace xpcs

extern "C" xpcs_status xpcs_stream_push(xpcs_stream* S, const void* frames_host, int64_t n_frames, uint64_t* ticket) {
  if (!S || !frames_host || n_frames < 0) return XPCS_EINVAL;
  xpcs_ctx* ctx = S->ctx;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t fb = (size_t)S->basis->rings->M * (S->dtype == XPCS_U8 ? 1 : 2);
  const char* src = static_cast<const char*>(frames_host);
  for (int64_t off = 0; off < n_frames; off += S->max_batch) {
    const int64_t n = std::min<int64_t>(S->max_batch, n_frames - off);
    XPCS_TRY(stream_push_host(S, src + off * fb, n, nullptr, true));
  }
  if (ticket) *ticket = (uint64_t)S->frames;
  return XPCS_OK;
}

namespace {

xpcs_status push_device(xpcs_stream* S, const void* frames, int64_t n_frames, const int64_t* arrive_ns,
                        uint64_t* ticket) {
  if (!S || !frames || n_frames < 0) return XPCS_EINVAL;
  xpcs_ctx* ctx = S->ctx;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t fb = (size_t)S->basis->rings->M * (S->dtype == XPCS_U8 ? 1 : 2);
  const int64_t t = now_ns();
  for (int64_t off = 0; off < n_frames; off += S->max_batch) {
    const int64_t n = std::min<int64_t>(S->max_batch, n_frames - off);
    auto* stamp = new xpcs_stream::Stamp();
    if (arrive_ns)
      stamp->arrive_ns.assign(arrive_ns + off, arrive_ns + off + n);
    else
      stamp->arrive_ns.assign(n, t);
    XPCS_TRY(enqueue_batch(S, static_cast<const char*>(frames) + off * fb, n, stamp));
  }
  if (ticket) *ticket = (uint64_t)S->frames;
  return XPCS_OK;
}

}  // namespace

namespace xpcs {

xpcs_status stream_push_device_stamped(xpcs_stream* S, const void* frames, int64_t n, const int64_t* arrive_ns) {
  return push_device(S, frames, n, arrive_ns, nullptr);
}

int stream_inflight(xpcs_stream* S) {
  if (retire(S) != XPCS_OK) return 0;  // the next push reports the error
  return (int)S->tickets.size();
}

}  // namespace xpcs

extern "C" xpcs_status xpcs_stream_push_device(xpcs_stream* S, const void* frames, int64_t n_frames,
                                               uint64_t* ticket) {
  return push_device(S, frames, n_frames, nullptr, ticket);
}

extern "C" xpcs_status xpcs_stream_push_device_at(xpcs_stream* S, const void* frames, int64_t n_frames,
                                                  const int64_t* arrive_ns_host, uint64_t* ticket) {
  if (!arrive_ns_host) return XPCS_EINVAL;
  return push_device(S, frames, n_frames, arrive_ns_host, ticket);
}

extern "C" int64_t xpcs_clock_ns(void) { return now_ns(); }

extern "C" xpcs_status xpcs_stream_poll(xpcs_stream* S, uint64_t ticket, int timeout_ms) {
  if (!S) return XPCS_EINVAL;
  xpcs_ctx* ctx = S->ctx;
  const int64_t t_end = now_ns() + (int64_t)std::max(0, timeout_ms) * 1000000;
  while (true) {
    XPCS_TRY(retire(S));
    // tickets are increasing: none pending at or below `ticket` means its frames are in
    if (S->tickets.empty() || S->tickets.front().frames > ticket) return XPCS_OK;
    if (now_ns() >= t_end) return XPCS_EBUSY;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

extern "C" xpcs_status xpcs_stream_read_g2(xpcs_stream* S, double* g2_host, int64_t* count_host) {
  if (!S) return XPCS_EINVAL;
  xpcs_ctx* ctx = S->ctx;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int n_q = S->basis->rings->n_q;
  const long long n = (long long)n_q * S->W;
  {  // the pair counts deferred by single-frame steps
    const cudaError_t e = flush_counts(S, true);
    if (e != cudaSuccess) return fail(ctx, XPCS_ECUDA, std::string("stream counts: ") + cudaGetErrorString(e));
  }
  if (g2_host) {
    cudaError_t e = launch_stream_g2(S->d_g2sum, S->d_cnt, n_q, S->W, wpitch(S->W), S->d_g2, S->stream);
    if (e != cudaSuccess) return fail(ctx, XPCS_ECUDA, std::string("stream g2: ") + cudaGetErrorString(e));
    ctx->launches += 1;
    XPCS_CUDA(ctx, cudaMemcpyAsync(g2_host, S->d_g2, n * 8, cudaMemcpyDeviceToHost, S->stream));
  }
  if (count_host)
    XPCS_CUDA(ctx, cudaMemcpy2DAsync(count_host, S->W * 8, S->d_cnt, wpitch(S->W) * 8, S->W * 8, n_q,
                                     cudaMemcpyDeviceToHost, S->stream));
  XPCS_CUDA(ctx, cudaStreamSynchronize(S->stream));
  return XPCS_OK;
}

extern "C" int64_t xpcs_stream_frames(const xpcs_stream* S) { return S ? S->frames : 0; }

extern "C" xpcs_status xpcs_stream_latency(xpcs_stream* S, int reset, double* p50_us, double* p99_us,
                                           double* max_us, int64_t* n_batches) {
  if (!S) return XPCS_EINVAL;
  XPCS_TRY(retire(S));
  std::vector<double> lat;
  std::vector<xpcs_stream::Stamp*> keep;
  for (auto* st : S->stamps) {
    const int64_t d = st->done_ns;
    if (d) {
      for (int64_t a : st->arrive_ns) lat.push_back((d - a) * 1e-3);
      if (reset) delete st;
      else keep.push_back(st);
    } else {
      keep.push_back(st);
    }
  }
  S->stamps.swap(keep);
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double f) { return lat.empty() ? 0.0 : lat[std::min(lat.size() - 1, (size_t)(f * lat.size()))]; };
  if (p50_us) *p50_us = pct(0.50);
  if (p99_us) *p99_us = pct(0.99);
  if (max_us) *max_us = lat.empty() ? 0.0 : lat.back();
  if (n_batches) *n_batches = (int64_t)lat.size();  // frames measured
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_stream_close(xpcs_stream* S) {
  if (!S) return XPCS_EINVAL;
  stream_free(S);
  return XPCS_OK;
}

// ====================================================================== checkpoint / resume
//
// A checkpoint is a header followed by the stream's state: the coefficient history ring
// (bf16 hi | lo rows), the ring-factor rows r_q(s), the validity bits, the g2 sums and the
// pair counts, each as stored on the device.  Everything else a stream holds is per-step
// scratch.  The header records the shape (k, n_q, M, W, ring slots, dtype), the frame
// count and a hash of the basis's ring factors (FNV-1a over G_q and s_q), so a checkpoint
// is restored only into a stream of the same shape and basis.

namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t k, n_q, dtype, precision;  // precision: 1 f16 rows, 0 bf16 hi | lo
  int64_t M, W, cap, frames;
  uint64_t basis_hash;
  uint64_t bytes[5];  // A2, Rh, vbits, g2sum, cnt
};

constexpr char CKPT_MAGIC[8] = {'X', 'P', 'C', 'S', 'C', 'K', 'P', 'T'};
constexpr uint32_t CKPT_VERSION = 3;  // 3: the row precision recorded; 2: g2 sums as f32 pairs (1: FP64)

xpcs_status basis_hash(xpcs_stream* S, uint64_t* h) {
  const xpcs_basis* B = S->basis;
  const int n_q = B->rings->n_q, k = B->k;
  std::vector<double> buf((size_t)n_q * k * k + (size_t)n_q * k);
  XPCS_CUDA(S->ctx, cudaMemcpy(buf.data(), B->d_G, (size_t)n_q * k * k * 8, cudaMemcpyDeviceToHost));
  XPCS_CUDA(S->ctx, cudaMemcpy(buf.data() + (size_t)n_q * k * k, B->d_s, (size_t)n_q * k * 8, cudaMemcpyDeviceToHost));
  uint64_t x = 1469598103934665603ull;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(buf.data());
  for (size_t i = 0; i < buf.size() * 8; ++i) x = (x ^ p[i]) * 1099511628211ull;
  *h = x;
  return XPCS_OK;
}

void ckpt_parts(xpcs_stream* S, void* ptr[5], uint64_t bytes[5]) {
  const Sizes z = stream_sizes(S->M, S->n_q, S->k, S->W, S->max_batch, S->dtype == XPCS_U8 ? 1 : 2);
  ptr[0] = S->d_A2;
  ptr[1] = S->d_Rh;
  ptr[2] = S->d_vbits;
  ptr[3] = S->d_g2sum;
  ptr[4] = S->d_cnt;
  bytes[0] = z.A2;
  bytes[1] = z.Rh;
  bytes[2] = z.vbits;
  bytes[3] = z.g2sum;
  bytes[4] = z.cnt;
}

}  // namespace

extern "C" xpcs_status xpcs_stream_checkpoint_size(const xpcs_stream* S, size_t* bytes) {
  if (!S || !bytes) return XPCS_EINVAL;
  void* ptr[5];
  uint64_t b[5];
  ckpt_parts(const_cast<xpcs_stream*>(S), ptr, b);
  *bytes = sizeof(CkptHeader) + b[0] + b[1] + b[2] + b[3] + b[4];
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_stream_checkpoint(xpcs_stream* S, void* host_buf, size_t bytes) {
  if (!S || !host_buf) return XPCS_EINVAL;
  xpcs_ctx* ctx = S->ctx;
  size_t need = 0;
  xpcs_stream_checkpoint_size(S, &need);
  if (bytes < need) return fail(ctx, XPCS_EINVAL, "checkpoint buffer too small: need " + std::to_string(need));
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  XPCS_CUDA(ctx, flush_counts(S, true));  // the pair counts deferred by single-frame steps
  XPCS_CUDA(ctx, cudaStreamSynchronize(S->stream));  // every queued batch folded in
  XPCS_TRY(retire(S));
  CkptHeader h{};
  memcpy(h.magic, CKPT_MAGIC, 8);
  h.version = CKPT_VERSION;
  h.k = S->basis->k;
  h.n_q = S->basis->rings->n_q;
  h.dtype = S->dtype;
  h.precision = S->sp;
  h.M = S->basis->rings->M;
  h.W = S->W;
  h.cap = S->cap;
  h.frames = S->frames;
  XPCS_TRY(basis_hash(S, &h.basis_hash));
  void* ptr[5];
  ckpt_parts(S, ptr, h.bytes);
  char* out = static_cast<char*>(host_buf);
  memcpy(out, &h, sizeof(h));
  size_t off = sizeof(h);
  for (int i = 0; i < 5; ++i) {
    XPCS_CUDA(ctx, cudaMemcpy(out + off, ptr[i], h.bytes[i], cudaMemcpyDeviceToHost));
    off += h.bytes[i];
  }
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_stream_restore(xpcs_stream* S, const void* host_buf, size_t bytes) {
  if (!S || !host_buf || bytes < sizeof(CkptHeader)) return XPCS_EINVAL;
  xpcs_ctx* ctx = S->ctx;
  CkptHeader h;
  memcpy(&h, host_buf, sizeof(h));
  if (memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != CKPT_VERSION) return fail(ctx, XPCS_EINVAL, "not a stream checkpoint");
  if (S->frames != 0) return fail(ctx, XPCS_EINVAL, "restore needs a freshly opened stream");
  if (h.k != S->basis->k || h.n_q != S->basis->rings->n_q || h.dtype != S->dtype || h.M != S->basis->rings->M ||
      h.W != S->W || h.cap != S->cap || h.precision != S->sp)
    return fail(ctx, XPCS_EINVAL,
                "checkpoint of a stream with another shape (k, rings, pixels, history, batch, precision)");
  void* ptr[5];
  uint64_t b[5];
  ckpt_parts(S, ptr, b);
  size_t need = sizeof(h);
  for (int i = 0; i < 5; ++i) {
    if (b[i] != h.bytes[i]) return fail(ctx, XPCS_EINVAL, "checkpoint layout does not match the stream");
    need += b[i];
  }
  if (bytes < need) return fail(ctx, XPCS_EINVAL, "checkpoint truncated");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  uint64_t hb = 0;
  XPCS_TRY(basis_hash(S, &hb));
  if (hb != h.basis_hash) return fail(ctx, XPCS_EINVAL, "checkpoint made with another basis");
  XPCS_CUDA(ctx, cudaStreamSynchronize(S->stream));
  const char* in = static_cast<const char*>(host_buf);
  size_t off = sizeof(h);
  for (int i = 0; i < 5; ++i) {
    XPCS_CUDA(ctx, cudaMemcpy(ptr[i], in + off, b[i], cudaMemcpyHostToDevice));
    off += b[i];
  }
  S->frames = h.frames;
  S->cf_blk = -1;  // a checkpoint holds every pair count
  S->cf_cur = S->cf_prev = S->cf_done = 0;
  return XPCS_OK;
}
