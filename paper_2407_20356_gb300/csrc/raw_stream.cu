// Online two-time correlation on RAW frames: the raw-path counterpart of the compressed
// stream (Sec. 2.2 online mode, against which Sec. 3.2 times the compressed path).
//
// The history is kept as the raw path keeps its frames: counts gathered into ring-sorted
// order as bf16 (exact for counts <= 256), one row per frame, in a ring of nb blocks of
// 128 frames (frame t in row t mod 128 nb).  A step of b <= 64 new frames, all in one
// 128-frame block J, costs:
//   1. ingest: gather the b frames into their rows, exact ring sums S_q(t) and sums of
//      squares (the 2^24 exactness bound of the f32 Gram);
//   2. factors: r_q(t) = sqrt(M_q) / S_q(t) (0 if undefined) for the row scales and, for
//      these frames only, the column scales;
//   3. the two-time tile kernel in raw mode over tiles (history block J - delta, block J)
//      for every ring and delta < nd: the exact integer Gram N_q(s, t) on the tensor
//      cores, C = r(s) r(t) N, and its diagonal sums by lag t - s (columns of frames that
//      are not new have scale 0, so only the new rows of the two-time matrix count);
//   4. fold: the diagonal sums of lags tau < W are added to running FP64 sums and the pair
//      counts (both frames defined) to running counts.
// Steps of one frame read the whole history window (W x M bf16) once, like a dense raw
// row update must; larger steps reuse every history tile for all their frames.
#include <math.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "handles.h"
#include "internal.h"

using namespace xpcs;

struct xpcs_raw_stream {
  xpcs_ctx* ctx = nullptr;
  const xpcs_rings* rings = nullptr;  // must stay alive while frames are pushed
  int64_t W = 0;                      // lags kept
  int nb = 0;                         // 128-frame blocks in the history ring
  int nd = 0;                         // tile diagonals that can hold a lag < W
  int n_q = 0;
  int dtype = 0;
  int64_t M = 0, Mp = 0;
  int64_t frames = 0;
  __nv_bfloat16* d_Xp = nullptr;  // (128 nb) x Mp ring-sorted bf16 counts
  float* d_r = nullptr;           // n_q x (128 nb) row scales sqrt(M_q)/S_q(t)
  float* d_rc = nullptr;          // n_q x (128 nb) column scales: nonzero only during a step
  long long* d_S = nullptr;       // n_q x 128 ring sums of a step's frames
  long long* d_S2 = nullptr;      // n_q x 128 sums of squares
  float* d_part = nullptr;        // n_q x nd x nb x 256 diagonal partial sums
  double* d_g2sum = nullptr;      // n_q x W
  long long* d_cnt = nullptr;     // n_q x W
  double* d_g2 = nullptr;         // n_q x W read-out
  size_t bytes = 0;
};

namespace {

constexpr int RS_STEP = 128;  // frames per step at most (one 128-frame block)

__global__ void raw_stream_factors_kernel(const long long* S, const long long* S2, const long long* Mq, int n_q,
                                          int b, long long slot0, long long rows, float* r, float* rc,
                                          uint32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_q * b) return;
  const int q = i / b, f = i - q * b;
  const long long s = S[(size_t)q * b + f];
  if (S2[(size_t)q * b + f] >= (1ll << 24)) set_status(status, XPCS_DEV_RANGE);
  const float v = s > 0 ? (float)(sqrt((double)Mq[q]) / (double)s) : 0.f;
  r[(size_t)q * rows + slot0 + f] = v;
  rc[(size_t)q * rows + slot0 + f] = v;
}

// Adds the step's diagonal sums of lags tau < W to the running sums, counts the step's
// defined pairs per lag, and clears the step's column scales.  Lag tau = 128 d + e is
// slot 128 + e of tile diagonal d and slot e of tile diagonal d + 1.
__global__ void raw_stream_fold_kernel(const float* part, int n_q, int nd, int nd_step, int nb, int J, long long W,
                                       long long t0, int b, long long rows, const float* r, float* rc, double* g2sum,
                                       long long* cnt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long span = W > b ? W : b;
  if (i >= (long long)n_q * span) return;
  const int q = (int)(i / span);
  const long long tau = i - (long long)q * span;
  if (tau < W) {
    const int d = (int)(tau >> 7), e = (int)(tau & 127);
    double sum = 0.0;
    if (d < nd_step) {
      const int c = ((J - d) % nb + nb) % nb;
      sum += (double)part[(((size_t)q * nd + d) * nb + c) * DIAG_SLOTS + TILE + e];
    }
    if (d + 1 < nd_step) {
      const int c = ((J - d - 1) % nb + nb) % nb;
      sum += (double)part[(((size_t)q * nd + d + 1) * nb + c) * DIAG_SLOTS + e];
    }
    long long n = 0;
    const float* rq = r + (size_t)q * rows;
    for (int f = 0; f < b; ++f) {
      const long long t = t0 + f, s = t - tau;
      if (s >= 0 && rq[t % rows] > 0.f && rq[s % rows] > 0.f) ++n;
    }
    g2sum[(size_t)q * W + tau] += sum;
    cnt[(size_t)q * W + tau] += n;
  }
  if (tau < b) rc[(size_t)q * rows + (t0 + tau) % rows] = 0.f;
}

__global__ void raw_stream_g2_kernel(const double* g2sum, const long long* cnt, long long n, double* g2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g2[i] = cnt[i] > 0 ? g2sum[i] / (double)cnt[i] : __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace

namespace {

void raw_stream_free(xpcs_raw_stream* R) {
  xpcs_ctx* ctx = R->ctx;
  cudaStreamSynchronize(ctx->stream);
  const size_t rows = (size_t)128 * R->nb;
  dev_free(ctx, R->d_Xp, rows * R->Mp * 2);
  dev_free(ctx, R->d_r, (size_t)R->n_q * rows * 4);
  dev_free(ctx, R->d_rc, (size_t)R->n_q * rows * 4);
  dev_free(ctx, R->d_S, (size_t)R->n_q * RS_STEP * 8);
  dev_free(ctx, R->d_S2, (size_t)R->n_q * RS_STEP * 8);
  dev_free(ctx, R->d_part, (size_t)R->n_q * R->nd * R->nb * DIAG_SLOTS * 4);
  dev_free(ctx, R->d_g2sum, (size_t)R->n_q * R->W * 8);
  dev_free(ctx, R->d_cnt, (size_t)R->n_q * R->W * 8);
  dev_free(ctx, R->d_g2, (size_t)R->n_q * R->W * 8);
  delete R;
}

// One step: b frames of one 128-frame block.
xpcs_status raw_stream_step(xpcs_raw_stream* R, const void* X, int b) {
  xpcs_ctx* ctx = R->ctx;
  const xpcs_rings* P = R->rings;
  const long long t0 = R->frames;
  const long long rows = 128LL * R->nb;
  const int J = (int)((t0 >> 7) % R->nb);
  const long long slot0 = t0 % rows;
  RawIngestParams ip{};
  ip.X = X;
  ip.dtype = R->dtype;
  ip.T = b;
  ip.M = R->M;
  ip.T_pad = b;
  ip.Mp = R->Mp;
  ip.perm = P->d_perm;
  ip.pos_ring = P->d_pos_ring;
  ip.n_q = R->n_q;
  ip.Xp = R->d_Xp;
  ip.xp_row0 = slot0;
  ip.S = R->d_S;
  ip.S2 = R->d_S2;
  ip.status = ctx->d_status;
  XPCS_LAUNCH(ctx, "raw_stream_ingest", 1, launch_raw_ingest(ip, ctx->stream));
  XPCS_LAUNCH(ctx, "raw_stream_factors", 1,
              (raw_stream_factors_kernel<<<(R->n_q * b + 127) / 128, 128, 0, ctx->stream>>>(
                   R->d_S, R->d_S2, P->d_Mq, R->n_q, b, slot0, rows, R->d_r, R->d_rc, ctx->d_status),
               cudaGetLastError()));
  // tile diagonals that exist so far (blocks before the first frame hold nothing)
  const int nd_step = (int)std::min<long long>(R->nd, (t0 >> 7) + 1);
  CUtensorMap tm;
  XPCS_TRY(make_map(ctx, &tm, R->d_Xp, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, R->Mp, rows, KCH, TILE,
                    CU_TENSOR_MAP_SWIZZLE_128B));
  GramParams gp{};
  gp.T = (int)rows;
  gp.nT = R->nd;  // partial layout: [n_q][nd][nb][256]
  gp.T_pad = (int)rows;
  gp.maxC = R->nb;
  gp.CH = 1;
  gp.n_items = R->n_q * nd_step;
  gp.items = nullptr;
  gp.ring_nb = R->nb;
  gp.ring_nd = nd_step;
  gp.ring_J = J;
  gp.k_off = P->d_off;
  gp.k_chunks = P->d_chunks;
  gp.ring_rows = 0;
  gp.fmt = 1;
  gp.raw = 1;
  gp.r = R->d_r;
  gp.rc = R->d_rc;
  gp.partials = R->d_part;
  gp.status = ctx->d_status;
  XPCS_LAUNCH(ctx, "raw_stream_gram", 1, launch_gram(tm, tm, gp, std::min(gp.n_items, ctx->num_sms), ctx->stream));
  const long long span = std::max<long long>(R->W, b);
  XPCS_LAUNCH(ctx, "raw_stream_fold", 1,
              (raw_stream_fold_kernel<<<(unsigned)((R->n_q * span + 255) / 256), 256, 0, ctx->stream>>>(
                   R->d_part, R->n_q, R->nd, nd_step, R->nb, J, R->W, t0, b, rows, R->d_r, R->d_rc, R->d_g2sum,
                   R->d_cnt),
               cudaGetLastError()));
  R->frames += b;
  return XPCS_OK;
}

}  // namespace

extern "C" xpcs_status xpcs_raw_stream_open(xpcs_ctx* ctx, const xpcs_rings* P, int64_t history, xpcs_dtype dtype,
                                            xpcs_raw_stream** out) {
  if (!ctx || !P || !out || P->ctx != ctx || history < 1 || history > (1 << 24) ||
      (dtype != XPCS_U8 && dtype != XPCS_U16))
    return fail(ctx, XPCS_EINVAL, "bad raw_stream_open args");
  *out = nullptr;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  auto* R = new xpcs_raw_stream();
  R->ctx = ctx;
  R->rings = P;
  R->W = history;
  R->nd = (int)((history + 126) / 128 + 1);  // lag 128 d + e < W needs d <= (W - 1 + 127) / 128
  R->nb = R->nd + 1;
  R->n_q = P->n_q;
  R->dtype = dtype;
  R->M = P->M;
  R->Mp = P->Mp;
  const size_t rows = (size_t)128 * R->nb;
  const size_t sz[9] = {rows * R->Mp * 2,
                        (size_t)R->n_q * rows * 4,
                        (size_t)R->n_q * rows * 4,
                        (size_t)R->n_q * RS_STEP * 8,
                        (size_t)R->n_q * RS_STEP * 8,
                        (size_t)R->n_q * R->nd * R->nb * DIAG_SLOTS * 4,
                        (size_t)R->n_q * history * 8,
                        (size_t)R->n_q * history * 8,
                        (size_t)R->n_q * history * 8};
  void* p[9] = {};
  xpcs_status st = XPCS_OK;
  for (int i = 0; i < 9 && st == XPCS_OK; ++i) st = dev_alloc(ctx, &p[i], sz[i]);
  R->d_Xp = static_cast<__nv_bfloat16*>(p[0]);
  R->d_r = static_cast<float*>(p[1]);
  R->d_rc = static_cast<float*>(p[2]);
  R->d_S = static_cast<long long*>(p[3]);
  R->d_S2 = static_cast<long long*>(p[4]);
  R->d_part = static_cast<float*>(p[5]);
  R->d_g2sum = static_cast<double*>(p[6]);
  R->d_cnt = static_cast<long long*>(p[7]);
  R->d_g2 = static_cast<double*>(p[8]);
  for (int i = 0; i < 9; ++i) R->bytes += p[i] ? sz[i] : 0;
  cudaError_t e = cudaSuccess;
  for (int i : {0, 1, 2, 6, 7})  // history rows, scales, running sums and counts start at zero
    if (st == XPCS_OK && e == cudaSuccess) e = cudaMemsetAsync(p[i], 0, sz[i], ctx->stream);
  if (st == XPCS_OK && e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (st == XPCS_OK && e != cudaSuccess) st = fail(ctx, XPCS_ECUDA, std::string("raw stream setup: ") + cudaGetErrorString(e));
  if (st != XPCS_OK) {
    raw_stream_free(R);
    return st;
  }
  *out = R;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_raw_stream_push_device(xpcs_raw_stream* R, const void* frames, int64_t n) {
  if (!R || !frames || n < 0) return XPCS_EINVAL;
  xpcs_ctx* ctx = R->ctx;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t fb = (size_t)R->M * (R->dtype == XPCS_U8 ? 1 : 2);
  for (int64_t f0 = 0; f0 < n;) {
    // steps that do not cross a 128-frame block
    const int64_t room = 128 - (R->frames & 127);
    const int b = (int)std::min<int64_t>({RS_STEP, room, n - f0});
    XPCS_TRY(raw_stream_step(R, static_cast<const char*>(frames) + f0 * fb, b));
    f0 += b;
  }
  return finish(ctx);
}

extern "C" xpcs_status xpcs_raw_stream_read_g2(xpcs_raw_stream* R, double* g2_host, int64_t* count_host) {
  if (!R) return XPCS_EINVAL;
  xpcs_ctx* ctx = R->ctx;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const long long n = (long long)R->n_q * R->W;
  XPCS_LAUNCH(ctx, "raw_stream_g2", 1,
              (raw_stream_g2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(R->d_g2sum, R->d_cnt, n,
                                                                                           R->d_g2),
               cudaGetLastError()));
  if (g2_host) XPCS_CUDA(ctx, cudaMemcpyAsync(g2_host, R->d_g2, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (count_host) XPCS_CUDA(ctx, cudaMemcpyAsync(count_host, R->d_cnt, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return xpcs_synchronize(ctx);
}

extern "C" int64_t xpcs_raw_stream_frames(const xpcs_raw_stream* R) { return R ? R->frames : -1; }

extern "C" xpcs_status xpcs_raw_stream_close(xpcs_raw_stream* R) {
  if (!R) return XPCS_EINVAL;
  raw_stream_free(R);
  return XPCS_OK;
}
