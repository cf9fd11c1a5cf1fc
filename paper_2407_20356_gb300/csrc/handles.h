// Library handle types and host helpers shared by the API translation units.
#pragma once
#include <cusolverDn.h>

#include <map>
#include <mutex>
#include <string>
#include <deque>
#include <vector>

#include "internal.h"

// Per-kernel CUDA-event timing (enabled with xpcs_profile_enable).
struct xpcs_prof_entry {
  std::string name;
  double ms = 0.0;
  int64_t launches = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

struct xpcs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  size_t held = 0;
  bool async = false;
  std::string err;
  std::mutex err_mu;  // error text may be written from a server's scheduler thread
  int num_sms = 0;
  uint32_t* d_status = nullptr;  // status word; the u64 8 bytes after it is the wait limit
  uint64_t wait_ns = 0;          // bounded-wait limit of the context's kernels (0: default)
  void* scratch = nullptr;
  size_t scratch_cap = 0;
  cusolverDnHandle_t solver = nullptr;
  uint64_t launches = 0;  // kernels this library has launched on the context
  // work items of the two-time kernel, cached for the last (n_q, nT, CH)
  int4* d_items = nullptr;
  size_t items_n = 0, items_bytes = 0;
  int items_key[4] = {-1, -1, -1, -1};  // (n_q, nT, tiles per item, tile pairs | 2 grouped order)
  bool prof = false;
  std::vector<xpcs_prof_entry> prof_entries;
  std::vector<cudaEvent_t> event_pool;
  // CUDA-graph capture of the context's stream: while capturing, and while graphs made
  // from it exist, nothing the captured work refers to (scratch, work items, lazily made
  // basis copies) may move or change
  // two-time configuration per workload shape (key from gram_tune_key), set by the
  // autotuner; `forced` overrides everything while the autotuner times a candidate
  std::map<uint64_t, std::pair<int, int>> gram_tune;  // key -> (tiles per work item, schedule)
  bool tune_forced = false;
  std::pair<int, int> tune_force{0, 0};
  std::pair<int, int> user_config{0, 0};  // xpcs_twotime_config: (tiles, schedule); tiles 0 = automatic
  bool capturing = false;
  bool async_before_capture = false;
  uint64_t launches_at_capture = 0;
  int graphs = 0;
  // xpcs_encode_host: two copy streams and the events of its staging buffers (made on
  // first use)
  cudaStream_t copy_stream[2] = {nullptr, nullptr};
  int copy_streams = 0;  // host-frame copies on 1 or 2 streams (0: not yet calibrated)
  cudaEvent_t ev_loaded[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_free[3] = {nullptr, nullptr, nullptr};
};

struct xpcs_rings {
  xpcs_ctx* ctx = nullptr;
  int64_t M = 0;
  int n_q = 0;
  int64_t Mp = 0;                 // ring-sorted row length, each ring padded to 64
  std::vector<int64_t> Mq;        // pixels per ring
  std::vector<int> off;           // start of each ring's segment (multiple of 64)
  std::vector<int> chunks;        // 64-wide chunks per ring segment (>= 1)
  int* d_qmap = nullptr;
  int* d_perm = nullptr;          // [Mp] pixel at each sorted position, -1 for padding
  int* d_pos_ring = nullptr;      // [Mp] ring of each sorted position, -1 for padding
  int* d_off = nullptr;
  int* d_chunks = nullptr;
  long long* d_Mq = nullptr;
  size_t bytes = 0;
};

struct xpcs_basis {
  xpcs_ctx* ctx = nullptr;
  const xpcs_rings* rings = nullptr;
  int k = 0;
  int kp = 0;                     // k rounded up to 16: lo half of Bcat starts at row kp
  int n_q = 0;                    // copies of the ring plan's shape: destroying the basis
  int64_t M = 0;                  // never reads the ring plan, which may be gone by then
  int64_t M_pad = 0;
  double* d_B = nullptr;          // M x k
  double* d_G = nullptr;          // n_q x k x k
  double* d_s = nullptr;          // n_q x k
  float2* d_s32 = nullptr;        // n_q x k: s_q as (hi, lo) f32 pieces
  float* d_B32 = nullptr;         // M x k f32 copy of V_K for the sparse streaming encode
                                  // (made on first use)
  float* d_G32 = nullptr;         // n_q x k x k
  __half* d_Bcat = nullptr;       // 2kp x M_pad: f16 hi/lo of V^T 2^enc_log2
  int* d_koff = nullptr;          // n_q zeros: K offsets of the compressed operands
  int* d_kch = nullptr;           // n_q x ceil(k/64): K chunks per operand piece
  __nv_bfloat16* d_Gpair = nullptr;  // n_q kq x 2 kq: bf16 [hi | lo] rows of G_q for the
                                     // tensor-core left operand (made on first use), kq = ceil64(k)
  int enc_log2 = 0;
  size_t bytes = 0;
};

// Online stream (Sec. 2.2, Fig. 1c): a device ring buffer of coefficient rows and
// per-ring factors, and running g2 sums over lags 0..W-1.
struct xpcs_stream {
  xpcs_ctx* ctx = nullptr;
  const xpcs_basis* basis = nullptr;
  cudaStream_t stream = nullptr;     // own CUDA stream: streams overlap on the device
  int64_t W = 0;                     // history window (lags kept)
  int64_t cap = 0;                   // ring slots = max(W + max_batch, 256)
  int max_batch = 0;
  int64_t M = 0;                     // copies of the basis's shape, so that closing the
  int n_q = 0, k = 0;                // stream never reads the basis (which may be gone)
  int64_t frames = 0;                // frames enqueued so far
  int nblk = 0;                      // pixel slices of the sparse encode
  int sp = 0;                        // 1: f16 coefficient rows, one product (XPCS_PREC_FP16);
                                     // 0: bf16 hi | lo rows, three products (XPCS_PREC_BF16X3)
  // pair counts deferred by single-frame steps (count blocks of 64 frames): cf_blk = the
  // block of the latest step (-1: none), cf_cur / cf_prev = deferred frames (bit f: frame
  // 64 block + f) of that block and of the one before, cf_done = the parts (of 64) of the
  // lag range already added for cf_prev
  int64_t cf_blk = -1;
  uint64_t cf_cur = 0, cf_prev = 0, cf_done = 0;
  // device
  void* d_frames = nullptr;          // max_batch x M counts (u16 or u8)
  __nv_bfloat16* d_A2 = nullptr;     // (cap + 128) x 2 kpad coefficient history, bf16 hi | lo
                                     // (f16 streams: 2^e_s a_s in the first kpad, as f16)
  float* d_Rh = nullptr;             // (cap + 128) x npad  r_q(s) = sqrt(M_q)/S~_q(s), 0 if undefined
                                     // (f16 streams: 2^-e_s r_q(s))
  unsigned long long* d_vbits = nullptr;  // n_q x vwords  validity bits r_q(s) > 0 per slot
  float2* d_g2sum = nullptr;         // n_q x Wp (W rounded up to 64): sums as f32 pairs (hi, lo)
  long long* d_cnt = nullptr;        // n_q x Wp
  float* d_part = nullptr;           // max_batch x nblk x k sparse-encode partials
  float* d_a = nullptr;              // max_batch x k
  unsigned* d_se_done = nullptr;     // 128 per-frame counters of the sparse encode's slice blocks
  __nv_bfloat16* d_W2 = nullptr;     // (max_batch n_q) x 2 kpad  r_q(t) a_t G_q, bf16 hi | lo
  double* d_g2 = nullptr;            // n_q x W read-out buffer
  // XPCS_QMEAN_EXACT_RAW: the stream's own copy of the ring labels (M) and a step's exact
  // ring sums (64 x n_q), both null otherwise
  int* d_qmap = nullptr;
  long long* d_Sx = nullptr;
  // steps on the two-time kernel: the block's w rows per ring (zero outside a step), partials
  __nv_bfloat16* d_Wg = nullptr;     // n_q x 128 x 2 kpad
  float* d_gpart = nullptr;          // n_q x nd x 256
  CUtensorMap tmWg, tmWg2;           // boxes of 128 and 256 rows
  CUtensorMap tmW48;                 // d_W2 in boxes of 64 x 48 (single-frame steps)
  int kpad = 0;                      // k rounded up to 64
  CUtensorMap tmA, tmW, tmR;         // tensor maps of d_A2, d_W2 (64 x 128 boxes) and d_Rh
  // tensor maps of d_g2sum and d_cnt (row pitch Wp), one per row-update lag tile RT_LTS[i]
  CUtensorMap tmG[xpcs::RT_N_LT], tmC[xpcs::RT_N_LT];
  uint32_t* h_status = nullptr;      // host-mapped status word of the stream's kernels
  uint32_t* d_status = nullptr;      // its device address
  size_t bytes = 0;
  // host
  void* h_stage[2] = {nullptr, nullptr};  // pinned staging, double-buffered
  cudaEvent_t stage_done[2] = {nullptr, nullptr};
  int stage_i = 0;
  int dtype = -1;
  // per-batch latency stamps: arrival and completion times (host steady clock, ns)
  struct Stamp {
    std::vector<int64_t> arrive_ns;  // one per frame of the batch
    int64_t done_ns = 0;             // 0 while the batch is in flight
  };
  struct Ticket {
    uint64_t frames;  // frames pushed up to and including this batch
    cudaEvent_t ev;   // recorded behind the batch's kernels (timing enabled)
    Stamp* stamp;
  };
  std::deque<Ticket> tickets;
  std::vector<cudaEvent_t> event_pool;
  std::vector<Stamp*> stamps;
  // completion times come from CUDA event timing relative to a base event whose host
  // time is known: done_ns = base_ns + elapsed(base_ev, ev)
  cudaEvent_t base_ev = nullptr;
  int64_t base_ns = 0;
};

namespace xpcs {

size_t stream_footprint(const xpcs_basis* B, int64_t W, int max_batch, int elem_bytes);
int64_t now_ns();
// Push n host frames through the next staging buffer.  arrive_ns (nullable) gives each
// frame's arrival time for the latency record.  With block == false the call does nothing
// and returns XPCS_EBUSY while that buffer's previous copy is still in flight.
xpcs_status stream_push_host(xpcs_stream* S, const void* frames, int64_t n, const int64_t* arrive_ns, bool block);
// Enqueue n frames that are already in device memory (read by the stream's kernels in place,
// so they must stay unchanged until the stream has folded them in), with arrival stamps.
xpcs_status stream_push_device_stamped(xpcs_stream* S, const void* frames, int64_t n, const int64_t* arrive_ns);
// Batches of the stream still on the device (after retiring the finished ones).
int stream_inflight(xpcs_stream* S);

xpcs_status fail(xpcs_ctx* ctx, xpcs_status s, const std::string& msg);
xpcs_status dev_alloc(xpcs_ctx* ctx, void** p, size_t bytes);
void dev_free(xpcs_ctx* ctx, void* p, size_t bytes);
xpcs_status ensure_scratch(xpcs_ctx* ctx, size_t need);
xpcs_status rings_from_host(xpcs_ctx* ctx, const int32_t* qmap_host, int64_t M, int n_q, xpcs_rings** out);
xpcs_status finish(xpcs_ctx* ctx);
xpcs_status make_map(xpcs_ctx* ctx, CUtensorMap* map, const void* base, CUtensorMapDataType dt, int elem_bytes,
                     uint64_t cols, uint64_t rows, uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle sw,
                     uint64_t pitch_bytes = 0);

// Default two-time configurations (tiles per work item, schedule: 0 = single tiles, 1 =
// tile pairs), from timings on one GB300.  Raw counts: tile pairs (the long K loop is
// bound by operand traffic, which pairs cut by a quarter), one tile pair per work item
// (512x512, T = 10^4: 17.5 ms against 24.4 ms with 4), more only where the g2 partial
// slots (1 KB per ring, tile diagonal and work-item chunk) would pass 512 MB.  Compressed
// with C stored: single tiles, 8 per item (bound by the C stores).  Compressed g2 only
// (merged items, one diagonal pass per item): tile pairs, 4 tiles per item.
inline std::pair<int, int> gram_default_raw(int n_q, int nT) {
  int ch = 1;
  while (ch < 64 && (double)n_q * nT * ((nT + ch - 1) / ch) * DIAG_SLOTS * 4 > 512.0 * (1 << 20)) ch *= 2;
  return {ch, 1};
}
inline std::pair<int, int> gram_default_compressed(bool merge) {
  if (merge) return {4, 1};
  return {CHUNK_TILES, 0};
}

// Key of a two-time workload shape in the context's tuning table.
inline uint64_t gram_tune_key(int n_q, int nT, int fmt, int split, int raw, bool C) {
  return ((uint64_t)n_q << 40) | ((uint64_t)nT << 16) | ((uint64_t)fmt << 4) | ((uint64_t)split << 3) |
         ((uint64_t)raw << 2) | (C ? 2u : 0u);
}

// Split-K partial floats of the encode of T frames, and the encode of device frames on a
// given CUDA stream (encode.cu)
size_t encode_partials(const xpcs_basis* B, int64_t T, int num_sms);
xpcs_status encode_on_stream(xpcs_ctx* ctx, const xpcs_basis* B, const void* X, xpcs_dtype dtype, int64_t T,
                             float* A_out, float* partials, uint32_t* status, cudaStream_t st);

// Scratch: one growing device buffer per context, carved per call.
struct Carve {
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Records CUDA events around one launch site when profiling is on.
struct ProfScope {
  xpcs_ctx* ctx;
  const char* name;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(xpcs_ctx* c, const char* n);
  void done();
};

}  // namespace xpcs

// Launch through a library launcher, counting `nk` kernels and timing the site.
#define XPCS_LAUNCH(ctx, name, nk, call)                                                              \
  do {                                                                                                \
    ::xpcs::ProfScope ps_((ctx), (name));                                                             \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      return ::xpcs::fail((ctx), XPCS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    (ctx)->launches += (nk);                                                                          \
    ps_.done();                                                                                       \
  } while (0)

#define XPCS_CUDA(ctx, call)                                                                          \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      return ::xpcs::fail((ctx), XPCS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

#define XPCS_TRY(expr)            \
  do {                            \
    xpcs_status s_ = (expr);      \
    if (s_ != XPCS_OK) return s_; \
  } while (0)
