// C ABI of the library: contexts, ring plans, bases and the offline correlation paths.
#include <cudaTypedefs.h>
#include <cusolverDn.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "handles.h"
#include "internal.h"

using namespace xpcs;

// ====================================================================== helpers

namespace xpcs {

xpcs_status fail(xpcs_ctx* ctx, xpcs_status s, const std::string& msg) {
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    ctx->err = msg;
  }
  return s;
}

xpcs_status dev_alloc(xpcs_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return XPCS_OK;
  if (ctx->budget && ctx->held + bytes > ctx->budget)
    return fail(ctx, XPCS_ENOMEM, "device memory budget exceeded (" + std::to_string(ctx->held + bytes) + " > " +
                                      std::to_string(ctx->budget) + " bytes)");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, XPCS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ctx->held += bytes;
  return XPCS_OK;
}

void dev_free(xpcs_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  ctx->held -= std::min(ctx->held, bytes);
}

xpcs_status ensure_scratch(xpcs_ctx* ctx, size_t need) {
  if (need <= ctx->scratch_cap) return XPCS_OK;
  if (ctx->capturing || ctx->graphs > 0)
    return fail(ctx, XPCS_EBUSY,
                "the context's scratch cannot grow during a capture or while captured graphs exist: run the "
                "largest call once before capturing");
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  dev_free(ctx, ctx->scratch, ctx->scratch_cap);
  ctx->scratch = nullptr;
  ctx->scratch_cap = 0;
  const size_t cap = need + need / 8;
  void* p = nullptr;
  XPCS_TRY(dev_alloc(ctx, &p, cap));
  ctx->scratch = p;
  ctx->scratch_cap = cap;
  return XPCS_OK;
}

// Wait for the context's work (unless asynchronous) and map the device status word.
xpcs_status finish(xpcs_ctx* ctx) {
  if (ctx->async) return XPCS_OK;
  return xpcs_synchronize(ctx);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// 2-D tiled map of a row-major [rows][cols] matrix (row pitch in bytes; 0 = dense),
// box = box_cols x box_rows, with the given swizzle.
xpcs_status make_map(xpcs_ctx* ctx, CUtensorMap* map, const void* base, CUtensorMapDataType dt, int elem_bytes,
                     uint64_t cols, uint64_t rows, uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle sw,
                     uint64_t pitch_bytes) {
  auto fn = get_encode_fn();
  if (!fn) return fail(ctx, XPCS_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  const uint64_t pitch = pitch_bytes ? pitch_bytes : cols * (uint64_t)elem_bytes;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (pitch & 15))
    return fail(ctx, XPCS_ENOTSUP, "tensor map needs 16-byte aligned base and row pitch");
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {pitch};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, XPCS_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return XPCS_OK;
}

ProfScope::ProfScope(xpcs_ctx* c, const char* n) : ctx(c), name(n) {
  if (!ctx->prof) return;
  for (cudaEvent_t* e : {&a, &b}) {
    if (!ctx->event_pool.empty()) {
      *e = ctx->event_pool.back();
      ctx->event_pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      *e = nullptr;
    }
  }
  if (a) cudaEventRecord(a, ctx->stream);
}

void ProfScope::done() {
  if (!ctx->prof || !a || !b) return;
  cudaEventRecord(b, ctx->stream);
  for (auto& en : ctx->prof_entries)
    if (en.name == name) {
      en.pending.push_back({a, b});
      en.launches += 1;
      return;
    }
  xpcs_prof_entry en;
  en.name = name;
  en.pending.push_back({a, b});
  en.launches = 1;
  ctx->prof_entries.push_back(std::move(en));
}

}  // namespace xpcs

namespace {

// Work items of the two-time kernel: (q, delta, I0, I1), the tiles (I, I+delta) of one
// tile diagonal (with tile pairs also (I, I+delta+1); delta then runs over even values),
// CH tiles per item.  Calls that store C take them ring by ring, chunk by chunk, delta
// ascending, so that the CTAs running together write neighbouring row blocks of C.  The
// others (raw counts with their long K loop, g2-only calls), bound by operand traffic,
// take this grouped order, ring by ring: items of full length first, then the shorter
// ones at the triangle's edge, so that items launched together also finish together;
// within each group items come in blocks of consecutive e = I0 + delta (the R row block of
// the item's first tile), all chunks c = I0 / CH of a block together.  Items with the same
// c read the same L row blocks at every step and items with the same e the same R row
// blocks, so the items that a persistent grid of `grid` CTAs runs at one time share their
// operand panels in L2.
std::vector<int4> make_items(int n_q, int nT, int CH, int pairs, int grid, bool grouped) {
  const int step = pairs ? 2 : 1;
  const int nC = (nT + CH - 1) / CH;
  if (!grouped) {  // ring by ring, chunk by chunk, delta ascending (consecutive C row blocks)
    std::vector<int4> items;
    for (int q = 0; q < n_q; ++q)
      for (int c = 0; c < nC; ++c)
        for (int d = 0; d < nT; d += step) {
          const int I0 = c * CH, I1 = std::min(c * CH + CH, nT - d);
          if (I0 < I1) items.push_back(make_int4(q, d, I0, I1));
        }
    return items;
  }
  // e-block width: about `grid` items per block over all chunks
  const int eb = std::max(step, (grid * step + nC - 1) / nC);
  std::vector<int4> items;
  std::vector<std::pair<long long, int4>> ring;
  for (int q = 0; q < n_q; ++q) {
    ring.clear();
    for (int c = 0; c < nC; ++c)
      for (int d = 0; d < nT; d += step) {
        const int I0 = c * CH, I1 = std::min(c * CH + CH, nT - d);
        if (I0 >= I1) continue;
        const int e = I0 + d;
        const long long full = (I1 - I0 == CH) ? 0 : 1;
        const long long key = ((full * (nT / eb + 1) + e / eb) * (long long)nC + c) * (nT + 1) + e;
        ring.push_back({key, make_int4(q, d, I0, I1)});
      }
    std::sort(ring.begin(), ring.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (const auto& kv : ring) items.push_back(kv.second);
  }
  return items;
}

// Device copy of the work items for (n_q, nT, CH), rebuilt only when they change.
xpcs_status cached_items(xpcs_ctx* ctx, int n_q, int nT, int CH, int pairs, bool grouped, int4** d_items,
                         int* n_items) {
  const int key3 = pairs | (grouped ? 2 : 0);
  if (ctx->items_key[0] != n_q || ctx->items_key[1] != nT || ctx->items_key[2] != CH ||
      ctx->items_key[3] != key3) {
    if (ctx->capturing || ctx->graphs > 0)
      return fail(ctx, XPCS_EBUSY,
                  "two-time work items of another shape cannot be built during a capture or while captured "
                  "graphs exist: run the call once before capturing");
    const std::vector<int4> items = make_items(n_q, nT, CH, pairs, ctx->num_sms, grouped);
    const size_t bytes = items.size() * sizeof(int4);
    if (bytes > ctx->items_bytes) {
      XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      dev_free(ctx, ctx->d_items, ctx->items_bytes);
      ctx->d_items = nullptr;
      ctx->items_bytes = 0;
      void* p = nullptr;
      XPCS_TRY(dev_alloc(ctx, &p, bytes));
      ctx->d_items = static_cast<int4*>(p);
      ctx->items_bytes = bytes;
    } else {
      XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // earlier kernels may still read them
    }
    XPCS_CUDA(ctx, cudaMemcpy(ctx->d_items, items.data(), bytes, cudaMemcpyHostToDevice));
    ctx->items_n = items.size();
    ctx->items_key[0] = n_q;
    ctx->items_key[1] = nT;
    ctx->items_key[2] = CH;
    ctx->items_key[3] = key3;
  }
  *d_items = ctx->d_items;
  *n_items = (int)ctx->items_n;
  return XPCS_OK;
}

}  // namespace

// ====================================================================== context

extern "C" int xpcs_version(void) { return 100; }

extern "C" xpcs_status xpcs_create(int device, size_t hbm_budget_bytes, void* cuda_stream, xpcs_ctx** out) {
  if (!out) return XPCS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return XPCS_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return XPCS_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return XPCS_ECUDA;
  if (prop.major * 10 + prop.minor < 100) return XPCS_ENOTSUP;
  auto* ctx = new xpcs_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  ctx->num_sms = prop.multiProcessorCount;
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return XPCS_ECUDA;
    }
    ctx->own_stream = true;
  }
  void* st = nullptr;
  if (dev_alloc(ctx, &st, 256) != XPCS_OK || cudaMemset(st, 0, 256) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return XPCS_ENOMEM;
  }
  ctx->d_status = static_cast<uint32_t*>(st);
  *out = ctx;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_destroy(xpcs_ctx* ctx) {
  if (!ctx) return XPCS_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, ctx->scratch, ctx->scratch_cap);
  dev_free(ctx, ctx->d_items, ctx->items_bytes);
  dev_free(ctx, ctx->d_status, 256);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  xpcs_profile_enable(ctx, 0);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i)
    if (ctx->copy_stream[i]) {
      cudaStreamSynchronize(ctx->copy_stream[i]);
      cudaStreamDestroy(ctx->copy_stream[i]);
    }
  for (int i = 0; i < 3; ++i) {
    if (ctx->ev_loaded[i]) cudaEventDestroy(ctx->ev_loaded[i]);
    if (ctx->ev_free[i]) cudaEventDestroy(ctx->ev_free[i]);
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return XPCS_OK;
}

extern "C" const char* xpcs_last_error(const xpcs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" xpcs_status xpcs_set_async(xpcs_ctx* ctx, int async) {
  if (!ctx) return XPCS_EINVAL;
  ctx->async = async != 0;
  return XPCS_OK;
}

extern "C" size_t xpcs_device_bytes(const xpcs_ctx* ctx) { return ctx ? ctx->held : 0; }

extern "C" uint64_t xpcs_launch_count(const xpcs_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" xpcs_status xpcs_profile_enable(xpcs_ctx* ctx, int on) {
  if (!ctx) return XPCS_EINVAL;
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto& en : ctx->prof_entries)
    for (auto& pr : en.pending) {
      ctx->event_pool.push_back(pr.first);
      ctx->event_pool.push_back(pr.second);
    }
  ctx->prof_entries.clear();
  ctx->prof = on != 0;
  return XPCS_OK;
}

extern "C" int xpcs_profile_count(const xpcs_ctx* ctx) { return ctx ? (int)ctx->prof_entries.size() : 0; }

extern "C" xpcs_status xpcs_profile_get(xpcs_ctx* ctx, int i, char* name_host, size_t name_cap, double* ms_host,
                                        int64_t* launches_host) {
  if (!ctx || i < 0 || i >= (int)ctx->prof_entries.size()) return fail(ctx, XPCS_EINVAL, "bad profile index");
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  auto& en = ctx->prof_entries[i];
  for (auto& pr : en.pending) {
    float ms = 0.f;
    XPCS_CUDA(ctx, cudaEventElapsedTime(&ms, pr.first, pr.second));
    en.ms += ms;
    ctx->event_pool.push_back(pr.first);
    ctx->event_pool.push_back(pr.second);
  }
  en.pending.clear();
  if (name_host && name_cap) {
    strncpy(name_host, en.name.c_str(), name_cap - 1);
    name_host[name_cap - 1] = 0;
  }
  if (ms_host) *ms_host = en.ms;
  if (launches_host) *launches_host = en.launches;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_synchronize(xpcs_ctx* ctx) {
  if (!ctx) return XPCS_EINVAL;
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  uint32_t st = 0;
  XPCS_CUDA(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st != XPCS_DEV_OK) {
    XPCS_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(uint32_t)));
    if (st == XPCS_DEV_TIMEOUT) return fail(ctx, XPCS_ETIMEOUT, "a bounded device wait expired");
    if (st == XPCS_DEV_RANGE)
      return fail(ctx, XPCS_ERANGE,
                  "counts outside the exact range (a count above 256, or a ring whose per-frame sum of squared "
                  "counts reaches 2^24)");
    return fail(ctx, XPCS_ECUDA, "device status " + std::to_string(st));
  }
  return XPCS_OK;
}

// ====================================================================== rings

namespace xpcs {

// Ring plan from a host label array (labels in [-1, n_q)).
xpcs_status rings_from_host(xpcs_ctx* ctx, const int32_t* h, int64_t M, int n_q, xpcs_rings** out) {
  *out = nullptr;
  auto* r = new xpcs_rings();
  r->ctx = ctx;
  r->M = M;
  r->n_q = n_q;
  r->Mq.assign(n_q, 0);
  for (int64_t p = 0; p < M; ++p) {
    if (h[p] >= n_q || h[p] < -1) {
      delete r;
      return fail(ctx, XPCS_EINVAL, "qmap label outside [-1, n_q)");
    }
    if (h[p] >= 0) r->Mq[h[p]]++;
  }
  r->off.resize(n_q);
  r->chunks.resize(n_q);
  int64_t o = 0;
  for (int q = 0; q < n_q; ++q) {
    r->off[q] = (int)o;
    const int64_t ch = std::max<int64_t>(1, (r->Mq[q] + KCH - 1) / KCH);
    r->chunks[q] = (int)ch;
    o += ch * KCH;
  }
  if (o > (int64_t)INT32_MAX / 2) {
    delete r;
    return fail(ctx, XPCS_ENOTSUP, "detector too large");
  }
  r->Mp = o;
  std::vector<int> perm(r->Mp, -1), pos(r->Mp, -1), fill(n_q, 0);
  for (int64_t p = 0; p < M; ++p) {
    const int q = h[p];
    if (q < 0) continue;
    const int at = r->off[q] + fill[q]++;
    perm[at] = (int)p;
    pos[at] = q;
  }
  std::vector<long long> mq(r->Mq.begin(), r->Mq.end());
  xpcs_status s = XPCS_OK;
  void* p[6] = {};
  const size_t sz[6] = {(size_t)M * 4, (size_t)r->Mp * 4, (size_t)r->Mp * 4, (size_t)n_q * 4, (size_t)n_q * 4,
                        (size_t)n_q * 8};
  for (int i = 0; i < 6 && s == XPCS_OK; ++i) s = dev_alloc(ctx, &p[i], sz[i]);
  if (s != XPCS_OK) {
    for (int i = 0; i < 6; ++i) dev_free(ctx, p[i], sz[i]);
    delete r;
    return s;
  }
  r->d_qmap = (int*)p[0];
  r->d_perm = (int*)p[1];
  r->d_pos_ring = (int*)p[2];
  r->d_off = (int*)p[3];
  r->d_chunks = (int*)p[4];
  r->d_Mq = (long long*)p[5];
  r->bytes = sz[0] + sz[1] + sz[2] + sz[3] + sz[4] + sz[5];
  cudaError_t e = cudaMemcpy(r->d_qmap, h, sz[0], cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_perm, perm.data(), sz[1], cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_pos_ring, pos.data(), sz[2], cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_off, r->off.data(), sz[3], cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_chunks, r->chunks.data(), sz[4], cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_Mq, mq.data(), sz[5], cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    xpcs_rings_destroy(r);
    return fail(ctx, XPCS_ECUDA, std::string("ring plan upload: ") + cudaGetErrorString(e));
  }
  *out = r;
  return XPCS_OK;
}

}  // namespace xpcs

extern "C" xpcs_status xpcs_rings_create(xpcs_ctx* ctx, const int32_t* qmap, int64_t M, int n_q, xpcs_rings** out) {
  if (!ctx || !qmap || !out || M <= 0 || n_q <= 0 || n_q > 1024) return fail(ctx, XPCS_EINVAL, "bad ring plan args");
  *out = nullptr;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  std::vector<int32_t> h(M);
  XPCS_CUDA(ctx, cudaMemcpyAsync(h.data(), qmap, M * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return rings_from_host(ctx, h.data(), M, n_q, out);
}

extern "C" xpcs_status xpcs_rings_destroy(xpcs_rings* r) {
  if (!r) return XPCS_EINVAL;
  xpcs_ctx* ctx = r->ctx;
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, r->d_qmap, (size_t)r->M * 4);
  dev_free(ctx, r->d_perm, (size_t)r->Mp * 4);
  dev_free(ctx, r->d_pos_ring, (size_t)r->Mp * 4);
  dev_free(ctx, r->d_off, (size_t)r->n_q * 4);
  dev_free(ctx, r->d_chunks, (size_t)r->n_q * 4);
  dev_free(ctx, r->d_Mq, (size_t)r->n_q * 8);
  delete r;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_rings_sizes(const xpcs_rings* r, int64_t* Mq_host) {
  if (!r || !Mq_host) return XPCS_EINVAL;
  for (int q = 0; q < r->n_q; ++q) Mq_host[q] = r->Mq[q];
  return XPCS_OK;
}

// ====================================================================== raw path

namespace {

struct RawBuffers {
  __nv_bfloat16* Xp;
  long long* S;
  long long* S2;  // per-frame sums of squares (the exactness bound; Frobenius scales)
  double* Sbar;   // ring means of S (Eq. 12 normalisation only)
  float* r;
  uint32_t* blk_bad;
  float* partials;
  uint32_t* vbits;
  long long* count;
  int4* items;
};

// Ingest (ring-sorted bf16 copy + ring sums) and the per-frame factors of Eq. 1.
xpcs_status raw_ingest(xpcs_ctx* ctx, const xpcs_rings* R, const void* X, xpcs_dtype dtype, int64_t T, int T_pad,
                       int nT, bool want_xp, long long* S, RawBuffers& b) {
  RawIngestParams ip{};
  ip.X = X;
  ip.dtype = dtype;
  ip.T = T;
  ip.M = R->M;
  ip.T_pad = T_pad;
  ip.Mp = R->Mp;
  ip.perm = R->d_perm;
  ip.pos_ring = R->d_pos_ring;
  ip.n_q = R->n_q;
  ip.Xp = want_xp ? b.Xp : nullptr;
  ip.S = S;
  ip.S2 = b.S2;
  ip.status = ctx->d_status;
  XPCS_LAUNCH(ctx, "ingest", 1, launch_raw_ingest(ip, ctx->stream));
  return XPCS_OK;
}

}  // namespace

extern "C" xpcs_status xpcs_ring_sums(xpcs_ctx* ctx, const xpcs_rings* R, const void* X, xpcs_dtype dtype,
                                      int64_t T, int64_t* S_out) {
  if (!ctx || !R || !X || !S_out || T <= 0 || R->ctx != ctx) return fail(ctx, XPCS_EINVAL, "bad ring_sums args");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  // ring sums only: the ingest kernel covers exactly T frames
  RawIngestParams ip{};
  ip.X = X;
  ip.dtype = dtype;
  ip.T = T;
  ip.M = R->M;
  ip.T_pad = (int)T;
  ip.Mp = R->Mp;
  ip.perm = R->d_perm;
  ip.pos_ring = R->d_pos_ring;
  ip.n_q = R->n_q;
  ip.Xp = nullptr;
  ip.S = reinterpret_cast<long long*>(S_out);
  ip.S2 = nullptr;
  ip.status = ctx->d_status;
  XPCS_LAUNCH(ctx, "ingest", 1, launch_raw_ingest(ip, ctx->stream));
  return finish(ctx);
}

namespace {

// Two-time configuration for a workload shape, (tiles per work item, schedule) with
// schedule 0 = single tiles (N = 128 MMAs), 1 = tile pairs (N = 256 MMAs): the autotuner's
// choice if there is one, else the given default.
std::pair<int, int> gram_tune_for(xpcs_ctx* ctx, uint64_t key, std::pair<int, int> dflt) {
  if (ctx->tune_forced) return ctx->tune_force;
  if (ctx->user_config.first > 0) return ctx->user_config;
  const auto it = ctx->gram_tune.find(key);
  if (it != ctx->gram_tune.end()) return it->second;
  return dflt;
}

// Shared tail of both two-time paths: the Gram launch, pair counts and g2.

xpcs_status run_twotime(xpcs_ctx* ctx, const CUtensorMap& tmL, const CUtensorMap& tmR, GramParams gp, int n_q,
                        int64_t T, int T_pad, int nT, int maxC, uint32_t* vbits, long long* count,
                        double* g2_out) {
  int4* d_items = nullptr;
  int n_items = 0;
  const bool grouped = gp.raw || gp.merge || !gp.C;
  XPCS_TRY(cached_items(ctx, n_q, nT, gp.CH, gp.pairs, grouped, &d_items, &n_items));
  gp.items = d_items;
  gp.n_items = n_items;
  const int grid = std::min<int>(gp.n_items, ctx->num_sms);
  XPCS_LAUNCH(ctx, "twotime_gram", 1, launch_gram(tmL, tmR, gp, grid, ctx->stream));
  if (count) {
    XPCS_LAUNCH(ctx, "pair_counts", 2, launch_counts(gp.r, n_q, T, T_pad, vbits, T_pad / 32, count, ctx->stream));
    if (g2_out)
      XPCS_LAUNCH(ctx, "g2_finalize", 1, launch_g2_finalize(gp.partials, count, n_q, T, nT, maxC, gp.CH, g2_out, ctx->stream));
  }
  return XPCS_OK;
}

}  // namespace

extern "C" xpcs_status xpcs_twotime_config(xpcs_ctx* ctx, int tiles, int schedule) {
  if (!ctx) return XPCS_EINVAL;
  if (tiles < 0 || tiles > 64 || schedule < 0 || schedule > 1)
    return fail(ctx, XPCS_EINVAL, "twotime_config: tiles must be 0..64 and schedule 0..1");
  ctx->user_config = {tiles, schedule};
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_twotime_raw(xpcs_ctx* ctx, const xpcs_rings* R, const void* X, xpcs_dtype dtype,
                                        int64_t T, float* C_out, int64_t* N_out, double* g2_out, int64_t* count_out) {
  return xpcs_twotime_raw_norm(ctx, R, X, dtype, T, XPCS_NORM_MEAN, C_out, N_out, g2_out, count_out);
}

extern "C" xpcs_status xpcs_twotime_raw_norm(xpcs_ctx* ctx, const xpcs_rings* R, const void* X, xpcs_dtype dtype,
                                             int64_t T, xpcs_norm norm, float* C_out, int64_t* N_out,
                                             double* g2_out, int64_t* count_out) {
  if (!ctx || !R || !X || T <= 0 || R->ctx != ctx || (dtype != XPCS_U8 && dtype != XPCS_U16) || (int)norm < 0 ||
      (int)norm > 2)
    return fail(ctx, XPCS_EINVAL, "bad twotime_raw args");
  if (T > (1 << 24)) return fail(ctx, XPCS_ENOTSUP, "T too large");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int n_q = R->n_q;
  const int nT = (int)((T + TILE - 1) / TILE);
  const int T_pad = nT * TILE;
  const std::pair<int, int> tune =
      gram_tune_for(ctx, gram_tune_key(n_q, nT, 1, 0, 1, C_out || N_out), gram_default_raw(n_q, nT));
  const int CH = tune.first;
  const int maxC = (nT + CH - 1) / CH;
  const bool want_g2 = g2_out != nullptr;
  const bool want_cnt = want_g2 || count_out;
  auto layout = [&](Carve& c, RawBuffers& b) {
    b.Xp = c.take<__nv_bfloat16>((size_t)T_pad * R->Mp);
    b.S = c.take<long long>((size_t)n_q * T);
    b.S2 = c.take<long long>((size_t)n_q * T);
    b.Sbar = norm == XPCS_NORM_EQ12 ? c.take<double>(n_q) : nullptr;
    b.r = c.take<float>((size_t)n_q * T_pad);
    b.blk_bad = c.take<uint32_t>((size_t)n_q * nT);
    b.partials = want_g2 ? c.take<float>((size_t)n_q * nT * maxC * DIAG_SLOTS) : nullptr;
    b.vbits = c.take<uint32_t>((size_t)n_q * (T_pad / 32) + n_q);  // + per-ring flags
    b.count = (want_cnt && !count_out) ? c.take<long long>((size_t)n_q * T) : nullptr;
  };
  RawBuffers b{};
  Carve c0;
  layout(c0, b);
  XPCS_TRY(ensure_scratch(ctx, c0.off));
  Carve c1{0, static_cast<char*>(ctx->scratch)};
  layout(c1, b);
  if (count_out) b.count = reinterpret_cast<long long*>(count_out);
  XPCS_TRY(raw_ingest(ctx, R, X, dtype, T, T_pad, nT, true, b.S, b));
  if (norm == XPCS_NORM_EQ12)
    XPCS_LAUNCH(ctx, "ring_mean", 1, launch_ring_mean(b.S, n_q, T, b.Sbar, ctx->stream));
  XPCS_LAUNCH(ctx, "raw_scales", 1,
              launch_raw_scales(b.S, b.S2, b.Sbar, (int)norm, R->d_Mq, n_q, T, T_pad, nT, b.r, b.blk_bad,
                                ctx->d_status, ctx->stream));
  const int pairs = tune.second == 1;
  CUtensorMap tm, tmR;
  XPCS_TRY(make_map(ctx, &tm, b.Xp, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, R->Mp, T_pad, KCH, TILE,
                    CU_TENSOR_MAP_SWIZZLE_128B));
  XPCS_TRY(make_map(ctx, &tmR, b.Xp, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, R->Mp, T_pad, KCH,
                    pairs ? 2 * TILE : TILE, CU_TENSOR_MAP_SWIZZLE_128B));
  GramParams gp{};
  gp.T = (int)T;
  gp.nT = nT;
  gp.T_pad = T_pad;
  gp.maxC = maxC;
  gp.CH = CH;
  gp.k_off = R->d_off;
  gp.k_chunks = R->d_chunks;
  gp.ring_rows = 0;
  gp.fmt = 1;
  gp.split = 0;
  gp.raw = 1;
  gp.pairs = pairs;
  gp.merge = 0;
  gp.r = b.r;
  gp.blk_bad = b.blk_bad;
  gp.C = C_out;
  gp.Nout = reinterpret_cast<long long*>(N_out);
  gp.partials = b.partials;
  gp.status = ctx->d_status;
  XPCS_TRY(run_twotime(ctx, tm, tmR, gp, n_q, T, T_pad, nT, maxC, b.vbits, want_cnt ? b.count : nullptr, g2_out));
  return finish(ctx);
}

// ====================================================================== basis

namespace {

xpcs_status basis_alloc(xpcs_ctx* ctx, const xpcs_rings* R, int k, xpcs_basis** out) {
  auto* B = new xpcs_basis();
  B->ctx = ctx;
  B->rings = R;
  B->n_q = R->n_q;
  B->M = R->M;
  B->k = k;
  B->kp = (k + 15) / 16 * 16;
  B->M_pad = (R->M + 63) / 64 * 64;
  const int n_q = R->n_q;
  const size_t szs[8] = {(size_t)R->M * k * 8, (size_t)n_q * k * k * 8, (size_t)n_q * k * 8,
                         (size_t)n_q * k * k * 4, (size_t)2 * B->kp * B->M_pad * 2, (size_t)n_q * 4,
                         (size_t)n_q * 4, (size_t)n_q * k * 8};
  void* p[8] = {};
  xpcs_status s = XPCS_OK;
  for (int i = 0; i < 8 && s == XPCS_OK; ++i) s = dev_alloc(ctx, &p[i], szs[i]);
  if (s != XPCS_OK) {
    for (int i = 0; i < 8; ++i) dev_free(ctx, p[i], szs[i]);
    delete B;
    return s;
  }
  B->d_koff = (int*)p[5];
  B->d_kch = (int*)p[6];
  B->d_s32 = (float2*)p[7];
  {
    const std::vector<int> koff(n_q, 0), kch(n_q, (k + KCH - 1) / KCH);
    cudaError_t e = cudaMemcpy(B->d_koff, koff.data(), szs[5], cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_kch, kch.data(), szs[6], cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      for (int i = 0; i < 8; ++i) dev_free(ctx, p[i], szs[i]);
      delete B;
      return fail(ctx, XPCS_ECUDA, std::string("basis metadata upload: ") + cudaGetErrorString(e));
    }
  }
  B->d_B = (double*)p[0];
  B->d_G = (double*)p[1];
  B->d_s = (double*)p[2];
  B->d_G32 = (float*)p[3];
  B->d_Bcat = (__half*)p[4];
  B->bytes = szs[0] + szs[1] + szs[2] + szs[3] + szs[4] + szs[5] + szs[6] + szs[7];
  *out = B;
  return XPCS_OK;
}

// Ring factors G_q = B_q^T B_q, s_q = B_q^T 1 (FP64) and the bf16 encode operand.
xpcs_status basis_finish(xpcs_ctx* ctx, xpcs_basis* B) {
  const xpcs_rings* R = B->rings;
  const int n_q = R->n_q, k = B->k;
  int64_t maxMq = 1;
  for (auto m : R->Mq) maxMq = std::max(maxMq, m);
  const int n_split = (int)std::max<int64_t>(1, std::min<int64_t>(16, maxMq / 4096));
  Carve c0;
  c0.take<double>((size_t)n_q * n_split * k * k);
  c0.take<double>((size_t)n_q * n_split * k);
  c0.take<double>(256);
  XPCS_TRY(ensure_scratch(ctx, c0.off));
  Carve c{0, static_cast<char*>(ctx->scratch)};
  double* Gpart = c.take<double>((size_t)n_q * n_split * k * k);
  double* spart = c.take<double>((size_t)n_q * n_split * k);
  XPCS_LAUNCH(ctx, "ring_factors", 1, launch_ring_factors2(B->d_B, k, R->d_perm, R->d_off, R->d_Mq, n_q, n_split, Gpart, spart,
                                      ctx->stream));
  XPCS_LAUNCH(ctx, "ring_factors_reduce", 1, launch_ring_factors_reduce(Gpart, spart, n_split, n_q, k, B->d_G, B->d_s, B->d_G32, B->d_s32,
                                                         ctx->stream));
  // power-of-two scale of the f16 encode operand: max|V| 2^s in [2^14, 2^15)
  double* mx = c.take<double>(256);
  XPCS_LAUNCH(ctx, "basis_absmax", 1, launch_basis_absmax(B->d_B, (long long)R->M * k, mx, ctx->stream));
  std::vector<double> hmx(256);
  XPCS_CUDA(ctx, cudaMemcpyAsync(hmx.data(), mx, 256 * 8, cudaMemcpyDeviceToHost, ctx->stream));
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const double amax = *std::max_element(hmx.begin(), hmx.end());
  B->enc_log2 = amax > 0 ? 14 - (int)std::floor(std::log2(amax)) : 0;
  XPCS_LAUNCH(ctx, "basis_pack", 1,
              launch_basis_pack(B->d_B, R->M, B->M_pad, k, B->kp, B->enc_log2, B->d_Bcat, ctx->stream));
  return XPCS_OK;
}

}  // namespace

extern "C" xpcs_status xpcs_basis_import(xpcs_ctx* ctx, const xpcs_rings* R, const double* B_host, int k,
                                         xpcs_basis** out) {
  if (!ctx || !R || !B_host || !out || k <= 0 || k > 256 || R->ctx != ctx)
    return fail(ctx, XPCS_EINVAL, "bad basis_import args");
  *out = nullptr;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  xpcs_basis* B = nullptr;
  XPCS_TRY(basis_alloc(ctx, R, k, &B));
  cudaError_t e = cudaMemcpy(B->d_B, B_host, (size_t)R->M * k * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    xpcs_basis_destroy(B);
    return fail(ctx, XPCS_ECUDA, std::string("basis upload: ") + cudaGetErrorString(e));
  }
  xpcs_status s = basis_finish(ctx, B);
  if (s == XPCS_OK) s = xpcs_synchronize(ctx);
  if (s != XPCS_OK) {
    xpcs_basis_destroy(B);
    return s;
  }
  *out = B;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_basis_export(xpcs_ctx* ctx, const xpcs_basis* B, double* B_host, double* G_host,
                                         double* s_host) {
  if (!ctx || !B || B->ctx != ctx) return fail(ctx, XPCS_EINVAL, "bad basis_export args");
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int n_q = B->rings->n_q, k = B->k;
  if (B_host) XPCS_CUDA(ctx, cudaMemcpy(B_host, B->d_B, (size_t)B->rings->M * k * 8, cudaMemcpyDeviceToHost));
  if (G_host) XPCS_CUDA(ctx, cudaMemcpy(G_host, B->d_G, (size_t)n_q * k * k * 8, cudaMemcpyDeviceToHost));
  if (s_host) XPCS_CUDA(ctx, cudaMemcpy(s_host, B->d_s, (size_t)n_q * k * 8, cudaMemcpyDeviceToHost));
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_basis_rank(const xpcs_basis* B, int* k) {
  if (!B || !k) return XPCS_EINVAL;
  *k = B->k;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_basis_destroy(xpcs_basis* B) {
  if (!B) return XPCS_EINVAL;
  xpcs_ctx* ctx = B->ctx;
  cudaStreamSynchronize(ctx->stream);
  const int n_q = B->n_q, k = B->k;
  dev_free(ctx, B->d_B, (size_t)B->M * k * 8);
  dev_free(ctx, B->d_G, (size_t)n_q * k * k * 8);
  dev_free(ctx, B->d_s, (size_t)n_q * k * 8);
  dev_free(ctx, B->d_G32, (size_t)n_q * k * k * 4);
  dev_free(ctx, B->d_Bcat, (size_t)2 * B->kp * B->M_pad * 2);
  dev_free(ctx, B->d_koff, (size_t)n_q * 4);
  dev_free(ctx, B->d_kch, (size_t)n_q * 4);
  dev_free(ctx, B->d_s32, (size_t)n_q * k * 8);
  if (B->d_B32) dev_free(ctx, B->d_B32, (size_t)B->M * k * 4);
  if (B->d_Gpair) {
    const int kq = (k + 63) / 64 * 64;
    dev_free(ctx, B->d_Gpair, (size_t)n_q * kq * 2 * kq * 2);
  }
  delete B;
  return XPCS_OK;
}


// ====================================================================== basis fit (Eq. 3-6)

extern "C" xpcs_status xpcs_fit_basis(xpcs_ctx* ctx, const xpcs_rings* R, const void* F, xpcs_dtype dtype,
                                      int64_t n_fit, int k, xpcs_basis** out, double* sigma_host) {
  if (!ctx || !R || !F || !out || R->ctx != ctx || n_fit < 1 || k < 1 || k > 256 || k > n_fit ||
      (dtype != XPCS_U8 && dtype != XPCS_U16))
    return fail(ctx, XPCS_EINVAL, "bad fit_basis args");
  if (n_fit > 32768) return fail(ctx, XPCS_ENOTSUP, "n_fit too large for the dense eigensolver");
  *out = nullptr;
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int n = (int)n_fit;
  const int64_t M = R->M;
  // 1. exact integer Gram F F^T of the fit frames over all pixels (one ring = every pixel)
  std::vector<int32_t> all(M, 0);
  xpcs_rings* P = nullptr;
  XPCS_TRY(rings_from_host(ctx, all.data(), M, 1, &P));
  struct Tmp {
    xpcs_ctx* ctx;
    std::vector<std::pair<void*, size_t>> v;
    ~Tmp() {
      for (auto& a : v) dev_free(ctx, a.first, a.second);
    }
    xpcs_status get(void** p, size_t b) {
      xpcs_status s = dev_alloc(ctx, p, b);
      if (s == XPCS_OK) v.push_back({*p, b});
      return s;
    }
  } tmp{ctx, {}};
  long long* N = nullptr;
  double *Gf = nullptr, *W = nullptr, *nrm = nullptr, *Z = nullptr, *work = nullptr;
  int* info = nullptr;
  xpcs_status s = tmp.get((void**)&N, (size_t)n * n * 8);
  if (s == XPCS_OK) s = tmp.get((void**)&Gf, (size_t)n * n * 8);
  if (s == XPCS_OK) s = tmp.get((void**)&W, (size_t)n * 8);
  if (s == XPCS_OK) s = tmp.get((void**)&nrm, (size_t)n * 8);
  if (s == XPCS_OK) s = tmp.get((void**)&Z, (size_t)n * k * 8);
  if (s == XPCS_OK) s = tmp.get((void**)&info, 4);
  if (s == XPCS_OK) s = xpcs_twotime_raw(ctx, P, F, dtype, n_fit, nullptr, reinterpret_cast<int64_t*>(N), nullptr,
                                         nullptr);
  xpcs_rings_destroy(P);
  XPCS_TRY(s);
  // 2. Gram of the Frobenius-normalised frames (Sec. 2.1)
  XPCS_LAUNCH(ctx, "fit_normalise", 1, launch_gram_normalise(N, n, Gf, nrm, ctx->stream));
  // 3. FP64 eigendecomposition (library call, setup only)
  if (!ctx->solver && cusolverDnCreate(&ctx->solver) != CUSOLVER_STATUS_SUCCESS)
    return fail(ctx, XPCS_ECUDA, "cusolverDnCreate failed");
  if (cusolverDnSetStream(ctx->solver, ctx->stream) != CUSOLVER_STATUS_SUCCESS)
    return fail(ctx, XPCS_ECUDA, "cusolverDnSetStream failed");
  int lwork = 0;
  if (cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Gf, n, W,
                                  &lwork) != CUSOLVER_STATUS_SUCCESS)
    return fail(ctx, XPCS_ECUDA, "cusolverDnDsyevd_bufferSize failed");
  XPCS_TRY(tmp.get((void**)&work, (size_t)std::max(1, lwork) * 8));
  if (cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Gf, n, W, work, lwork,
                       info) != CUSOLVER_STATUS_SUCCESS)
    return fail(ctx, XPCS_ECUDA, "cusolverDnDsyevd failed");
  std::vector<double> lam(n);
  int hinfo = 0;
  XPCS_CUDA(ctx, cudaMemcpyAsync(lam.data(), W, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  XPCS_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, 4, cudaMemcpyDeviceToHost, ctx->stream));
  XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hinfo != 0) return fail(ctx, XPCS_ECUDA, "eigensolver did not converge: info " + std::to_string(hinfo));
  // 4. rank and singular values (eigenvalues ascending from the solver)
  const double lmax = std::max(lam[n - 1], 0.0);
  const double tol = (double)n * 2.220446049250313e-16 * lmax;
  int rank = 0;
  for (int i = 0; i < n; ++i) rank += lam[i] > tol;
  if (sigma_host)
    for (int i = 0; i < n; ++i) sigma_host[i] = std::sqrt(std::max(lam[n - 1 - i], 0.0));
  if (k > rank) return fail(ctx, XPCS_EINVAL, "k=" + std::to_string(k) + " exceeds the rank " + std::to_string(rank));
  // 5. V_K = F^T U_k Sigma_k^-1 with the row norms folded in, sign convention, ring factors
  XPCS_LAUNCH(ctx, "fit_z", 1, launch_basis_z(Gf, W, nrm, n, k, Z, ctx->stream));
  xpcs_basis* B = nullptr;
  XPCS_TRY(basis_alloc(ctx, R, k, &B));
  xpcs_status st = XPCS_OK;
  if (launch_basis_build(F, dtype, n, M, Z, k, B->d_B, ctx->stream) != cudaSuccess ||
      launch_basis_sign(B->d_B, M, k, ctx->stream) != cudaSuccess)
    st = fail(ctx, XPCS_ECUDA, "basis build launch failed");
  ctx->launches += 2;
  if (st == XPCS_OK) st = basis_finish(ctx, B);
  if (st == XPCS_OK) st = xpcs_synchronize(ctx);
  if (st != XPCS_OK) {
    xpcs_basis_destroy(B);
    return st;
  }
  *out = B;
  return XPCS_OK;
}

extern "C" int xpcs_rank_from_spectrum(const double* sigma, int n, double factor) {
  if (!sigma || n <= 0 || !(factor > 0.0)) return -1;
  for (int i = 1; i < n; ++i)
    if (!(sigma[i] <= sigma[i - 1])) return -1;  // descending (NaN fails too)
  const double smax = std::max(sigma[0], 0.0);
  const double tol = (double)n * 2.220446049250313e-16 * smax * smax;
  int rank = 0;
  while (rank < n && sigma[rank] * sigma[rank] > tol && sigma[rank] > 0.0) ++rank;
  if (rank == 0) return 0;
  const double cut = factor * sigma[rank - 1];
  int K = 0;
  while (K < rank && sigma[K] >= cut) ++K;
  return K;
}

// ====================================================================== compressed path

extern "C" xpcs_status xpcs_twotime(xpcs_ctx* ctx, const xpcs_basis* B, const float* A, int64_t T,
                                    xpcs_precision prec, float* C_out, double* g2_out, int64_t* count_out) {
  const xpcs_options o{(int)prec, XPCS_NORM_MEAN, XPCS_QMEAN_COMPRESSED};
  return xpcs_twotime_opts(ctx, B, A, T, &o, nullptr, C_out, g2_out, count_out);
}

extern "C" xpcs_status xpcs_twotime_norm(xpcs_ctx* ctx, const xpcs_basis* B, const float* A, int64_t T,
                                         xpcs_precision prec, xpcs_norm norm, float* C_out, double* g2_out,
                                         int64_t* count_out) {
  const xpcs_options o{(int)prec, (int)norm, XPCS_QMEAN_COMPRESSED};
  return xpcs_twotime_opts(ctx, B, A, T, &o, nullptr, C_out, g2_out, count_out);
}

extern "C" xpcs_status xpcs_twotime_opts(xpcs_ctx* ctx, const xpcs_basis* B, const float* A, int64_t T,
                                         const xpcs_options* opt, const int64_t* S_raw, float* C_out,
                                         double* g2_out, int64_t* count_out) {
  const xpcs_options o = opt ? *opt : xpcs_options{0, 0, 0};
  const xpcs_precision prec = (xpcs_precision)o.precision;
  const xpcs_norm norm = (xpcs_norm)o.norm;
  if (!ctx || !B || !A || T <= 0 || B->ctx != ctx || (int)prec < 0 || (int)prec > 2 || (int)norm < 0 ||
      (int)norm > 2 || o.qmean < 0 || o.qmean > 1)
    return fail(ctx, XPCS_EINVAL, "bad twotime args");
  const bool exact = o.qmean == XPCS_QMEAN_EXACT_RAW;
  if (exact && (!S_raw || norm == XPCS_NORM_FROB))
    return fail(ctx, XPCS_EINVAL, "qmean EXACT_RAW needs the raw ring sums S_raw and a ring-sum normalisation");
  const long long* S_exact = exact ? reinterpret_cast<const long long*>(S_raw) : nullptr;
  if (T > (1 << 24)) return fail(ctx, XPCS_ENOTSUP, "T too large");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int n_q = B->rings->n_q, k = B->k;
  const int nT = (int)((T + TILE - 1) / TILE);
  const int T_pad = nT * TILE;
  const bool split = prec == XPCS_PREC_BF16X3;
  const bool merge = C_out == nullptr && g2_out != nullptr;  // g2 only: one diagonal pass per item
  const std::pair<int, int> tune =
      gram_tune_for(ctx, gram_tune_key(n_q, nT, prec == XPCS_PREC_FP16 ? 0 : 1, split ? 1 : 0, 0, C_out != nullptr),
                    gram_default_compressed(merge));
  const int CH = tune.first;
  const int maxC = (nT + CH - 1) / CH;
  const int nkp = (k + KCH - 1) / KCH;           // 64-wide chunks per operand piece
  const int Kc = (split ? 2 : 1) * nkp * KCH;
  const bool want_g2 = g2_out != nullptr;
  const bool want_cnt = want_g2 || count_out;
  // the left operand on the tensor cores when k <= 128 and the scale does not need W
  // (Eq. 1 and Eq. 12): the CUDA-core pass forms the ring sums, scales and R rows, then A
  // pieces + G pieces give L; else the CUDA-core kernel forms L as well
  const int kq = (k + 63) / 64 * 64;
  const bool use_tc = norm != XPCS_NORM_FROB && kq <= 128;
  if (use_tc && !B->d_Gpair) {
    if (ctx->capturing)
      return fail(ctx, XPCS_EBUSY, "run the two-time call once before capturing it (basis pieces are made on first use)");
    xpcs_basis* Bm = const_cast<xpcs_basis*>(B);
    void* p = nullptr;
    const size_t gb = (size_t)n_q * kq * 2 * kq * 2;
    XPCS_TRY(dev_alloc(ctx, &p, gb));
    Bm->d_Gpair = static_cast<__nv_bfloat16*>(p);
    Bm->bytes += gb;
    XPCS_LAUNCH(ctx, "gram_pieces", 1, launch_gram_pieces(B->d_G, n_q, k, kq, Bm->d_Gpair, ctx->stream));
  }
  struct Bufs {
    uint16_t *L, *R;
    __nv_bfloat16* Apair;
    double* Sbar;
    float* r;
    uint32_t* blk_bad;
    float* partials;
    uint32_t* vbits;
    long long* count;
  } b{};
  auto layout = [&](Carve& c) {
    b.L = c.take<uint16_t>((size_t)n_q * T_pad * Kc);
    b.R = c.take<uint16_t>((size_t)n_q * T_pad * Kc);
    b.Apair = use_tc ? c.take<__nv_bfloat16>((size_t)T_pad * 2 * kq) : nullptr;
    b.Sbar = norm == XPCS_NORM_EQ12 ? c.take<double>(n_q) : nullptr;
    b.r = c.take<float>((size_t)n_q * T_pad);
    b.blk_bad = c.take<uint32_t>((size_t)n_q * nT);
    b.partials = want_g2 ? c.take<float>((size_t)n_q * nT * maxC * DIAG_SLOTS) : nullptr;
    b.vbits = c.take<uint32_t>((size_t)n_q * (T_pad / 32) + n_q);  // + per-ring flags
    b.count = (want_cnt && !count_out) ? c.take<long long>((size_t)n_q * T) : nullptr;
  };
  Carve c0;
  layout(c0);
  XPCS_TRY(ensure_scratch(ctx, c0.off));
  Carve c1{0, static_cast<char*>(ctx->scratch)};
  layout(c1);
  if (count_out) b.count = reinterpret_cast<long long*>(count_out);
  PrepParams pp{};
  pp.A = A;
  pp.T = T;
  pp.k = k;
  pp.n_q = n_q;
  pp.T_pad = T_pad;
  pp.nT = nT;
  pp.G32 = B->d_G32;
  pp.s64 = B->d_s;
  pp.s32 = B->d_s32;
  pp.Mq = B->rings->d_Mq;
  pp.prec = prec;
  pp.Kc = Kc;
  pp.L = b.L;
  pp.R = b.R;
  pp.r = b.r;
  pp.blk_bad = b.blk_bad;
  pp.St = nullptr;
  pp.norm = (int)norm;
  pp.Sbar = b.Sbar;
  pp.S_exact = S_exact;
  pp.skip_L = use_tc ? 1 : 0;
  if (norm == XPCS_NORM_EQ12) {
    if (S_exact)  // mean of the exact ring sums
      XPCS_LAUNCH(ctx, "ring_mean", 1, launch_ring_mean(S_exact, n_q, T, b.Sbar, ctx->stream));
    else
      XPCS_LAUNCH(ctx, "coef_mean", 1, launch_coef_mean(A, T, k, B->d_s, n_q, b.Sbar, ctx->stream));
  }
  XPCS_LAUNCH(ctx, "compressed_prep", 1, launch_prep_compressed(pp, ctx->stream));
  if (use_tc) {
    XPCS_LAUNCH(ctx, "coef_pieces", 1, launch_coef_pieces(A, T, k, kq, T_pad, b.Apair, ctx->stream));
    CUtensorMap tmA, tmG;
    XPCS_TRY(make_map(ctx, &tmA, b.Apair, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2 * kq, T_pad, 64, TILE,
                      CU_TENSOR_MAP_SWIZZLE_128B));
    XPCS_TRY(make_map(ctx, &tmG, B->d_Gpair, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2 * kq, (uint64_t)n_q * kq, 64,
                      kq, CU_TENSOR_MAP_SWIZZLE_128B));
    CompTcParams cp{};
    cp.r = b.r;
    cp.L = b.L;
    cp.T_pad = T_pad;
    cp.Kc = Kc;
    cp.kq = kq;
    cp.status = ctx->d_status;
    XPCS_LAUNCH(ctx, "ring_w_tc", 1, launch_ring_w_tc(tmA, tmG, cp, n_q, nT, (int)prec, ctx->stream));
  }
  const CUtensorMapDataType dt =
      prec == XPCS_PREC_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const int pairs = tune.second == 1;
  CUtensorMap tmL, tmR;
  XPCS_TRY(make_map(ctx, &tmL, b.L, dt, 2, Kc, (uint64_t)n_q * T_pad, KCH, TILE, CU_TENSOR_MAP_SWIZZLE_128B));
  XPCS_TRY(make_map(ctx, &tmR, b.R, dt, 2, Kc, (uint64_t)n_q * T_pad, KCH, pairs ? 2 * TILE : TILE,
                    CU_TENSOR_MAP_SWIZZLE_128B));
  GramParams gp{};
  gp.T = (int)T;
  gp.nT = nT;
  gp.T_pad = T_pad;
  gp.maxC = maxC;
  gp.CH = CH;
  gp.k_off = B->d_koff;
  gp.k_chunks = B->d_kch;
  gp.ring_rows = T_pad;
  gp.fmt = prec == XPCS_PREC_FP16 ? 0 : 1;
  gp.split = split ? 1 : 0;
  gp.raw = 0;
  gp.pairs = pairs;
  gp.merge = merge ? 1 : 0;
  gp.rmerge = (C_out && want_g2 && !merge && !pairs) ? 1 : 0;
  gp.r = b.r;
  gp.blk_bad = b.blk_bad;
  gp.C = C_out;
  gp.Nout = nullptr;
  gp.partials = b.partials;
  gp.status = ctx->d_status;
  XPCS_TRY(run_twotime(ctx, tmL, tmR, gp, n_q, T, T_pad, nT, maxC, b.vbits, want_cnt ? b.count : nullptr, g2_out));
  return finish(ctx);
}

// ====================================================================== g2 over stored C

extern "C" xpcs_status xpcs_g2(xpcs_ctx* ctx, const float* C, int n_q, int64_t T, double* g2_out,
                               int64_t* count_out) {
  if (!ctx || !C || !g2_out || n_q <= 0 || T <= 0) return fail(ctx, XPCS_EINVAL, "bad g2 args");
  if (n_q > XPCS_G2_MAX_RINGS)
    return fail(ctx, XPCS_ERANGE,
                "xpcs_g2: n_q = " + std::to_string(n_q) + " rings exceeds the limit of " +
                    std::to_string(XPCS_G2_MAX_RINGS));
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int splits = g2_from_C_splits(T, n_q, ctx->num_sms);
  Carve c0;
  c0.take<double>((size_t)splits * n_q * T);
  c0.take<long long>((size_t)splits * n_q * T);
  XPCS_TRY(ensure_scratch(ctx, c0.off));
  Carve c{0, static_cast<char*>(ctx->scratch)};
  double* part = c.take<double>((size_t)splits * n_q * T);
  long long* cpart = c.take<long long>((size_t)splits * n_q * T);
  XPCS_LAUNCH(ctx, "g2_from_C", 1, launch_g2_from_C(C, n_q, T, part, splits, cpart, ctx->stream));
  XPCS_LAUNCH(ctx, "g2_from_C_reduce", 1, launch_g2_from_C_reduce(part, cpart, n_q, T, splits, g2_out,
                                         reinterpret_cast<long long*>(count_out), ctx->stream));
  return finish(ctx);
}
