// Serving layer: several online streams on one GPU, fed by one scheduler thread.
//
// Clients submit frames (host frames are copied into per-stream host queues; device frames
// are queued by pointer and read in place) and return at once.  The
// scheduler loops over the admitted streams; for each one with queued frames whose
// staging buffer is free it takes every frame that has arrived, up to the stream's batch
// limit (continuous batching: a batch grows while the previous one is on the device), and
// enqueues it on that stream's own CUDA stream, so the streams' work overlaps on the GPU.
// Streams are admitted against the context's device-memory budget; an open may wait for
// memory that other streams release when they close.  Each stream's results depend only
// on its own frames, so they are the same alone and in a mix (up to the f32 rounding of
// the per-batch partial sums, which depends on how frames were batched).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "handles.h"
#include "internal.h"

using namespace xpcs;

struct xpcs_server {
  struct Chunk {
    std::vector<char> data;        // host frames (copied at submit)
    const char* dev = nullptr;     // or frames in device memory, read in place
    std::vector<int64_t> arrive;
    int64_t n = 0, off = 0;  // frames in the chunk, frames already taken
  };
  struct Slot {
    xpcs_stream* s = nullptr;
    std::deque<Chunk> q;
    int64_t queued = 0;
    uint64_t submitted = 0;
    uint64_t pushed = 0;
    bool closing = false;
    std::mutex mu;  // serialises device calls on this stream
    std::vector<char> gather;
    std::vector<int64_t> gather_arrive;
  };
  xpcs_ctx* ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_mem;
  std::vector<Slot*> slots;
  std::thread worker;
  bool stop = false;
  xpcs_status worker_status = XPCS_OK;
  uint64_t batches = 0;
};

namespace {

size_t frame_bytes(const xpcs_stream* s) {
  return (size_t)s->basis->rings->M * (s->dtype == XPCS_U8 ? 1 : 2);
}

xpcs_server::Slot* find_slot(xpcs_server* sv, const xpcs_stream* s) {
  for (auto* sl : sv->slots)
    if (sl->s == s) return sl;
  return nullptr;
}

void worker_loop(xpcs_server* sv) {
  cudaSetDevice(sv->ctx->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  size_t rr = 0;
  while (!sv->stop) {
    bool did = false;
    const size_t ns = sv->slots.size();
    for (size_t u = 0; u < ns && !sv->stop; ++u) {
      xpcs_server::Slot* sl = sv->slots[(rr + u) % ns];
      if (sl->queued == 0) continue;
      xpcs_stream* s = sl->s;
      const size_t fb = frame_bytes(s);
      const xpcs_server::Chunk& c0 = sl->q.front();
      int64_t n = std::min<int64_t>(sl->queued, s->max_batch);
      xpcs_status st;
      if (c0.dev) {
        // continuous batching: while two batches of this stream are on the device, frames
        // keep queueing and the next batch grows (the host path gets the same back-pressure
        // from its staging buffers)
        {
          std::lock_guard<std::mutex> sg(sl->mu);
          if (stream_inflight(s) >= 2) continue;
        }
        // device frames: within one submitted block the batch is read in place; a batch
        // spanning blocks (continuous batching of small submissions) is gathered into the
        // stream's device staging buffer by copies on the stream's own CUDA stream, ordered
        // after its previous kernels
        struct Piece {
          const char* src;
          int64_t n;
        };
        std::vector<Piece> pieces;
        sl->gather_arrive.clear();
        int64_t got = 0;
        for (auto& c : sl->q) {
          if (!c.dev || got == n) break;
          const int64_t take = std::min(n - got, c.n - c.off);
          pieces.push_back({c.dev + c.off * fb, take});
          sl->gather_arrive.insert(sl->gather_arrive.end(), c.arrive.begin() + c.off, c.arrive.begin() + c.off + take);
          got += take;
        }
        n = got;
        std::lock_guard<std::mutex> sg(sl->mu);
        lk.unlock();
        if (pieces.size() == 1) {
          st = stream_push_device_stamped(s, pieces[0].src, n, sl->gather_arrive.data());
        } else {
          st = XPCS_OK;
          int64_t at = 0;
          for (const Piece& pc : pieces) {
            if (cudaMemcpyAsync(static_cast<char*>(s->d_frames) + at * fb, pc.src, pc.n * fb, cudaMemcpyDeviceToDevice,
                                s->stream) != cudaSuccess) {
              st = fail(s->ctx, XPCS_ECUDA, "server device gather failed");
              break;
            }
            at += pc.n;
          }
          if (st == XPCS_OK) st = stream_push_device_stamped(s, s->d_frames, n, sl->gather_arrive.data());
        }
        lk.lock();
      } else {
        // host frames: gather the first n queued host frames (up to the next device chunk)
        sl->gather.resize(n * fb);
        sl->gather_arrive.resize(n);
        int64_t got = 0;
        for (auto& c : sl->q) {
          if (c.dev) break;
          const int64_t take = std::min(n - got, c.n - c.off);
          memcpy(sl->gather.data() + got * fb, c.data.data() + c.off * fb, take * fb);
          std::copy(c.arrive.begin() + c.off, c.arrive.begin() + c.off + take, sl->gather_arrive.begin() + got);
          got += take;
          if (got == n) break;
        }
        n = got;
        std::lock_guard<std::mutex> sg(sl->mu);
        lk.unlock();
        st = stream_push_host(s, sl->gather.data(), n, sl->gather_arrive.data(), false);
        lk.lock();
      }
      if (ns != sv->slots.size() || std::find(sv->slots.begin(), sv->slots.end(), sl) == sv->slots.end())
        break;  // cannot happen while frames are queued (close waits for them); rescan anyway
      if (st == XPCS_EBUSY) continue;  // its previous copy is still in flight: keep queueing
      if (st != XPCS_OK) {
        sv->worker_status = st;
        sl->q.clear();
        sl->queued = 0;
        sv->cv_done.notify_all();
        continue;
      }
      // consume the frames from the queue
      int64_t left = n;
      while (left > 0) {
        auto& c = sl->q.front();
        const int64_t take = std::min(left, c.n - c.off);
        c.off += take;
        left -= take;
        if (c.off == c.n) sl->q.pop_front();
      }
      sl->queued -= n;
      sl->pushed += n;
      ++sv->batches;
      did = true;
      sv->cv_done.notify_all();
      rr = (rr + u + 1) % ns;
      break;  // the slot list may have changed while unlocked: rescan
    }
    if (!did) sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" xpcs_status xpcs_server_create(xpcs_ctx* ctx, xpcs_server** out) {
  if (!ctx || !out) return XPCS_EINVAL;
  auto* sv = new xpcs_server();
  sv->ctx = ctx;
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_server_open(xpcs_server* sv, const xpcs_basis* basis, int64_t history, int max_batch,
                                        xpcs_dtype dtype, int wait_ms, xpcs_stream** out) {
  if (!sv || !out) return XPCS_EINVAL;
  *out = nullptr;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, wait_ms));
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    xpcs_stream* s = nullptr;
    const xpcs_status st = xpcs_stream_open(sv->ctx, basis, history, max_batch, dtype, &s);
    if (st == XPCS_OK) {
      auto* sl = new xpcs_server::Slot();
      sl->s = s;
      sv->slots.push_back(sl);
      *out = s;
      return XPCS_OK;
    }
    if (st != XPCS_EBUSY) return st;
    if (sv->cv_mem.wait_until(lk, deadline) == std::cv_status::timeout) return XPCS_EBUSY;
  }
}

extern "C" xpcs_status xpcs_server_submit(xpcs_server* sv, xpcs_stream* s, const void* frames_host, int64_t n,
                                          uint64_t* ticket) {
  if (!sv || !s || !frames_host || n < 0) return XPCS_EINVAL;
  xpcs_server::Chunk c;
  const size_t fb = frame_bytes(s);
  c.data.resize(n * fb);
  memcpy(c.data.data(), frames_host, n * fb);
  c.arrive.assign(n, now_ns());
  c.n = n;
  std::lock_guard<std::mutex> lk(sv->mu);
  xpcs_server::Slot* sl = find_slot(sv, s);
  if (!sl || sl->closing) return XPCS_EINVAL;
  if (n) sl->q.push_back(std::move(c));
  sl->queued += n;
  sl->submitted += n;
  if (ticket) *ticket = sl->submitted;
  sv->cv_work.notify_one();
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_server_submit_device(xpcs_server* sv, xpcs_stream* s, const void* frames_dev, int64_t n,
                                                 uint64_t* ticket) {
  if (!sv || !s || !frames_dev || n < 0) return XPCS_EINVAL;
  xpcs_server::Chunk c;
  c.dev = static_cast<const char*>(frames_dev);
  c.arrive.assign(n, now_ns());
  c.n = n;
  std::lock_guard<std::mutex> lk(sv->mu);
  xpcs_server::Slot* sl = find_slot(sv, s);
  if (!sl || sl->closing) return XPCS_EINVAL;
  if (n) sl->q.push_back(std::move(c));
  sl->queued += n;
  sl->submitted += n;
  if (ticket) *ticket = sl->submitted;
  sv->cv_work.notify_one();
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_server_poll(xpcs_server* sv, xpcs_stream* s, uint64_t ticket, int timeout_ms) {
  if (!sv || !s) return XPCS_EINVAL;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  xpcs_server::Slot* sl = nullptr;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    sl = find_slot(sv, s);
    if (!sl) return XPCS_EINVAL;
    while (sl->pushed < ticket && sv->worker_status == XPCS_OK)
      if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return XPCS_EBUSY;
    if (sv->worker_status != XPCS_OK) return sv->worker_status;
  }
  const int left = (int)std::max<int64_t>(
      0, std::chrono::duration_cast<std::chrono::milliseconds>(deadline - std::chrono::steady_clock::now()).count());
  std::lock_guard<std::mutex> sg(sl->mu);
  return xpcs_stream_poll(s, ticket, left);
}

extern "C" xpcs_status xpcs_server_read_g2(xpcs_server* sv, xpcs_stream* s, double* g2_host, int64_t* count_host) {
  if (!sv || !s) return XPCS_EINVAL;
  xpcs_server::Slot* sl = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sl = find_slot(sv, s);
    if (!sl) return XPCS_EINVAL;
  }
  std::lock_guard<std::mutex> sg(sl->mu);
  return xpcs_stream_read_g2(s, g2_host, count_host);
}

extern "C" xpcs_status xpcs_server_latency(xpcs_server* sv, xpcs_stream* s, int reset, double* p50_us,
                                           double* p99_us, double* max_us, int64_t* n_frames) {
  if (!sv || !s) return XPCS_EINVAL;
  xpcs_server::Slot* sl = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sl = find_slot(sv, s);
    if (!sl) return XPCS_EINVAL;
  }
  std::lock_guard<std::mutex> sg(sl->mu);
  return xpcs_stream_latency(s, reset, p50_us, p99_us, max_us, n_frames);
}

extern "C" xpcs_status xpcs_server_close(xpcs_server* sv, xpcs_stream* s) {
  if (!sv || !s) return XPCS_EINVAL;
  xpcs_server::Slot* sl = nullptr;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    sl = find_slot(sv, s);
    if (!sl) return XPCS_EINVAL;
    sl->closing = true;
    // let the scheduler push what is queued (bounded: the work only needs the GPU)
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(60);
    while (sl->queued > 0 && sv->worker_status == XPCS_OK)
      if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
    sv->slots.erase(std::find(sv->slots.begin(), sv->slots.end(), sl));
    {
      std::lock_guard<std::mutex> sg(sl->mu);
      xpcs_stream_close(s);
    }
    delete sl;
  }
  sv->cv_mem.notify_all();  // memory released: waiting opens retry
  return XPCS_OK;
}

extern "C" uint64_t xpcs_server_batches(const xpcs_server* sv) { return sv ? sv->batches : 0; }

extern "C" xpcs_status xpcs_server_destroy(xpcs_server* sv) {
  if (!sv) return XPCS_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  sv->worker.join();
  for (auto* sl : sv->slots) {
    xpcs_stream_close(sl->s);
    delete sl;
  }
  delete sv;
  return XPCS_OK;
}
