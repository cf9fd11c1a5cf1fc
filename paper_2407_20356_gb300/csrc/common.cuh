// Shared device helpers for the sm_103a kernels: mbarriers, TMA, tcgen05 (TMEM + MMA).
//
// All waits are bounded: a wait that does not complete within its limit (nanoseconds of
// %globaltimer) records an error code in the kernel's status word and returns false, and
// the caller unwinds (frees its TMEM and exits) instead of spinning forever.  The limit is
// the context's (or stream's) setting, a u64 stored 8 bytes after the status word; 0
// there, or no status word, means XPCS_WAIT_NS.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "internal.h"

#define XPCS_DEV __device__ __forceinline__

namespace xpcs {

#ifndef XPCS_WAIT_NS
#define XPCS_WAIT_NS 2000000000ull  // 2 s
#endif

XPCS_DEV uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

XPCS_DEV uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

XPCS_DEV void set_status(uint32_t* status, uint32_t code) {
  if (status) atomicCAS(status, 0u, code);
}

// ------------------------------------------------------------------ mbarrier

XPCS_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

XPCS_DEV void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

XPCS_DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

XPCS_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

XPCS_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded-wait limit of the kernel whose status word is `status` (see above).
XPCS_DEV uint64_t wait_limit_ns(const uint32_t* status) {
  if (status) {
    const uint64_t v = *reinterpret_cast<const volatile uint64_t*>(status + 2);
    if (v) return v;
  }
  return XPCS_WAIT_NS;
}

// Wait until the phase with the given parity has completed, within the kernel's limit.
// The first poll is inline; the rest of the wait is one out-of-line function, which keeps
// the code at each of the many wait sites of a kernel small (inlined everywhere, the waits
// made the two-time kernel 8 % slower).  Every limit is at least 1 ms, so the limit word
// (device or host-mapped memory) is read only once a wait has already lasted that long.
static __device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, uint32_t* status) {
  const uint64_t t0 = globaltimer();
  uint64_t limit = 1000000ull;  // 1 ms, until the real limit is read
  bool have_limit = false;
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    const uint64_t dt = globaltimer() - t0;
    if (dt > limit && !have_limit) {
      limit = wait_limit_ns(status);
      have_limit = true;
    }
    if (dt > limit) {
      set_status(status, XPCS_DEV_TIMEOUT);
      return false;
    }
  }
}

XPCS_DEV bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* status) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_slow(bar, parity, status);
}

// Warp-wide bounded wait: lane 0 polls, the warp then agrees on the outcome.  The
// __syncwarp orders the other lanes after lane 0's acquire of the phase.
XPCS_DEV bool mbar_wait_warp(uint64_t* bar, uint32_t parity, uint32_t* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, status);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  __syncwarp();
  return ok;
}

// ------------------------------------------------------------------ dependent launches
// A kernel launched with programmatic stream serialization may start before the kernel
// ahead of it in the stream has finished: pdl_wait blocks the calling thread until that
// kernel has completed and its memory operations are visible (at once when the launch was
// an ordinary one), and pdl_trigger lets the kernel behind this one start launching.
// Every kernel of such a chain waits before it ends, so completion stays transitive.
XPCS_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
XPCS_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------------ TMA (no multicast)

XPCS_DEV void tma_prefetch_desc(const void* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

XPCS_DEV void tma_load_2d(void* smem_dst, const void* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(smem_dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Tiled store of a shared-memory box to global memory (elements outside the tensor are
// not written), in the issuing thread's bulk group.
XPCS_DEV void tma_store_2d(const void* map, const void* smem_src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(smem_src)), "r"(x), "r"(y)
               : "memory");
}
XPCS_DEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the sources of this thread's bulk stores have been read (shared memory reusable)
XPCS_DEV void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
XPCS_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ------------------------------------------------------------------ tcgen05

XPCS_DEV void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
               "r"(ncols)
               : "memory");
}
XPCS_DEV void tmem_relinquish() {  // whole warp
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
XPCS_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
XPCS_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
XPCS_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (f16 or bf16 operands, f32 accumulator). One thread.
XPCS_DEV void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on an mbarrier when all previously issued MMAs of this thread have completed.
XPCS_DEV void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

XPCS_DEV void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 32 consecutive 32-bit columns: thread l of the warp gets row (lane base + l).
XPCS_DEV void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns from registers (thread = lane); asynchronous
// until tc_wait_st.
XPCS_DEV void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
      :
      : "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
XPCS_DEV void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 32 lanes x 4 consecutive 32-bit columns.
XPCS_DEV void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
}

// Running sum held as an f32 pair (hi, lo), value hi + lo: add x with Knuth's TwoSum
// (s + e = hi + x exactly, no precondition on magnitudes), fold e into lo, then
// renormalise with a second TwoSum so that |lo| <= ulp(hi) / 2.  Each addition loses only
// the rounding of lo (about 2^-48 of the sum), with f32 operations only.
XPCS_DEV float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
XPCS_DEV float2 f32pair_add(float2 acc, float x) {
  const float2 t = two_sum(acc.x, x);
  return two_sum(t.x, __fadd_rn(acc.y, t.y));
}

// Shared-memory matrix descriptor for a K-major operand tile stored with the 128-byte
// swizzle: rows of 128 bytes, 8-row core groups 1024 bytes apart (tile base 1024-aligned).
XPCS_DEV uint64_t smem_desc_sw128(const void* tile) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;         // start address
  d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;               // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;               // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16, f32 accumulate, both operands K-major.
// fmt: 0 = f16, 1 = bf16 (A and B always share the type).
__host__ __device__ constexpr uint32_t idesc_f16(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

XPCS_DEV void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also returns, to every participating thread, the OR of `pred`.
XPCS_DEV bool named_bar_sync_or(int id, int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

XPCS_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Two float32 additions in one instruction (round to nearest, each lane of the pair exact
// as a scalar add.rn.f32).
XPCS_DEV unsigned long long add_f32x2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

XPCS_DEV float2 u64_as_float2(unsigned long long x) {
  return make_float2(__uint_as_float((uint32_t)x), __uint_as_float((uint32_t)(x >> 32)));
}

// Sum of one row (32 floats, 16-byte aligned, row pitch LD floats) of a skewed buffer
// whose entries lie in columns [lo, hi); the 16-byte groups outside that range hold zeros
// and are not read (lanes that skip a group issue no shared-memory traffic for it).
template <int LD>
XPCS_DEV float skew_row_sum(const float* Q, int row, int lo, int hi) {
  const ulonglong2* v = reinterpret_cast<const ulonglong2*>(Q + row * LD);
  ulonglong2 s = make_ulonglong2(0ull, 0ull);
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    if (4 * m + 3 >= lo && 4 * m < hi) {
      const ulonglong2 x = v[m];
      s.x = add_f32x2(s.x, x.x);
      s.y = add_f32x2(s.y, x.y);
    }
  }
  const float2 a = u64_as_float2(s.x), b = u64_as_float2(s.y);
  return (a.x + a.y) + (b.x + b.y);
}

// ------------------------------------------------------------------ stream pair counts
// Bits [slot, slot + n) (n <= 64) of one ring's validity words (slots past the ring's end
// are its mirror, so no wrap is needed for slot < cap).
XPCS_DEV unsigned long long vbits_window(const unsigned long long* vb, long long slot, int n) {
  const int sh = (int)(slot & 63);
  const unsigned long long lo = vb[slot >> 6] >> sh;
  const unsigned long long hi = sh ? vb[(slot >> 6) + 1] << (64 - sh) : 0ull;
  const unsigned long long v = lo | hi;
  return n >= 64 ? v : v & ((1ull << n) - 1ull);
}

// Defined pairs (t0 + f, t0 + f - tau) of one ring over the frames f of `mask` (bit f:
// frame t0 + f, f < 64) whose partner exists (t0 + f - tau >= 0): both validity bits set.
XPCS_DEV long long masked_pair_count(const unsigned long long* vb, long long cap, long long t0,
                                     unsigned long long mask, long long tau) {
  const long long f0 = tau > t0 ? tau - t0 : 0;  // first frame with a partner
  if (f0 >= 64) return 0;
  const unsigned long long m = mask >> f0;
  if (!m) return 0;
  const int n = 64 - (int)f0;
  const unsigned long long a = vbits_window(vb, (t0 + f0) % cap, n) & m;
  const unsigned long long h = vbits_window(vb, (t0 + f0 - tau) % cap, n);
  return __popcll(a & h);
}

}  // namespace xpcs
