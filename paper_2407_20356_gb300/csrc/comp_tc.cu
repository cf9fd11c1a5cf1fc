// Compressed-path left operand on the tcgen05 tensor cores (sm_103a):
//     L_q(t) = r_q(t) * (a_t G_q),   a 128-frame tile of one ring per CTA.
//
// W = A G_q is a (128 x kq) x (kq x kq) product per tile (kq = k rounded up to 64, at most
// 128), done as three bf16 products of hi/lo pieces, A_hi G_hi + A_lo G_hi + A_hi G_lo,
// accumulated in f32 in TMEM (the dropped A_lo G_lo term is about 2^-16 of each product,
// below the rounding of the bf16 operand rows this kernel writes).  Thread 0 issues the
// TMA loads of the A tile (hi and lo pieces, 64-column chunks with the 128-byte swizzle)
// and of G_q (hi and lo, N = kq rows), then the MMAs; the four warps then read their TMEM
// lane quarter (thread = frame), scale by r_q(t) and write the row in the operand format
// of the two-time kernel: [hi | lo] bf16 pieces for the split format, else one 16-bit
// piece.  r_q(t), the ring sums and the R rows come from the CUDA-core operand pass run
// just before (r = 0 for undefined and padding frames, so those rows are zero).  Folding
// that pass in here (one thread per frame for the compensated ring sum) measured slower:
// the serial dot product of each frame is latency-bound at this occupancy.  Every
// mbarrier wait is bounded; on expiry the kernel records XPCS_DEV_TIMEOUT, waits
// (bounded) for its copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace xpcs {

namespace {

constexpr int CT_THREADS = 128;
constexpr int CT_ROWS = 128;
constexpr int CT_CHUNK = CT_ROWS * 64 * 2;  // 16 KB: one 64-column bf16 chunk of the A tile

template <typename T16>
XPCS_DEV T16 cvt16(float x);
template <>
XPCS_DEV __half cvt16<__half>(float x) { return __float2half_rn(x); }
template <>
XPCS_DEV __nv_bfloat16 cvt16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename T16, bool SPLIT>
__global__ void __launch_bounds__(CT_THREADS) ring_w_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                               const __grid_constant__ CUtensorMap tmG,
                                                               const CompTcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kq = p.kq, nkc = kq / 64;
  const int gch = kq * 128;  // bytes of one 64-column chunk of G (kq rows x 128 B)
  uint8_t* a_hi = smem;
  uint8_t* a_lo = a_hi + nkc * CT_CHUNK;
  uint8_t* g_hi = a_lo + nkc * CT_CHUNK;
  uint8_t* g_lo = g_hi + nkc * gch;
  uint64_t* bars = reinterpret_cast<uint64_t*>(g_lo + nkc * gch);
  uint64_t* full = bars;
  uint64_t* done = bars + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  volatile int* flag = reinterpret_cast<volatile int*>(tmem_slot + 1);  // 1: MMAs issued, -1: abort

  const int tile = blockIdx.x, q = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(done, 1);
    mbar_fence_init();
    *flag = 0;
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, (uint32_t)kq);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmG);
    mbar_arrive_expect_tx(full, (uint32_t)(nkc * (2 * CT_CHUNK + 2 * gch)));
    for (int c = 0; c < nkc; ++c) {
      tma_load_2d(a_hi + c * CT_CHUNK, &tmA, full, 64 * c, tile * CT_ROWS);
      tma_load_2d(a_lo + c * CT_CHUNK, &tmA, full, kq + 64 * c, tile * CT_ROWS);
      tma_load_2d(g_hi + c * gch, &tmG, full, 64 * c, q * kq);
      tma_load_2d(g_lo + c * gch, &tmG, full, kq + 64 * c, q * kq);
    }
    if (mbar_wait(full, 0, p.status)) {
      tc_fence_after();
      const uint32_t idesc = idesc_f16(1, CT_ROWS, kq);
      for (int c = 0; c < nkc; ++c) {
        const uint64_t ah = smem_desc_sw128(a_hi + c * CT_CHUNK), al = smem_desc_sw128(a_lo + c * CT_CHUNK);
        const uint64_t gh = smem_desc_sw128(g_hi + c * gch), gl = smem_desc_sw128(g_lo + c * gch);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {  // 16 elements = 32 B per MMA
          tc_mma_f16(tmem, ah + 2 * kk, gh + 2 * kk, idesc, (c > 0 || kk > 0) ? 1u : 0u);
          tc_mma_f16(tmem, al + 2 * kk, gh + 2 * kk, idesc, 1u);
          tc_mma_f16(tmem, ah + 2 * kk, gl + 2 * kk, idesc, 1u);
        }
      }
      tc_commit(done);
      *flag = 1;
    } else {
      *flag = -1;
      mbar_wait(full, 0, p.status);  // never leave with bulk copies in flight
    }
  }
  __syncthreads();
  const long long t = (long long)tile * CT_ROWS + warp * 32 + lane;
  const bool ok = *flag == 1 && mbar_wait_warp(done, 0, p.status);
  if (ok) {
    tc_fence_after();
    const float rv = p.r[(size_t)q * p.T_pad + t];
    T16* row = static_cast<T16*>(p.L) + ((size_t)q * p.T_pad + t) * p.Kc;
    for (int c32 = 0; c32 < kq / 32; ++c32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32 * c32, v);
      tc_wait_ld();
      alignas(16) T16 hi[32];
      alignas(16) T16 lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float x = rv * __uint_as_float(v[j]);
        hi[j] = cvt16<T16>(x);
        if (SPLIT) lo[j] = cvt16<T16>(x - (float)hi[j]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) reinterpret_cast<uint4*>(row + 32 * c32)[u] = reinterpret_cast<const uint4*>(hi)[u];
      if (SPLIT) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          reinterpret_cast<uint4*>(row + kq + 32 * c32)[u] = reinterpret_cast<const uint4*>(lo)[u];
      }
    }
  } else if (threadIdx.x == 0 && *flag == 1) {
    mbar_wait(done, 0, p.status);  // MMAs complete before TMEM is released
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)kq);
  }
}

}  // namespace

int comp_tc_smem(int kq) { return 1024 + (kq / 64) * (2 * CT_CHUNK + 2 * kq * 128) + 64; }

cudaError_t launch_ring_w_tc(const CUtensorMap& tmA, const CUtensorMap& tmG, const CompTcParams& p, int n_q,
                             int n_tiles, int prec, cudaStream_t st) {
  const int smem = comp_tc_smem(p.kq);
  const dim3 grid(n_tiles, n_q);
#define XPCS_CT_LAUNCH(T16, SPLIT)                                                                         \
  do {                                                                                                     \
    static int attr = 0;                                                                                   \
    if (smem > attr) {                                                                                     \
      cudaError_t e = cudaFuncSetAttribute(ring_w_tc_kernel<T16, SPLIT>,                                   \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);             \
      if (e != cudaSuccess) return e;                                                                      \
      attr = smem;                                                                                         \
    }                                                                                                      \
    ring_w_tc_kernel<T16, SPLIT><<<grid, CT_THREADS, smem, st>>>(tmA, tmG, p);                             \
  } while (0)
  if (prec == XPCS_PREC_FP16)
    XPCS_CT_LAUNCH(__half, false);
  else if (prec == XPCS_PREC_BF16)
    XPCS_CT_LAUNCH(__nv_bfloat16, false);
  else
    XPCS_CT_LAUNCH(__nv_bfloat16, true);
#undef XPCS_CT_LAUNCH
  return cudaGetLastError();
}

}  // namespace xpcs
