// Encode: coefficients A = X V_K (Eq. 7) on the tcgen05 tensor cores, sm_103a.
//
// X (T x M counts, u8 or u16) streams from HBM once.  V_K is held as Bcat, a 2kp x M f16
// matrix (kp = k rounded up to 16) scaled by 2^s (s chosen so max|V| 2^s < 2^15): rows
// 0..k-1 hold hi = f16(V 2^s), rows kp..kp+k-1 hold lo = f16(V 2^s - hi).  One MMA with
// N = 2kp gives X hi and X lo in two halves of the accumulator (about 22 bits of the
// basis); the reduction adds them and multiplies by 2^-s, which is exact.
// Counts become f16 without any conversion instruction: for v < 1024 the f16 with bits
// 0x6400 | v is exactly 1024 + v, so one OR and one packed subtract give v.  Counts of
// 1024 or more are flagged (XPCS_ERANGE).
//
// Work item = (group of mb frame blocks of 128 frames, pixel split s); mb = 2 when two
// accumulators fit TMEM (N <= 256), so each Bcat tile loaded serves 256 frames.  Per
// 64-pixel chunk:
//   warp 0      TMA: mb X tiles (128 x 64) and the Bcat tile (2kp x 64, 128-byte swizzle)
//   warps 2..5  convert X to f16: u16 tiles in place (loaded with the same swizzle the
//               MMA reads, so the conversion is position-agnostic); u8 tiles into a
//               separate swizzled buffer
//   warp 1      MMA into mb 128 x 2kp f32 TMEM accumulators (N <= 256 per instruction)
// After the split's last chunk warps 2..5 drain TMEM, add the two halves and write the
// split's partial coefficients; a second kernel sums the splits in a fixed order.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "handles.h"
#include "internal.h"

namespace xpcs {

namespace {

constexpr int ENC_THREADS = 64 + 128;
constexpr int CONV_BYTES = TILE * KCH * 2;  // converted bf16 tile: 16 KB

struct EncLayout {
  int k, kp, N, nload, ns, mb, raw_bytes, b_bytes, stage_bytes, tmem_cols;
  __host__ __device__ EncLayout(int k_, int dtype) {
    k = k_;
    kp = (k_ + 15) / 16 * 16;  // lo half starts at column kp; N = 2 kp is a multiple of 32
    N = 2 * kp;
    nload = (N + 255) / 256;
    tmem_cols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : (N <= 256 ? 256 : 512)));
    mb = 2 * tmem_cols <= 512 ? 2 : 1;        // frame blocks sharing each basis tile
    raw_bytes = dtype == 0 ? TILE * KCH : 0;  // u16 converts in place
    b_bytes = N * 128;
    stage_bytes = mb * (raw_bytes + CONV_BYTES) + b_bytes;
    ns = (200 * 1024) / stage_bytes;
    if (ns > 8) ns = 8;
  }
  __host__ __device__ int smem() const { return 1024 + ns * stage_bytes + 256; }
};

__global__ void __launch_bounds__(ENC_THREADS, 1)
encode_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, const EncodeParams p,
              int n_items) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const EncLayout lay(p.k, p.dtype);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.ns * lay.stage_bytes);
  uint64_t* full = bars;               // [8] TMA landed (X + B)
  uint64_t* empty = bars + 8;          // [8] MMA done with the stage
  uint64_t* cfull = bars + 16;         // [8] conversion done
  uint64_t* tfull = bars + 24;         // accumulator ready
  uint64_t* tempty = bars + 25;        // accumulator drained
  uint64_t* mma_done = bars + 26;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 27);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // stage s: [B tile][conv tile 0..mb-1][raw tile 0..mb-1 (u8 only)]; 1024-aligned pieces
  auto b_of = [&](int s) { return smem + s * lay.stage_bytes; };
  auto conv_of = [&](int s, int i) { return smem + s * lay.stage_bytes + lay.b_bytes + i * CONV_BYTES; };
  auto raw_of = [&](int s, int i) {
    return smem + s * lay.stage_bytes + lay.b_bytes + lay.mb * CONV_BYTES + i * lay.raw_bytes;
  };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_chunks = (int)(p.px_per_split / KCH);
  const int n_m = p.T_pad / TILE;
  const int n_mp = (n_m + lay.mb - 1) / lay.mb;  // items: (group of mb frame blocks, pixel split)

  if (threadIdx.x == 0) {
    for (int s = 0; s < lay.ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&cfull[s], 128);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 4);
    mbar_init(mma_done, 1);
    mbar_fence_init();
    *abort_flag = 0;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, lay.mb * lay.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      tma_prefetch_desc(&tmX);
      tma_prefetch_desc(&tmB);
      uint32_t it = 0;
      bool ok = true;
      const uint32_t tx = (uint32_t)(lay.mb * TILE * KCH * (p.dtype == 0 ? 1 : 2) + lay.b_bytes);
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        const int mp = item % n_mp, sp = item / n_mp;
        const long long px0 = (long long)sp * p.px_per_split;
        for (int c = 0; c < n_chunks; ++c, ++it) {
          const uint32_t s = it % lay.ns, ph = (it / lay.ns) & 1;
          if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1, p.status)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          const int x = (int)(px0 + (long long)c * KCH);
          mbar_arrive_expect_tx(&full[s], tx);
          // frame blocks past the end read as zeros (rows beyond T)
          for (int i = 0; i < lay.mb; ++i)
            tma_load_2d(p.dtype == 0 ? raw_of(s, i) : conv_of(s, i), &tmX, &full[s], x, (mp * lay.mb + i) * TILE);
          for (int l = 0; l < lay.nload; ++l)
            tma_load_2d(b_of(s) + l * (lay.N / lay.nload) * 128, &tmB, &full[s], x, l * (lay.N / lay.nload));
        }
      }
      for (uint32_t j = (it > (uint32_t)lay.ns ? it - lay.ns : 0); j < it; ++j)
        mbar_wait(&full[j % lay.ns], (j / lay.ns) & 1, p.status);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const int nmma = (lay.N + 255) / 256;
      const int nper = lay.N / nmma;
      const uint32_t idesc = idesc_f16(0, TILE, nper);
      uint32_t it = 0, item_i = 0;
      bool ok = true, issued = false;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, ++item_i) {
        if (*abort_flag || !mbar_wait(tempty, (item_i & 1) ^ 1, p.status)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        for (int c = 0; c < n_chunks; ++c, ++it) {
          const uint32_t s = it % lay.ns, ph = (it / lay.ns) & 1;
          if (*abort_flag || !mbar_wait(&cfull[s], ph, p.status)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          for (int i = 0; i < lay.mb; ++i) {
            const uint64_t ad = smem_desc_sw128(conv_of(s, i));
            for (int h = 0; h < nmma; ++h) {
              const uint64_t bd = smem_desc_sw128(b_of(s) + h * nper * 128);
#pragma unroll
              for (int kk = 0; kk < KCH / 16; ++kk)
                tc_mma_f16(tmem_base + i * lay.tmem_cols + h * nper, ad + 2 * kk, bd + 2 * kk, idesc,
                           (c > 0 || kk > 0) ? 1u : 0u);
            }
          }
          issued = true;
          tc_commit(&empty[s]);
        }
        if (!ok) break;
        tc_commit(tfull);
      }
      if (issued) {
        tc_commit(mma_done);
        mbar_wait(mma_done, 0, p.status);
      }
    }
    __syncwarp();
  } else {
    // converters + epilogue: 128 threads
    const int ct = threadIdx.x - 64;
    const int quarter = warp & 3;
    const bool vec_out = p.k % 4 == 0 && reinterpret_cast<uintptr_t>(p.partials) % 16 == 0;
    uint32_t it = 0, item_i = 0;
    uint32_t over = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++item_i) {
      const int mp = item % n_mp, sp = item / n_mp;
      bool ok = true;
      for (int c = 0; c < n_chunks; ++c, ++it) {
        const uint32_t s = it % lay.ns, ph = (it / lay.ns) & 1;
        // warp-uniform decision so the warp stays converged for tcgen05.ld
        if (!__all_sync(0xffffffffu, !*abort_flag && mbar_wait(&full[s], ph, p.status))) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        for (int i = 0; i < lay.mb; ++i) {
        uint8_t* conv = conv_of(s, i);
        if (p.dtype == 1) {
          // in place: 1024 16-byte chunks, 8 per thread
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            uint4* ptr = reinterpret_cast<uint4*>(conv) + u * 128 + ct;
            uint4 v = *ptr;
            uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              over |= w[e] & 0xFC00FC00u;
              __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&(w[e] |= 0x64006400u)),
                                  __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
              w[e] = *reinterpret_cast<uint32_t*>(&h);
            }
            *ptr = make_uint4(w[0], w[1], w[2], w[3]);
          }
        } else {
          const uint8_t* raw = raw_of(s, i);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int unit = u * 128 + ct;
            const int row = unit >> 3, ch = unit & 7;
            const uint2 v = *reinterpret_cast<const uint2*>(raw + row * 64 + ch * 8);
            uint32_t w[4] = {__byte_perm(v.x, 0, 0x4140), __byte_perm(v.x, 0, 0x4342), __byte_perm(v.y, 0, 0x4140),
                             __byte_perm(v.y, 0, 0x4342)};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              w[e] |= 0x64006400u;
              __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&w[e]),
                                  __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
              w[e] = *reinterpret_cast<uint32_t*>(&h);
            }
            *reinterpret_cast<uint4*>(conv + row * 128 + ((ch ^ (row & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        }
        fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
        mbar_arrive(&cfull[s]);
      }
      if (!ok) break;
      // drain the accumulator: partial coefficients of this split
      if (!__all_sync(0xffffffffu, mbar_wait(tfull, item_i & 1, p.status))) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int row = quarter * 32 + lane;
      for (int i = 0; i < lay.mb; ++i) {
        const int m = mp * lay.mb + i;
        if (m >= n_m) break;  // warp-uniform
        float* dst = p.partials + ((size_t)sp * p.T_pad + (size_t)m * TILE + row) * p.k;
        for (int j0 = 0; j0 < p.k; j0 += 32) {
          uint32_t hi[32], lo[32];
          const uint32_t lane_base = tmem_base + i * lay.tmem_cols + ((uint32_t)(quarter * 32) << 16);
          tmem_ld32(lane_base + j0, hi);
          tmem_ld32(lane_base + lay.kp + j0, lo);
          tc_wait_ld();
          const int nj = min(32, p.k - j0);
          if (nj == 32 && vec_out) {  // the row's 32 coefficients as eight 16-byte stores
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(dst + j0 + j) =
                  make_float4(__uint_as_float(hi[j]) + __uint_as_float(lo[j]),
                              __uint_as_float(hi[j + 1]) + __uint_as_float(lo[j + 1]),
                              __uint_as_float(hi[j + 2]) + __uint_as_float(lo[j + 2]),
                              __uint_as_float(hi[j + 3]) + __uint_as_float(lo[j + 3]));
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nj) dst[j0 + j] = __uint_as_float(hi[j]) + __uint_as_float(lo[j]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
    }
    if (over) set_status(p.status, XPCS_DEV_RANGE);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, lay.mb * lay.tmem_cols);
  }
}

// A = scale * (sum of the split partials), added in split order.  Element g of A (row t,
// column j, g = t k + j) is element g of every split's slab of T_pad x k floats, so the
// sum runs over flat indices: four consecutive ones per thread (16-byte loads when A and
// the slabs allow it) and four splits' loads in flight before any is added.
__global__ void encode_reduce_kernel(const float* partials, int n_split, long long T, int T_pad, int k, float scale,
                                     float* A, int vec) {
  const long long g0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const long long n = T * k;
  if (g0 >= n) return;
  const size_t slab = (size_t)T_pad * k;
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  if (vec && g0 + 4 <= n) {
    const float4* p4 = reinterpret_cast<const float4*>(partials + g0);
    const size_t s4 = slab / 4;
    int s = 0;
    for (; s + 4 <= n_split; s += 4) {
      float4 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = __ldcs(p4 + (size_t)(s + u) * s4);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[0] += x[u].x;
        a[1] += x[u].y;
        a[2] += x[u].z;
        a[3] += x[u].w;
      }
    }
    for (; s < n_split; ++s) {
      const float4 x = __ldcs(p4 + (size_t)s * s4);
      a[0] += x.x;
      a[1] += x.y;
      a[2] += x.z;
      a[3] += x.w;
    }
    *reinterpret_cast<float4*>(A + g0) = make_float4(a[0] * scale, a[1] * scale, a[2] * scale, a[3] * scale);
    return;
  }
  for (long long g = g0; g < g0 + 4 && g < n; ++g) {
    float x = 0.f;
    for (int s = 0; s < n_split; ++s) x += partials[(size_t)s * slab + g];
    A[g] = x * scale;
  }
}

}  // namespace

int encode_smem_bytes(int k) { return EncLayout(k, 1).smem(); }
int encode_frame_blocks(int k) { return EncLayout(k, 1).mb; }

cudaError_t launch_encode(const CUtensorMap& tmX, const CUtensorMap& tmB, const EncodeParams& p, int grid,
                          cudaStream_t st) {
  const EncLayout lay(p.k, p.dtype);
  static int attr_bytes = 0;  // the attribute only ever grows
  if (lay.smem() > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.smem());
    if (e != cudaSuccess) return e;
    attr_bytes = lay.smem();
  }
  const int n_items = (p.T_pad / TILE + lay.mb - 1) / lay.mb * p.n_split;
  encode_kernel<<<grid, ENC_THREADS, lay.smem(), st>>>(tmX, tmB, p, n_items);
  return cudaGetLastError();
}

cudaError_t launch_encode_reduce(const float* partials, int n_split, long long T, int T_pad, int k, float scale,
                                 float* A, cudaStream_t st) {
  const long long n4 = (T * k + 3) / 4;  // four elements per thread
  const int vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0 && reinterpret_cast<uintptr_t>(partials) % 16 == 0) ? 1 : 0;
  encode_reduce_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>(partials, n_split, T, T_pad, k, scale, A, vec);
  return cudaGetLastError();
}

}  // namespace xpcs

// ====================================================================== ABI

using namespace xpcs;

// Pixel splits: choose the count whose item total best fills whole waves of SMs.
static int pick_splits(int n_m, long long M_pad, int num_sms) {
  const long long max_split = std::max<long long>(1, M_pad / (KCH * 8));
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= 64 && s <= max_split; ++s) {
    const long long items = (long long)n_m * s;
    const long long waves = (items + num_sms - 1) / num_sms;
    // per-item work shrinks as s grows; efficiency of the last wave and a mild
    // preference for fewer, longer items
    const double eff = (double)items / (double)(waves * num_sms) - 0.002 * s;
    if (items >= num_sms / 2 && eff > best_eff) {
      best_eff = eff;
      best = s;
    }
  }
  if (best_eff == 0.0) best = (int)std::min<long long>(max_split, std::max(1, (num_sms + n_m - 1) / n_m));
  return best;
}

// Partial-sum floats an encode of T frames needs (its pixel splits x padded frames x k).
size_t xpcs::encode_partials(const xpcs_basis* B, int64_t T, int num_sms) {
  const int nT = (int)((T + TILE - 1) / TILE);
  const int n_mp = (nT + encode_frame_blocks(B->k) - 1) / encode_frame_blocks(B->k);
  return (size_t)pick_splits(n_mp, B->M_pad, num_sms) * nT * TILE * B->k;
}

// Enqueue the encode of T frames X (device) into A_out on the context's stream, with
// `partials` (encode_partials floats) as its split-K scratch.
static xpcs_status enqueue_encode(xpcs_ctx* ctx, const xpcs_basis* B, const void* X, xpcs_dtype dtype, int64_t T,
                                  float* A_out, float* partials) {
  const int64_t M = B->rings->M;
  const int eb = dtype == XPCS_U8 ? 1 : 2;
  const int k = B->k;
  const int nT = (int)((T + TILE - 1) / TILE);
  const int T_pad = nT * TILE;
  const int mb = encode_frame_blocks(k);
  const int n_mp = (nT + mb - 1) / mb;  // work items: groups of mb frame blocks x pixel splits
  const int n_split = pick_splits(n_mp, B->M_pad, ctx->num_sms);
  const long long per = ((B->M_pad + n_split - 1) / n_split + KCH - 1) / KCH * KCH;
  CUtensorMap tmX, tmB;
  XPCS_TRY(make_map(ctx, &tmX, X, dtype == XPCS_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                    eb, M, T, KCH, TILE, dtype == XPCS_U8 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B));
  const int N = 2 * B->kp;
  XPCS_TRY(make_map(ctx, &tmB, B->d_Bcat, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, B->M_pad, N, KCH,
                    N / ((N + 255) / 256), CU_TENSOR_MAP_SWIZZLE_128B));
  EncodeParams p{};
  p.T = T;
  p.M = M;
  p.k = k;
  p.dtype = dtype;
  p.n_split = n_split;
  p.px_per_split = per;
  p.partials = partials;
  p.T_pad = T_pad;
  p.status = ctx->d_status;
  const int n_items = n_mp * n_split;
  XPCS_LAUNCH(ctx, "encode", 1, launch_encode(tmX, tmB, p, std::min(n_items, ctx->num_sms), ctx->stream));
  XPCS_LAUNCH(ctx, "encode_reduce", 1,
              launch_encode_reduce(partials, n_split, T, T_pad, k, std::ldexp(1.0f, -B->enc_log2), A_out, ctx->stream));
  return XPCS_OK;
}

// The encode of T frames X (device, 16-byte aligned rows) on stream `st` into A_out, with
// `partials` (encode_partials floats) as its split-K scratch and device status `status`:
// the stream's large steps, on the stream's own CUDA stream.
xpcs_status xpcs::encode_on_stream(xpcs_ctx* ctx, const xpcs_basis* B, const void* X, xpcs_dtype dtype,
                                   int64_t T, float* A_out, float* partials, uint32_t* status, cudaStream_t st) {
  const int64_t M = B->rings->M;
  const int eb = dtype == XPCS_U8 ? 1 : 2;
  const int k = B->k;
  const int nT = (int)((T + TILE - 1) / TILE);
  const int T_pad = nT * TILE;
  const int mb = encode_frame_blocks(k);
  const int n_mp = (nT + mb - 1) / mb;
  const int n_split = pick_splits(n_mp, B->M_pad, ctx->num_sms);
  const long long per = ((B->M_pad + n_split - 1) / n_split + KCH - 1) / KCH * KCH;
  CUtensorMap tmX, tmB;
  XPCS_TRY(make_map(ctx, &tmX, X, dtype == XPCS_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                    eb, M, T, KCH, TILE, dtype == XPCS_U8 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B));
  const int N = 2 * B->kp;
  XPCS_TRY(make_map(ctx, &tmB, B->d_Bcat, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, B->M_pad, N, KCH,
                    N / ((N + 255) / 256), CU_TENSOR_MAP_SWIZZLE_128B));
  EncodeParams p{};
  p.T = T;
  p.M = M;
  p.k = k;
  p.dtype = dtype;
  p.n_split = n_split;
  p.px_per_split = per;
  p.partials = partials;
  p.T_pad = T_pad;
  p.status = status;
  const int n_items = n_mp * n_split;
  cudaError_t e = launch_encode(tmX, tmB, p, std::min(n_items, ctx->num_sms), st);
  if (e == cudaSuccess)
    e = launch_encode_reduce(partials, n_split, T, T_pad, k, std::ldexp(1.0f, -B->enc_log2), A_out, st);
  if (e != cudaSuccess) return fail(ctx, XPCS_ECUDA, std::string("stream encode: ") + cudaGetErrorString(e));
  return XPCS_OK;
}

static xpcs_status encode_args(xpcs_ctx* ctx, const xpcs_basis* B, const void* X, xpcs_dtype dtype, int64_t T,
                               float* A_out) {
  if (!ctx || !B || !X || !A_out || T <= 0 || B->ctx != ctx || (dtype != XPCS_U8 && dtype != XPCS_U16))
    return fail(ctx, XPCS_EINVAL, "bad encode args");
  if ((B->rings->M * (dtype == XPCS_U8 ? 1 : 2)) % 16)
    return fail(ctx, XPCS_ENOTSUP, "encode needs M*elem_bytes to be a multiple of 16");
  return XPCS_OK;
}

extern "C" xpcs_status xpcs_encode(xpcs_ctx* ctx, const xpcs_basis* B, const void* X, xpcs_dtype dtype, int64_t T,
                                   float* A_out) {
  XPCS_TRY(encode_args(ctx, B, X, dtype, T, A_out));
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  Carve c0;
  c0.take<float>(encode_partials(B, T, ctx->num_sms));
  XPCS_TRY(ensure_scratch(ctx, c0.off));
  Carve c{0, static_cast<char*>(ctx->scratch)};
  float* partials = c.take<float>(encode_partials(B, T, ctx->num_sms));
  XPCS_TRY(enqueue_encode(ctx, B, X, dtype, T, A_out, partials));
  return finish(ctx);
}

// Encode of frames in host memory with the host-to-device copy overlapped: the frames go
// in blocks of ENC_HOST_BLOCK frames through ENC_HOST_BUFS device staging buffers, the
// copies alternating between two copy streams (so two copy engines can run at once), and
// each block is encoded on the context's stream as soon as it has landed while the next
// blocks are copied.  A buffer is refilled only after the encode that read it is done.
// The frames should be in pinned memory (pageable memory is copied synchronously).
constexpr int ENC_HOST_BUFS = 3;

extern "C" xpcs_status xpcs_encode_host(xpcs_ctx* ctx, const xpcs_basis* B, const void* X_host, xpcs_dtype dtype,
                                        int64_t T, float* A_out) {
  XPCS_TRY(encode_args(ctx, B, X_host, dtype, T, A_out));
  if (ctx->capturing) return fail(ctx, XPCS_EBUSY, "xpcs_encode_host cannot be captured");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t fb = (size_t)B->rings->M * (dtype == XPCS_U8 ? 1 : 2);  // bytes per frame
  // blocks of about 256 MB, a multiple of 128 frames
  const int64_t blk = std::max<int64_t>(TILE, std::min<int64_t>(T, ((256ll << 20) / (int64_t)fb) / TILE * TILE));
  const size_t part = encode_partials(B, blk, ctx->num_sms);
  Carve c0;
  for (int i = 0; i < ENC_HOST_BUFS; ++i) c0.take<char>((size_t)blk * fb);
  c0.take<float>(part);
  XPCS_TRY(ensure_scratch(ctx, c0.off));
  Carve c{0, static_cast<char*>(ctx->scratch)};
  char* stage[ENC_HOST_BUFS];
  for (int i = 0; i < ENC_HOST_BUFS; ++i) stage[i] = c.take<char>((size_t)blk * fb);
  float* partials = c.take<float>(part);
  if (!ctx->copy_stream[0]) {
    for (int i = 0; i < 2; ++i)
      XPCS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream[i], cudaStreamNonBlocking));
    for (int i = 0; i < ENC_HOST_BUFS; ++i) {
      XPCS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_loaded[i], cudaEventDisableTiming));
      XPCS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_free[i], cudaEventDisableTiming));
    }
  }
  // Copy scheme: whether two block copies in flight at once (two copy engines) move the
  // frames faster than one after the other depends on the host link of the machine, so the
  // first call times both on two 128 MB pieces of the caller's frames and keeps the faster
  // (two only when at least 5 % faster).  Each scheme is timed twice, alternating, and its
  // best time counts: the first copy of the caller's pages can be the slowest, which would
  // otherwise favour whichever scheme is timed after it.
  if (ctx->copy_streams == 0) {
    XPCS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the staging buffers are free
    const size_t piece = std::min<size_t>((size_t)blk * fb, (size_t)128 << 20);
    const size_t avail = (size_t)T * fb;
    if (avail < 2 * piece) {
      ctx->copy_streams = 1;
    } else {
      cudaEvent_t e[4];
      for (int i = 0; i < 4; ++i) XPCS_CUDA(ctx, cudaEventCreate(&e[i]));
      const char* hs = static_cast<const char*>(X_host);
      float best_one = 0.f, best_two = 0.f;
      cudaError_t ce = cudaSuccess;
      for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {
        // one stream: the two pieces one after the other
        ce = cudaEventRecord(e[0], ctx->copy_stream[0]);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(stage[0], hs, piece, cudaMemcpyHostToDevice, ctx->copy_stream[0]);
        if (ce == cudaSuccess)
          ce = cudaMemcpyAsync(stage[1], hs + piece, piece, cudaMemcpyHostToDevice, ctx->copy_stream[0]);
        if (ce == cudaSuccess) ce = cudaEventRecord(e[1], ctx->copy_stream[0]);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e[1]);
        // two streams: one piece on each, started together
        if (ce == cudaSuccess) ce = cudaEventRecord(e[2], ctx->copy_stream[0]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ctx->copy_stream[1], e[2], 0);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(stage[0], hs, piece, cudaMemcpyHostToDevice, ctx->copy_stream[0]);
        if (ce == cudaSuccess)
          ce = cudaMemcpyAsync(stage[1], hs + piece, piece, cudaMemcpyHostToDevice, ctx->copy_stream[1]);
        if (ce == cudaSuccess) ce = cudaEventRecord(ctx->ev_loaded[0], ctx->copy_stream[1]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ctx->copy_stream[0], ctx->ev_loaded[0], 0);
        if (ce == cudaSuccess) ce = cudaEventRecord(e[3], ctx->copy_stream[0]);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e[3]);
        float one = 0.f, two = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&one, e[0], e[1]);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&two, e[2], e[3]);
        if (ce == cudaSuccess) {
          best_one = rep ? std::min(best_one, one) : one;
          best_two = rep ? std::min(best_two, two) : two;
        }
      }
      for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
      if (ce != cudaSuccess) return fail(ctx, XPCS_ECUDA, std::string("copy calibration: ") + cudaGetErrorString(ce));
      ctx->copy_streams = best_two < 0.95f * best_one ? 2 : 1;
    }
  }
  // the staging buffers are scratch: earlier work on the context's stream may still use it
  XPCS_CUDA(ctx, cudaEventRecord(ctx->ev_free[0], ctx->stream));
  for (int i = 1; i < ENC_HOST_BUFS; ++i) XPCS_CUDA(ctx, cudaEventRecord(ctx->ev_free[i], ctx->stream));
  const char* src = static_cast<const char*>(X_host);
  for (int64_t t0 = 0, i = 0; t0 < T; t0 += blk, ++i) {
    const int64_t n = std::min(blk, T - t0);
    const int buf = (int)(i % ENC_HOST_BUFS);
    cudaStream_t cs = ctx->copy_stream[ctx->copy_streams == 2 ? i % 2 : 0];
    XPCS_CUDA(ctx, cudaStreamWaitEvent(cs, ctx->ev_free[buf], 0));
    XPCS_CUDA(ctx, cudaMemcpyAsync(stage[buf], src + (size_t)t0 * fb, (size_t)n * fb, cudaMemcpyHostToDevice, cs));
    XPCS_CUDA(ctx, cudaEventRecord(ctx->ev_loaded[buf], cs));
    XPCS_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_loaded[buf], 0));
    XPCS_TRY(enqueue_encode(ctx, B, stage[buf], dtype, n, A_out + (size_t)t0 * B->k, partials));
    XPCS_CUDA(ctx, cudaEventRecord(ctx->ev_free[buf], ctx->stream));
  }
  return finish(ctx);
}

// Encode plus the exact ring sums of the raw frames (the XPCS_QMEAN_EXACT_RAW option): the
// encode, then the ring-sum pass of the raw path over the same frames, both on the
// context's stream; waits once at the end unless the context is asynchronous.
extern "C" xpcs_status xpcs_encode_sums(xpcs_ctx* ctx, const xpcs_basis* B, const void* X, xpcs_dtype dtype,
                                        int64_t T, float* A_out, int64_t* S_out) {
  if (!ctx || !B || !S_out) return fail(ctx, XPCS_EINVAL, "bad encode_sums args");
  const bool async = ctx->async;
  ctx->async = true;
  xpcs_status st = xpcs_encode(ctx, B, X, dtype, T, A_out);
  if (st == XPCS_OK) st = xpcs_ring_sums(ctx, B->rings, X, dtype, T, S_out);
  ctx->async = async;
  return st == XPCS_OK ? finish(ctx) : st;
}
