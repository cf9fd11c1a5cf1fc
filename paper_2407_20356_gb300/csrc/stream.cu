// Online compression and correlation (Sec. 2.2, Fig. 1c; timings of Sec. 3.2): each
// pushed frame is encoded, appended to the coefficient history, and its two-time row
// against the whole window is folded into running g2 sums, without storing C.
//
// Per batch of b frames t0 .. t0 + b - 1:
//   1. sparse encode: a_t = sum over pixels with x_p > 0 of x_p V_K[p, :] (f32).  Only the
//      nonzero pixels' basis rows are read, a few percent of V_K at low photon rates.
//      Per-slice partials are summed in a fixed order (deterministic).
//   2. frame factors: S~_q(t) = a_t s_q, r_q(t) = sqrt(M_q)/S~_q(t) (0 if undefined),
//      w_q(t) = r_q(t) a_t G_q; a_t and r_q(t) go into the ring buffer slot of t.
//   3. row update: for every lag tau < W, thread tau takes history row s = t - tau and adds
//      C_q(t, s) = w_q(t) . a_s r_q(s) to g2sum_q[tau] (count_q[tau] += 1) for all rings.
//      Each thread owns its lag bins: no atomics, deterministic for a given batching.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace xpcs {

namespace {

constexpr int SE_PX = 4096;   // pixels per sparse-encode slice
constexpr int RU_LAGS = 128;  // lags per row-update block
constexpr int RU_QG = 12;     // rings per register group in the row update
constexpr int RU_KC = 32;     // coefficient chunk held in registers

// --------------------------------------------------------------------------- 1. encode
__global__ void __launch_bounds__(256) sparse_encode_kernel(const StreamStep s) {
  __shared__ int nz_idx[SE_PX];
  __shared__ float nz_val[SE_PX];
  __shared__ int warp_tot[8];
  __shared__ float red[256];
  const int blk = blockIdx.x, fi = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long p0 = (long long)blk * SE_PX + (long long)tid * 16;
  const uint8_t* x8 = static_cast<const uint8_t*>(s.X) + (size_t)fi * s.M;
  const uint16_t* x16 = static_cast<const uint16_t*>(s.X) + (size_t)fi * s.M;
  uint32_t xv[16];
  int cnt = 0;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const long long p = p0 + e;
    uint32_t x = 0;
    if (p < s.M) x = s.dtype == 0 ? x8[p] : x16[p];
    xv[e] = x;
    cnt += x != 0;
  }
  // block-wide exclusive scan of the nonzero counts
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int base = 0, total = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    if (w < warp) base += warp_tot[w];
    total += warp_tot[w];
  }
  int off = base + incl - cnt;
#pragma unroll
  for (int e = 0; e < 16; ++e)
    if (xv[e]) {
      nz_idx[off] = (int)(p0 + e);
      nz_val[off] = (float)xv[e];
      ++off;
    }
  __syncthreads();
  // accumulate: ng groups of k threads split the nonzero list
  const int k = s.k;
  for (int j0 = 0; j0 < k; j0 += 256) {
    const int kk = min(256, k - j0);
    const int ng = max(1, 256 / kk);
    const int g = tid / kk, j = tid % kk;
    float acc = 0.f;
    if (g < ng) {
      const float* Bc = s.B32 + j0 + j;
      for (int e = g; e < total; e += ng) acc = fmaf(nz_val[e], Bc[(size_t)nz_idx[e] * k], acc);
    }
    red[tid] = acc;
    __syncthreads();
    if (tid < kk) {
      float a = 0.f;
      for (int gg = 0; gg < ng; ++gg) a += red[gg * kk + tid];
      s.part[((size_t)fi * s.nblk + blk) * k + j0 + tid] = a;
    }
    __syncthreads();
  }
}

__global__ void stream_reduce_kernel(const StreamStep s) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= s.b * s.k) return;
  const int fi = gid / s.k, j = gid % s.k;
  float a = 0.f;
  for (int b = 0; b < s.nblk; ++b) a += s.part[((size_t)fi * s.nblk + b) * s.k + j];
  s.a[gid] = a;
}

// --------------------------------------------------------------------------- 2. factors
// Block (frame i, ring q), 128 threads.  Rows of Ah and w are padded to ka = k rounded up
// to 32 (zeros), and w to a multiple of RU_QG rings, so the row update needs no bounds.
__global__ void __launch_bounds__(128) frame_factors_kernel(const StreamStep s, int ka, int nqp) {
  __shared__ float as[256];
  __shared__ double dred[4];
  const int fi = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
  const int k = s.k;
  const long long t = s.t0 + fi;
  const long long slot = t % s.cap;
  for (int c = tid; c < k; c += blockDim.x) as[c] = s.a[(size_t)fi * k + c];
  __syncthreads();
  float r = 0.f;
  if (q < s.n_q) {
    // S~_q(t) in FP64 (k terms)
    double d = 0.0;
    for (int c = tid; c < k; c += blockDim.x) d = fma((double)as[c], s.s64[(size_t)q * k + c], d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((tid & 31) == 0) dred[tid >> 5] = d;
    __syncthreads();
    const double S = dred[0] + dred[1] + dred[2] + dred[3];
    r = S > 0.0 ? (float)(sqrt((double)s.Mq[q]) / S) : 0.f;
    if (tid == 0) s.Rh[slot * s.n_q + q] = r;
  }
  float* wrow = s.w + ((size_t)fi * nqp + q) * ka;
  const float* Gq = s.G32 + (size_t)(q < s.n_q ? q : 0) * k * k;
  for (int j = tid; j < ka; j += blockDim.x) {
    float v = 0.f;
    if (q < s.n_q && j < k && r > 0.f) {
      for (int c = 0; c < k; ++c) v = fmaf(as[c], Gq[(size_t)c * k + j], v);
      v *= r;
    }
    wrow[j] = v;
  }
  if (q == 0)
    for (int c = tid; c < ka; c += blockDim.x) s.Ah[slot * ka + c] = c < k ? as[c] : 0.f;
}

// --------------------------------------------------------------------------- 3. rows
// Block = 128 consecutive lags, thread = one lag tau.  For each group of RU_QG rings and
// each frame of the batch: w for those rings is staged in shared memory (broadcast
// reads), the thread streams its history row s = t - tau through registers in chunks of
// RU_KC and forms RU_QG dot products; valid pairs are summed in registers and the lag's
// bins are updated once per ring group.
__global__ void __launch_bounds__(RU_LAGS) row_update_kernel(const StreamStep s, int ka, int nqp) {
  extern __shared__ float wq[];  // [RU_QG][ka]
  const int tid = threadIdx.x;
  const long long tau = (long long)blockIdx.x * RU_LAGS + tid;
  const bool lag_ok = tau < s.W;
  for (int qg = 0; qg < s.n_q; qg += RU_QG) {
    float sums[RU_QG];
    int cnts[RU_QG];
#pragma unroll
    for (int u = 0; u < RU_QG; ++u) {
      sums[u] = 0.f;
      cnts[u] = 0;
    }
    for (int fi = 0; fi < s.b; ++fi) {
      __syncthreads();
      const float* wsrc = s.w + ((size_t)fi * nqp + qg) * ka;
      for (int e = tid; e < RU_QG * ka; e += RU_LAGS) wq[e] = wsrc[e];
      __syncthreads();
      const long long t = s.t0 + fi;
      const long long sidx = t - tau;
      if (!lag_ok || sidx < 0) continue;
      const long long slot = sidx % s.cap;
      const long long tslot = t % s.cap;
      const float* row = s.Ah + slot * ka;
      float dots[RU_QG];
#pragma unroll
      for (int u = 0; u < RU_QG; ++u) dots[u] = 0.f;
      for (int c0 = 0; c0 < ka; c0 += RU_KC) {
        float rv[RU_KC];
#pragma unroll
        for (int c = 0; c < RU_KC; c += 4) {
          const float4 v4 = *reinterpret_cast<const float4*>(row + c0 + c);
          rv[c] = v4.x;
          rv[c + 1] = v4.y;
          rv[c + 2] = v4.z;
          rv[c + 3] = v4.w;
        }
#pragma unroll
        for (int u = 0; u < RU_QG; ++u) {
          const float* wu = wq + u * ka + c0;
#pragma unroll
          for (int c = 0; c < RU_KC; c += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(wu + c);
            dots[u] = fmaf(w4.x, rv[c], dots[u]);
            dots[u] = fmaf(w4.y, rv[c + 1], dots[u]);
            dots[u] = fmaf(w4.z, rv[c + 2], dots[u]);
            dots[u] = fmaf(w4.w, rv[c + 3], dots[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < RU_QG; ++u) {
        const int q = qg + u;
        if (q < s.n_q) {
          const float rs = s.Rh[slot * s.n_q + q];
          const float rt = s.Rh[tslot * s.n_q + q];
          if (rs > 0.f && rt > 0.f) {
            sums[u] += dots[u] * rs;
            cnts[u] += 1;
          }
        }
      }
    }
    if (lag_ok) {
#pragma unroll
      for (int u = 0; u < RU_QG; ++u) {
        const int q = qg + u;
        if (q < s.n_q && cnts[u]) {
          s.g2sum[(size_t)q * s.W + tau] += (double)sums[u];
          s.cnt[(size_t)q * s.W + tau] += cnts[u];
        }
      }
    }
  }
}

__global__ void stream_g2_kernel(const double* g2sum, const long long* cnt, long long n, double* g2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g2[i] = cnt[i] > 0 ? g2sum[i] / (double)cnt[i] : __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void basis_f32_kernel(const double* B, long long n, float* B32) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    B32[i] = (float)B[i];
}

}  // namespace

cudaError_t launch_stream_step(const StreamStep& s, cudaStream_t st) {
  const int ka = (s.k + RU_KC - 1) / RU_KC * RU_KC;
  const int nqp = (s.n_q + RU_QG - 1) / RU_QG * RU_QG;
  sparse_encode_kernel<<<dim3(s.nblk, s.b), 256, 0, st>>>(s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stream_reduce_kernel<<<(s.b * s.k + 255) / 256, 256, 0, st>>>(s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  frame_factors_kernel<<<dim3(s.b, nqp), 128, 0, st>>>(s, ka, nqp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int smem = RU_QG * ka * (int)sizeof(float);
  const unsigned grid = (unsigned)((s.W + RU_LAGS - 1) / RU_LAGS);
  row_update_kernel<<<grid, RU_LAGS, smem, st>>>(s, ka, nqp);
  return cudaGetLastError();
}

cudaError_t launch_stream_g2(const double* g2sum, const long long* cnt, long long n, double* g2, cudaStream_t st) {
  stream_g2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g2sum, cnt, n, g2);
  return cudaGetLastError();
}

cudaError_t launch_basis_f32(const double* B, long long n, float* B32, cudaStream_t st) {
  basis_f32_kernel<<<1024, 256, 0, st>>>(B, n, B32);
  return cudaGetLastError();
}

}  // namespace xpcs
