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
constexpr int RU_QG = 12;     // w rows are padded to a multiple of RU_QG rings
constexpr int RU_KC = 32;     // coefficient rows are padded to a multiple of RU_KC

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
  if (p0 + 16 <= s.M && ((s.dtype == 0 ? (size_t)s.M : (size_t)s.M * 2) % 16) == 0) {
    // 16 counts: one 16-byte load (u8) or two (u16); frame rows are 16-byte aligned
    if (s.dtype == 0) {
      const uint4 v = *reinterpret_cast<const uint4*>(x8 + p0);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 16; ++e) xv[e] = (w[e >> 2] >> (8 * (e & 3))) & 0xffu;
    } else {
      const uint4 v0 = *reinterpret_cast<const uint4*>(x16 + p0);
      const uint4 v1 = *reinterpret_cast<const uint4*>(x16 + p0 + 8);
      const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int e = 0; e < 16; ++e) xv[e] = (w[e >> 1] >> (16 * (e & 1))) & 0xffffu;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const long long p = p0 + e;
      xv[e] = p < s.M ? (s.dtype == 0 ? (uint32_t)x8[p] : (uint32_t)x16[p]) : 0u;
    }
  }
#pragma unroll
  for (int e = 0; e < 16; ++e) cnt += xv[e] != 0;
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
      // eight independent sums keep eight basis-row loads in flight; fixed combine order
      const float* Bc = s.B32 + j0 + j;
      float a8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      int e = g;
      for (; e + 7 * ng < total; e += 8 * ng) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a8[u] = fmaf(nz_val[e + u * ng], Bc[(size_t)nz_idx[e + u * ng] * k], a8[u]);
      }
      for (; e < total; e += ng) a8[0] = fmaf(nz_val[e], Bc[(size_t)nz_idx[e] * k], a8[0]);
      acc = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
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
  const float* src = s.part + (size_t)fi * s.nblk * s.k + j;
  float a8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int b = 0;
  for (; b + 8 <= s.nblk; b += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a8[u] += src[(size_t)(b + u) * s.k];
  }
  for (; b < s.nblk; ++b) a8[0] += src[(size_t)b * s.k];
  s.a[gid] = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
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
      float v4[4] = {0.f, 0.f, 0.f, 0.f};
      int c = 0;
      for (; c + 4 <= k; c += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) v4[u] = fmaf(as[c + u], Gq[(size_t)(c + u) * k + j], v4[u]);
      }
      for (; c < k; ++c) v4[0] = fmaf(as[c], Gq[(size_t)c * k + j], v4[0]);
      v = ((v4[0] + v4[1]) + (v4[2] + v4[3])) * r;
    }
    wrow[j] = v;
  }
  if (q == 0)
    for (int c = tid; c < ka; c += blockDim.x) s.Ah[slot * ka + c] = c < k ? as[c] : 0.f;
}

// --------------------------------------------------------------------------- 3. rows
// CTA = 128 consecutive lags tau0 .. tau0 + 127 x a group of RU_QG rings; warp = 6 rings
// (RU_RQ), lane = lags tau0 + lane + 32 m (m = 0..3).  For frame t of the batch and lag
// tau the history row is s = t - tau, so the CTA needs rows t - tau0 - 127 .. t - tau0:
// they sit in a circular shared window of RU_WIN rows, and each chunk of RU_FB frames
// shifts it by RU_FB rows, loaded (cp.async) while the previous chunk computes.  Per frame
// the rings' w rows are staged (double buffer, broadcast reads); every thread forms its
// 6 x 4 dot products over k from shared memory and folds the valid ones into per-thread
// lag-bin sums, written back once per batch (each bin has one owner: no atomics).
// Consecutive lanes read consecutive window rows; the row pitch ka + 4 floats puts a
// quarter-warp's 16-byte reads on distinct banks.
constexpr int RU_RQ = 6;                 // rings per warp
constexpr int RU_M = 4;                  // lags per lane
constexpr int RU_FB = 16;                // frames per window shift
constexpr int RU_WIN = RU_LAGS + 2 * RU_FB;

XPCS_DEV void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
XPCS_DEV void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
XPCS_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
XPCS_DEV void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
XPCS_DEV void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

struct RuLayout {
  int ka, qg, pitch;
  __host__ __device__ int a_floats() const { return RU_WIN * pitch; }
  __host__ __device__ int r_floats() const { return RU_WIN * qg; }
  __host__ __device__ int w_floats() const { return qg * ka; }
  __host__ __device__ int bytes() const { return (a_floats() + r_floats() + 2 * w_floats()) * 4; }
};

// window row of history frame s (s may be negative: such rows are zero)
XPCS_DEV int win_row(long long s) { return (int)(((s % RU_WIN) + RU_WIN) % RU_WIN); }

// Issue the copies of window rows s0 .. s1 - 1 (A and the group's r values): one warp
// per row, 16-byte pieces for A, 4-byte pieces for r.
XPCS_DEV void load_rows(const StreamStep& s, const RuLayout& L, float* Aw, float* Rw, int q_base, long long s0,
                        long long s1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int pieces = L.ka / 4;
  for (long long sr = s0 + warp; sr < s1; sr += nwarps) {
    const int wr = win_row(sr);
    float* arow = Aw + wr * L.pitch;
    float* rrow = Rw + wr * L.qg;
    if (sr >= 0) {
      const size_t slot = (size_t)(sr % s.cap);
      const float* asrc = s.Ah + slot * L.ka;
      for (int c = lane; c < pieces; c += 32) cp_async16(arow + 4 * c, asrc + 4 * c);
      const float* rsrc = s.Rh + slot * s.n_q + q_base;
      for (int u = lane; u < L.qg; u += 32) {
        if (q_base + u < s.n_q)
          cp_async4(rrow + u, rsrc + u);
        else
          rrow[u] = 0.f;
      }
    } else {
      for (int c = lane; c < pieces; c += 32)
        *reinterpret_cast<float4*>(arow + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int u = lane; u < L.qg; u += 32) rrow[u] = 0.f;
    }
  }
}

XPCS_DEV void load_w(const StreamStep& s, const RuLayout& L, float* Wd, int fi, int nqp, int q_base) {
  const int rows = min(L.qg, nqp - q_base);
  const int n = rows * L.ka / 4;
  const float* src = s.w + ((size_t)fi * nqp + q_base) * L.ka;
  for (int e = threadIdx.x; e < n; e += blockDim.x) cp_async16(Wd + 4 * e, src + 4 * e);
}

__global__ void row_update_kernel(const StreamStep s, int ka, int nqp, RuLayout L) {
  extern __shared__ __align__(16) float ru_smem[];
  float* Aw = ru_smem;
  float* Rw = Aw + L.a_floats();
  float* Wb = Rw + L.r_floats();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long tau0 = (long long)blockIdx.x * RU_LAGS;
  const int q_base = blockIdx.y * L.qg;
  const int qw = warp * RU_RQ;       // first ring of this warp within the group
  const bool active = q_base + qw < s.n_q;

  float sum[RU_RQ][RU_M];
  int cnt[RU_RQ][RU_M];
#pragma unroll
  for (int u = 0; u < RU_RQ; ++u)
#pragma unroll
    for (int m = 0; m < RU_M; ++m) {
      sum[u][m] = 0.f;
      cnt[u][m] = 0;
    }

  // rows of the first chunk, and w of frame 0
  const long long base0 = s.t0 - tau0;
  load_rows(s, L, Aw, Rw, q_base, base0 - (RU_LAGS - 1), base0 + RU_FB);
  load_w(s, L, Wb, 0, nqp, q_base);
  cp_async_commit();
  for (int fi = 0; fi < s.b; ++fi) {
    // prefetch: w of the next frame; at a chunk's first frame, the next chunk's rows
    if (fi + 1 < s.b) load_w(s, L, Wb + ((fi + 1) & 1) * L.w_floats(), fi + 1, nqp, q_base);
    if (fi % RU_FB == 0 && fi + RU_FB < s.b) {
      const long long nb = base0 + fi + RU_FB;  // first frame of the next chunk, relative
      load_rows(s, L, Aw, Rw, q_base, nb, nb + RU_FB);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const long long t = s.t0 + fi;
    if (active) {
      const float* Wf = Wb + (fi & 1) * L.w_floats() + qw * L.ka;
      int wr[RU_M];
      bool lag_ok[RU_M];
#pragma unroll
      for (int m = 0; m < RU_M; ++m) {
        const long long tau = tau0 + lane + 32 * m;
        const long long sr = t - tau;
        lag_ok[m] = tau < s.W && sr >= 0;
        wr[m] = win_row(sr);
      }
      float dot[RU_RQ][RU_M];
#pragma unroll
      for (int u = 0; u < RU_RQ; ++u)
#pragma unroll
        for (int m = 0; m < RU_M; ++m) dot[u][m] = 0.f;
#pragma unroll 2
      for (int c = 0; c < ka; c += 4) {
        float4 a[RU_M];
#pragma unroll
        for (int m = 0; m < RU_M; ++m) a[m] = *reinterpret_cast<const float4*>(Aw + wr[m] * L.pitch + c);
#pragma unroll
        for (int u = 0; u < RU_RQ; ++u) {
          const float4 wv = *reinterpret_cast<const float4*>(Wf + u * L.ka + c);
#pragma unroll
          for (int m = 0; m < RU_M; ++m) {
            dot[u][m] = fmaf(wv.x, a[m].x, dot[u][m]);
            dot[u][m] = fmaf(wv.y, a[m].y, dot[u][m]);
            dot[u][m] = fmaf(wv.z, a[m].z, dot[u][m]);
            dot[u][m] = fmaf(wv.w, a[m].w, dot[u][m]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < RU_RQ; ++u) {
        const int q = q_base + qw + u;
        const float rt = q < s.n_q ? __ldg(s.Rh + (size_t)(t % s.cap) * s.n_q + q) : 0.f;
#pragma unroll
        for (int m = 0; m < RU_M; ++m) {
          const float rs = Rw[wr[m] * L.qg + qw + u];
          if (lag_ok[m] && rt > 0.f && rs > 0.f) {
            sum[u][m] = fmaf(dot[u][m], rs, sum[u][m]);
            cnt[u][m] += 1;
          }
        }
      }
    }
    __syncthreads();  // buffers of this frame may be overwritten from here on
  }
  cp_async_wait0();
  if (!active) return;
#pragma unroll
  for (int u = 0; u < RU_RQ; ++u) {
    const int q = q_base + qw + u;
    if (q >= s.n_q) continue;
#pragma unroll
    for (int m = 0; m < RU_M; ++m) {
      const long long tau = tau0 + lane + 32 * m;
      if (tau < s.W && cnt[u][m]) {
        s.g2sum[(size_t)q * s.W + tau] += (double)sum[u][m];
        s.cnt[(size_t)q * s.W + tau] += cnt[u][m];
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
  RuLayout L{ka, ka <= 128 ? 36 : 18, ka + 4};
  const int smem = L.bytes();
  static int attr_bytes = 0;  // the attribute only ever grows
  if (smem > attr_bytes) {
    if ((e = cudaFuncSetAttribute(row_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    attr_bytes = smem;
  }
  const dim3 grid((unsigned)((s.W + RU_LAGS - 1) / RU_LAGS), (unsigned)((s.n_q + L.qg - 1) / L.qg));
  row_update_kernel<<<grid, 32 * (L.qg / RU_RQ), smem, st>>>(s, ka, nqp, L);
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
