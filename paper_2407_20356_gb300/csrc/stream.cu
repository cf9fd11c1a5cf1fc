// Online compression and correlation (Sec. 2.2, Fig. 1c; timings of Sec. 3.2): each
// pushed frame is encoded, appended to the coefficient history, and its two-time row
// against the whole window is folded into running g2 sums, without storing C.
//
// Per batch of b frames t0 .. t0 + b - 1:
//   1. sparse encode: a_t = sum over pixels with x_p > 0 of x_p V_K[p, :] (f32).  Only the
//      nonzero pixels' basis rows are read, a few percent of V_K at low photon rates.
//      Per-slice partials are summed in a fixed order (deterministic).
//      With exact ring sums (XPCS_QMEAN_EXACT_RAW) the same pass adds each nonzero count
//      into its ring's sum S_q(t).
//   2. frame factors: S~_q(t) = a_t s_q (or the exact S_q(t)), r_q(t) = sqrt(M_q)/S~_q(t)
//      (0 if undefined),
//      w_q(t) = r_q(t) a_t G_q; a_t and r_q(t) go into the ring buffer slot of t.
//   3. row update: for every lag tau < W and ring q, C_q(t, s) = w_q(t) . a_s r_q(s) with
//      s = t - tau is added to g2sum_q[tau] and the pair to count_q[tau] (on the tensor
//      cores: the single-frame kernel, the row update kernel, or the two-time kernel and
//      its fold for steps of 32 frames or more; single frames defer their pair counts to
//      64-frame blocks).  Each (ring, lag) bin has one owner per step: no atomics,
//      deterministic for a given batching.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace xpcs {

namespace {

constexpr int SE_PX = 4096;   // pixels per sparse-encode slice

// --------------------------------------------------------------------------- 1. encode
constexpr int SE_MAX_RINGS = 1024;
__global__ void __launch_bounds__(256) sparse_encode_kernel(const StreamStep s) {
  __shared__ int nz_idx[SE_PX];
  __shared__ float nz_val[SE_PX];
  __shared__ int warp_tot[8];
  __shared__ float red[256];
  __shared__ float4 red4[256];
  __shared__ int se_last;
  __shared__ unsigned ring_acc[SE_MAX_RINGS];  // exact ring sums of this slice (at most 2^28)
  pdl_trigger();
  const int blk = blockIdx.x, fi = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long p0 = (long long)blk * SE_PX + (long long)tid * 16;
  const uint8_t* x8 = static_cast<const uint8_t*>(s.X) + (size_t)fi * s.M;
  const uint16_t* x16 = static_cast<const uint16_t*>(s.X) + (size_t)fi * s.M;
  uint32_t xv[16];
  int cnt = 0;
  if (s.vec16 && p0 + 16 <= s.M) {
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
  if (s.Sx) {  // exact ring sums: each nonzero count into its ring, then one atomic per ring
    for (int q = tid; q < s.n_q; q += 256) ring_acc[q] = 0u;
    __syncthreads();
    for (int e = tid; e < total; e += 256) {
      const int q = s.qmap[nz_idx[e]];
      if (q >= 0) atomicAdd(&ring_acc[q], (unsigned)nz_val[e]);
    }
    __syncthreads();
    for (int q = tid; q < s.n_q; q += 256)
      if (ring_acc[q]) atomicAdd(reinterpret_cast<unsigned long long*>(s.Sx + (size_t)fi * s.n_q + q),
                                 (unsigned long long)ring_acc[q]);
  }
  // accumulate: ng groups of k threads split the nonzero list
  const int k = s.k;
  if ((k & 3) == 0) {
    // 16-byte loads: a group of k / 4 threads reads a basis row (a warp reads 512 bytes at
    // once for k = 128), 256 / (k / 4) groups split the nonzero list and each thread keeps
    // eight rows' loads in flight; the groups' sums are added in a fixed order
    const int k4 = k >> 2, ng = 256 / k4;
    const int g = tid / k4, j4 = tid - g * k4;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g < ng) {
      const float4* B4 = reinterpret_cast<const float4*>(s.B32) + j4;
      float4 a8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a8[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      int e = g;
      for (; e + 7 * ng < total; e += 8 * ng) {
        float4 b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) b[u] = __ldg(B4 + (size_t)nz_idx[e + u * ng] * k4);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float x = nz_val[e + u * ng];
          a8[u].x = fmaf(x, b[u].x, a8[u].x);
          a8[u].y = fmaf(x, b[u].y, a8[u].y);
          a8[u].z = fmaf(x, b[u].z, a8[u].z);
          a8[u].w = fmaf(x, b[u].w, a8[u].w);
        }
      }
      for (; e < total; e += ng) {
        const float4 b = __ldg(B4 + (size_t)nz_idx[e] * k4);
        const float x = nz_val[e];
        a8[0].x = fmaf(x, b.x, a8[0].x);
        a8[0].y = fmaf(x, b.y, a8[0].y);
        a8[0].z = fmaf(x, b.z, a8[0].z);
        a8[0].w = fmaf(x, b.w, a8[0].w);
      }
#pragma unroll
      for (int u = 1; u < 8; ++u) {
        a8[0].x += a8[u].x;
        a8[0].y += a8[u].y;
        a8[0].z += a8[u].z;
        a8[0].w += a8[u].w;
      }
      a = a8[0];
    }
    red4[tid] = a;
    // the slice partials are rewritten only once the kernels ahead (the previous step's,
    // which read them) have completed
    pdl_wait();
    __syncthreads();
    float4* part4 = reinterpret_cast<float4*>(s.part);
    if (tid < k4) {
      float4 t = red4[tid];
      for (int gg = 1; gg < ng; ++gg) {
        const float4 v = red4[gg * k4 + tid];
        t.x += v.x;
        t.y += v.y;
        t.z += v.z;
        t.w += v.w;
      }
      part4[((size_t)fi * s.nblk + blk) * k4 + tid] = t;
    }
    // the frame's last slice block adds the nblk partials: a_t[j], 8 slice groups x 32
    // column quads (group g: slices g, g + 8, ... in order, then the groups in order)
    __threadfence();
    __syncthreads();
    if (tid == 0) se_last = atomicAdd(s.se_done + fi, 1u) == (unsigned)(s.nblk - 1);
    __syncthreads();
    if (!se_last) return;
    __threadfence();
    const int cg = tid >> 5;
    for (int c0 = 0; c0 < k4; c0 += 32) {
      const int c4 = c0 + lane;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c4 < k4) {
        const float4* src = part4 + (size_t)fi * s.nblk * k4 + c4;
        float4 a4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        int b0 = cg;
        for (; b0 + 3 * 8 < s.nblk; b0 += 4 * 8) {
          float4 x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) x[u] = __ldcg(src + (size_t)(b0 + 8 * u) * k4);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            a4[u].x += x[u].x;
            a4[u].y += x[u].y;
            a4[u].z += x[u].z;
            a4[u].w += x[u].w;
          }
        }
        for (; b0 < s.nblk; b0 += 8) {
          const float4 x = __ldcg(src + (size_t)b0 * k4);
          a4[0].x += x.x;
          a4[0].y += x.y;
          a4[0].z += x.z;
          a4[0].w += x.w;
        }
        acc.x = (a4[0].x + a4[1].x) + (a4[2].x + a4[3].x);
        acc.y = (a4[0].y + a4[1].y) + (a4[2].y + a4[3].y);
        acc.z = (a4[0].z + a4[1].z) + (a4[2].z + a4[3].z);
        acc.w = (a4[0].w + a4[1].w) + (a4[2].w + a4[3].w);
      }
      red4[tid] = acc;
      __syncthreads();
      if (cg == 0 && c4 < k4) {
        float4 t = red4[lane];
#pragma unroll
        for (int gg = 1; gg < 8; ++gg) {
          const float4 v = red4[gg * 32 + lane];
          t.x += v.x;
          t.y += v.y;
          t.z += v.z;
          t.w += v.w;
        }
        reinterpret_cast<float4*>(s.a + (size_t)fi * k)[c4] = t;
      }
      __syncthreads();
    }
    if (tid == 0) s.se_done[fi] = 0u;  // ready for the next step
    return;
  }
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
    if (j0 == 0) pdl_wait();  // the previous step's kernels read the partials
    __syncthreads();
    if (tid < kk) {
      float a = 0.f;
      for (int gg = 0; gg < ng; ++gg) a += red[gg * kk + tid];
      s.part[((size_t)fi * s.nblk + blk) * k + j0 + tid] = a;
    }
    __syncthreads();
  }
  // (it waited before its first partial store: the kernels ahead, the previous step's,
  // read the partials, and the frame factors behind it rewrite rows they read; waiting
  // also keeps completion transitive along the chain)
}

// a_t[j] = sum of the nblk slice partials of frame t.  Block = 32 (frame, column) pairs x
// 8 slice groups: group g sums slices g, g + 8, g + 16, ... (32 loads in flight per thread,
// each warp reading 32 consecutive columns), then group 0 adds the eight group sums in
// order.  The order is fixed by nblk alone (deterministic, the same for every batching).
constexpr int RD_GROUPS = 8;
__global__ void __launch_bounds__(256) stream_reduce_kernel(const StreamStep s) {
  __shared__ float red[RD_GROUPS][32];
  pdl_trigger();
  pdl_wait();  // the slice partials
  const int jj = threadIdx.x & 31, g = threadIdx.x >> 5;
  const long long col = (long long)blockIdx.x * 32 + jj;  // (frame, column) = (col / k, col mod k)
  const bool live = col < (long long)s.b * s.k;
  float acc = 0.f;
  if (live) {
    const int fi = (int)(col / s.k), j = (int)(col - (long long)fi * s.k);
    const float* src = s.part + (size_t)fi * s.nblk * s.k + j;
    const size_t stride = (size_t)RD_GROUPS * s.k;  // between a group's consecutive slices
    float a4[4] = {0.f, 0.f, 0.f, 0.f};
    int blk = g;
    for (; blk + 31 * RD_GROUPS < s.nblk; blk += 32 * RD_GROUPS) {
      float x[32];
      const float* p0 = src + (size_t)blk * s.k;
#pragma unroll
      for (int u = 0; u < 32; ++u) x[u] = p0[u * stride];
#pragma unroll
      for (int u = 0; u < 32; ++u) a4[u & 3] += x[u];
    }
    for (; blk < s.nblk; blk += RD_GROUPS) a4[0] += src[(size_t)blk * s.k];
    acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
  }
  red[g][jj] = acc;
  __syncthreads();
  if (g == 0 && live) {
    float a = red[0][jj];
#pragma unroll
    for (int gg = 1; gg < RD_GROUPS; ++gg) a += red[gg][jj];
    s.a[col] = a;
  }
}

// --------------------------------------------------------------------------- 2. factors
// Block (frame i, ring q), 128 threads: S~_q(t) = a_t . s_q (FP64), r_q(t) = sqrt(M_q)/S~
// (0 if undefined) into Rh (and its mirror row), w_q(t) = r_q(t) a_t G_q as a bf16 hi | lo
// row of W2 in pair order; the q = 0 block also writes a_t as a bf16 hi | lo history row
// of A2 (and its mirror row).  A stream in f16 writes the rows as one f16 piece (the first
// kpad elements): w_q(t) as it is (its elements are r_q(t)-normalised, like the operand
// rows of the offline f16 path), the history row as 2^e a_t with e chosen so that the
// largest |a_t| lies in [2^13, 2^14) (no overflow, small elements stay normal), and
// 2^-e r_q(t) in Rh, so that the products r_q(s) (w_q(t) . a_s) are unchanged.
XPCS_DEV void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// SPLIT (1 or 4) threads per w column split the k terms of w_q(t) (one-frame steps: the
// G_q loads of a column in one round instead of four), their sums added in split order.
template <int SPLIT>
XPCS_DEV void frame_factors(const StreamStep& s) {
  constexpr int NW = 4 * SPLIT;  // warps
  __shared__ float as[256];
  __shared__ double dred[NW];
  __shared__ unsigned mred[NW];
  __shared__ float vpart[SPLIT][256];
  pdl_trigger();
  pdl_wait();  // the coefficients
  const int fi = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
  const int k = s.k, kp = s.kpad;
  const long long t = s.t0 + fi;
  const long long slot = t % s.cap;
  for (int c = tid; c < k; c += blockDim.x) as[c] = s.a[(size_t)fi * k + c];
  __syncthreads();
  // S~_q(t) in FP64 (k terms), and max |a_t| (the bits of non-negative floats order as
  // the values)
  double d = 0.0;
  unsigned amax = 0u;
  for (int c = tid; c < k; c += blockDim.x) {
    d = fma((double)as[c], s.s64[(size_t)q * k + c], d);
    amax = max(amax, __float_as_uint(fabsf(as[c])));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  amax = __reduce_max_sync(0xffffffffu, amax);
  if ((tid & 31) == 0) {
    dred[tid >> 5] = d;
    mred[tid >> 5] = amax;
  }
  __syncthreads();
  int e2 = 0;  // f16 history rows: 2^e2 a_t
  if (s.sp) {
    unsigned mb = mred[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) mb = max(mb, mred[w]);
    const float am = __uint_as_float(mb);
    if (am > 0.f && isfinite(am)) {
      int ex;
      frexpf(am, &ex);  // am in [2^(ex-1), 2^ex)
      e2 = min(64, max(-64, 14 - ex));
    }
  }
  double Sd = dred[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) Sd += dred[w];  // warps past the k terms add zeros
  const double S = s.Sx ? (double)s.Sx[(size_t)fi * s.n_q + q] : Sd;
  const float r = S > 0.0 ? (float)(sqrt((double)s.Mq[q]) / S) : 0.f;
  const int npad = stream_npad(s.n_q);
  if (tid == 0) {
    const float rs = s.sp ? ldexpf(r, -e2) : r;
    s.Rh[slot * npad + q] = rs;
    if (slot < 128) s.Rh[(s.cap + slot) * npad + q] = rs;
    // validity bit of (q, slot), and of its mirror slot; other frames of the step may
    // touch the same words
    unsigned long long* vb = s.vbits + (size_t)q * s.vwords;
    for (long long sl = slot; sl >= 0; sl = (sl == slot && slot < 128) ? s.cap + slot : -1) {
      const unsigned long long bit = 1ull << (sl & 63);
      if (r > 0.f)
        atomicOr(vb + (sl >> 6), bit);
      else
        atomicAnd(vb + (sl >> 6), ~bit);
    }
  }
  // the w row: pair order for the row update kernel, or row t mod 128 of the ring's block
  // for the two-time kernel (its other rows are zero, so only the step's frames count)
  const bool gram = s.b >= STREAM_GRAM_MIN;
  __nv_bfloat16* wrow = gram ? s.Wg + ((size_t)q * 128 + (t & 127)) * 2 * kp
                             : s.W2 + (size_t)w2_pair_row(fi, q, s.b, s.n_q) * 2 * kp;
  const float* Gq = s.G32 + (size_t)q * k * k;
  const int jt = SPLIT == 1 ? tid : tid & 127, ks = SPLIT == 1 ? 0 : tid >> 7;  // column thread, k split
  const int c_lo = SPLIT == 1 ? 0 : ks * k / SPLIT, c_hi = SPLIT == 1 ? k : (ks + 1) * k / SPLIT;
  for (int j = jt; j < kp; j += 128) {
    float v = 0.f;
    if (j < k && r > 0.f) {
      float v4[4] = {0.f, 0.f, 0.f, 0.f};
      int c = c_lo;
      // 32 loads of G_q in flight at a time (a one-frame step has only n_q blocks); chain
      // u takes rows u, u + 4, u + 8, ... of the split in order
      for (; c + 32 <= c_hi; c += 32) {
        float g[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) g[u] = Gq[(size_t)(c + u) * k + j];
#pragma unroll
        for (int u = 0; u < 32; ++u) v4[u & 3] = fmaf(as[c + u], g[u], v4[u & 3]);
      }
      for (; c + 4 <= c_hi; c += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) v4[u] = fmaf(as[c + u], Gq[(size_t)(c + u) * k + j], v4[u]);
      }
      for (; c < c_hi; ++c) v4[0] = fmaf(as[c], Gq[(size_t)c * k + j], v4[0]);
      v = (v4[0] + v4[1]) + (v4[2] + v4[3]);
    }
    if (SPLIT > 1) {
      vpart[ks][j] = v;
      continue;
    }
    v *= r;
    if (s.sp) {
      reinterpret_cast<__half*>(wrow)[j] = __float2half_rn(v);
    } else {
      __nv_bfloat16 hi, lo;
      split_bf16(v, hi, lo);
      wrow[j] = hi;
      wrow[kp + j] = lo;
    }
  }
  if (SPLIT > 1) {
    __syncthreads();
    for (int j = tid; j < kp; j += blockDim.x) {
      float v = 0.f;
      if (j < k && r > 0.f) {
        v = vpart[0][j];
#pragma unroll
        for (int u = 1; u < SPLIT; ++u) v += vpart[u][j];
        v *= r;
      }
      if (s.sp) {
        reinterpret_cast<__half*>(wrow)[j] = __float2half_rn(v);
      } else {
        __nv_bfloat16 hi, lo;
        split_bf16(v, hi, lo);
        wrow[j] = hi;
        wrow[kp + j] = lo;
      }
    }
  }
  if (q == 0 && s.sp) {
    __half* arow = reinterpret_cast<__half*>(s.A2 + (size_t)slot * 2 * kp);
    __half* mrow = slot < 128 ? reinterpret_cast<__half*>(s.A2 + (size_t)(s.cap + slot) * 2 * kp) : nullptr;
    for (int c = tid; c < kp; c += blockDim.x) {
      const __half x = __float2half_rn(c < k ? ldexpf(as[c], e2) : 0.f);
      arow[c] = x;
      if (mrow) mrow[c] = x;
    }
  } else if (q == 0) {
    __nv_bfloat16* arow = s.A2 + (size_t)slot * 2 * kp;
    __nv_bfloat16* mrow = slot < 128 ? s.A2 + (size_t)(s.cap + slot) * 2 * kp : nullptr;
    for (int c = tid; c < kp; c += blockDim.x) {
      __nv_bfloat16 hi, lo;
      split_bf16(c < k ? as[c] : 0.f, hi, lo);
      arow[c] = hi;
      arow[kp + c] = lo;
      if (mrow) {
        mrow[c] = hi;
        mrow[kp + c] = lo;
      }
    }
  }
}

__global__ void __launch_bounds__(128) frame_factors_kernel(const StreamStep s) { frame_factors<1>(s); }
__global__ void __launch_bounds__(512, 1) frame_factors_split_kernel(const StreamStep s) { frame_factors<4>(s); }

// After a step on the two-time kernel: lag tau = 128 d + e gets slot 128 + e of tile
// diagonal d and slot e of tile diagonal d + 1 (TwoSum into the f32-pair sums), its pair
// count from the validity bits of the step's frames and of the frames tau earlier, and the
// step's w rows are cleared (the next step of the block must not see them).
__global__ void stream_fold_kernel(const StreamStep s, int nd_step) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long span = s.W > s.b ? s.W : s.b;
  if (i >= (long long)s.n_q * span) return;
  const int q = (int)(i / span);
  const long long tau = i - (long long)q * span;
  if (tau < s.W) {
    const int d = (int)(tau >> 7), e = (int)(tau & 127);
    float sum = 0.f;
    if (d < nd_step) sum += s.gpart[((size_t)q * s.nd + d) * DIAG_SLOTS + TILE + e];
    if (d + 1 < nd_step) sum += s.gpart[((size_t)q * s.nd + d + 1) * DIAG_SLOTS + e];
    // pairs (t0 + f, t0 + f - tau), f < b, both frames defined and t0 + f - tau >= 0
    const unsigned long long* vb = s.vbits + (size_t)q * s.vwords;
    const long long f0 = tau > s.t0 ? tau - s.t0 : 0;  // first frame with a partner
    long long n = 0;
    for (long long f = f0; f < s.b; f += 64) {  // up to 128 frames: two 64-bit windows
      const int nf = (int)min(64LL, s.b - f);
      const unsigned long long a = vbits_window(vb, (s.t0 + f) % s.cap, nf);
      const unsigned long long h = vbits_window(vb, (s.t0 + f - tau) % s.cap, nf);
      n += __popcll(a & h);
    }
    const size_t j = (size_t)q * s.Wp + tau;
    if (sum != 0.f) s.g2sum[j] = f32pair_add(s.g2sum[j], sum);
    s.cnt[j] += n;
  }
  if (tau < s.b) {  // clear w row (q, t0 + tau) of the block: 2 kpad bf16, 16 bytes at a time
    uint4* row = reinterpret_cast<uint4*>(s.Wg + ((size_t)q * 128 + ((s.t0 + tau) & 127)) * 2 * s.kpad);
    for (int c = 0; c < s.kpad / 4; ++c) row[c] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// Deferred pair counts of count block [t0, t0 + 64) (the frames of `mask`) for the lags of
// the parts not in `done` (part j: lags j L .. j L + L - 1, L = ceil(W / 64)): thread =
// (ring, lag).
__global__ void count_flush_kernel(const unsigned long long* vbits, long long vwords, long long cap, int n_q,
                                   long long W, long long Wp, long long* cnt, long long t0, unsigned long long mask,
                                   unsigned long long done) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n_q * W) return;
  const int q = (int)(i / W);
  const long long tau = i - (long long)q * W;
  if ((done >> (tau / cf_part_len(W))) & 1ull) return;
  const long long n = masked_pair_count(vbits + (size_t)q * vwords, cap, t0, mask, tau);
  if (n) cnt[(size_t)q * Wp + tau] += n;
}

// g2 = (hi + lo) / count of each lag bin (f32 pair sums, added in FP64); NaN without pairs
__global__ void stream_g2_kernel(const float2* g2sum, const long long* cnt, int n_q, long long W, long long Wp,
                                 double* g2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n_q * W) return;
  const long long j = i / W * Wp + i % W;
  const float2 v = g2sum[j];
  g2[i] = cnt[j] > 0 ? ((double)v.x + (double)v.y) / (double)cnt[j] : __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void basis_f32_kernel(const double* B, long long n, float* B32) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    B32[i] = (float)B[i];
}

}  // namespace

bool stream_step_row1(const StreamStep& s) {
  const int n_kc = s.kpad / 64;
  return s.b == 1 && s.n_q <= 36 && s.tmW48 && n_kc <= (s.sp ? 4 : 2) &&
         row1_tc_smem(n_kc, stream_npad(s.n_q), s.sp, 0, std::min(36, s.n_q)) <= 227 * 1024;
}

cudaError_t launch_count_flush(const unsigned long long* vbits, long long vwords, long long cap, int n_q,
                               long long W, long long Wp, long long* cnt, long long t0, unsigned long long mask,
                               unsigned long long done, cudaStream_t st) {
  if (!mask || done == ~0ull) return cudaSuccess;
  const long long n = (long long)n_q * W;
  count_flush_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(vbits, vwords, cap, n_q, W, Wp, cnt, t0, mask,
                                                                  done);
  return cudaGetLastError();
}

cudaError_t launch_stream_step(const StreamStep& s, cudaStream_t st) {
  // the pair-ordered w rows of this step must fit the W2 allocation
  if (s.b < 1 || s.b > 128 ||
      (s.b < STREAM_GRAM_MIN && (long long)((s.n_q + 35) / 36) * w2_mtiles(s.b, s.n_q) * 128 > s.w2_rows))
    return cudaErrorInvalidValue;
  if (s.Sx && s.n_q > SE_MAX_RINGS) return cudaErrorInvalidValue;
  cudaError_t e = s.Sx ? cudaMemsetAsync(s.Sx, 0, (size_t)s.b * s.n_q * sizeof(long long), st) : cudaSuccess;
  if (e != cudaSuccess) return e;
  // dependent launches: each kernel may start while the one ahead of it finishes
  if (!s.pre_encoded) {
    if ((e = launch_pdl(sparse_encode_kernel, dim3(s.nblk, s.b), dim3(256), 0, st, s)) != cudaSuccess) return e;
    // with k a multiple of 4 the sparse encode's last slice block of a frame adds the
    // partials itself
    if ((s.k & 3) &&
        (e = launch_pdl(stream_reduce_kernel, dim3((s.b * s.k + 31) / 32), dim3(256), 0, st, s)) != cudaSuccess)
      return e;
  }
  if ((e = s.b == 1 ? launch_pdl(frame_factors_split_kernel, dim3(s.b, s.n_q), dim3(512), 0, st, s)
                     : launch_pdl(frame_factors_kernel, dim3(s.b, s.n_q), dim3(128), 0, st, s)) != cudaSuccess)
    return e;
  if (s.b >= STREAM_GRAM_MIN) {
    // the two-time kernel on (history block J - delta, the step's block J) tiles of every
    // ring: L = the coefficient history (shared by the rings), R = the block's w rows of
    // ring q (scaled by r_q(t); zero for frames outside the step), row scale r_q(s); the
    // diagonal sums then go into the running lag sums
    if (s.cap % 128 || ((s.t0 & 127) + s.b) > 128) return cudaErrorInvalidValue;
    const int nb = (int)(s.cap / 128);
    const int nd_step = (int)std::min<long long>(s.nd, (s.t0 >> 7) + 1);
    GramParams gp{};
    gp.T = (int)s.cap;
    gp.nT = s.nd;  // partials [n_q][nd][1][256]
    gp.T_pad = 0;
    gp.maxC = 1;
    gp.CH = nb + 1;  // chunk index I / CH = 0
    // ring pairs: one N = 256 MMA per K step covers rings q and q + 1 against one history
    // chunk (the w blocks of neighbouring rings are consecutive rows; a last odd ring runs
    // alone, N = 128)
    const int pairs = 1;
    gp.pairs = pairs;
    gp.sm_nq = s.n_q;
    gp.n_items = (s.n_q + 1) / 2 * nd_step;
    gp.items = nullptr;
    gp.ring_nb = nb;
    gp.ring_nd = nd_step;
    gp.ring_J = (int)((s.t0 >> 7) % nb);
    gp.sm = 1;
    gp.sm_nk = s.kpad / 64;
    gp.sm_c0 = (int)(s.t0 & 127);
    gp.sm_c1 = gp.sm_c0 + s.b;
    gp.r_ld = stream_npad(s.n_q);
    gp.fmt = s.sp ? 0 : 1;  // f16 rows (one product) or bf16 hi | lo pieces (three)
    gp.split = s.sp ? 0 : 1;
    gp.raw = 1;  // epilogue scales: r_q(s) for the history rows, the mask for the columns
    gp.r = s.Rh;
    gp.partials = s.gpart;
    gp.status = s.status;
    e = launch_gram(*s.tmA, *s.tmWg2, gp, std::min(gp.n_items, s.num_sms), st);
    if (e != cudaSuccess) return e;
    const long long span = std::max<long long>(s.W, s.b);
    stream_fold_kernel<<<(unsigned)((s.n_q * span + 255) / 256), 256, 0, st>>>(s, nd_step);
    return cudaGetLastError();
  }
  if (stream_step_row1(s)) {
    // one frame: the persistent single-frame kernel (lag tiles of 128, direct fold; its
    // pair count is deferred to its count block, and it adds one part of the deferred
    // counts of the block before)
    Row1Params p1{};
    p1.t = s.t0;
    p1.W = s.W;
    p1.cap = s.cap;
    p1.n_q = s.n_q;
    p1.kpad = s.kpad;
    p1.n_kc = s.kpad / 64;
    p1.npad = stream_npad(s.n_q);
    p1.qb = p1.npad;
    p1.n_tiles = (int)((std::min<long long>(s.W, s.t0 + 1) + 127) / 128);
    p1.Wp = s.Wp;
    p1.sp = s.sp;
    p1.qg2 = std::min(36, s.n_q);
    // the tiles' g2 sums staged in shared memory in as many slices (two, one) as fit
    p1.sb = row1_tc_smem(p1.n_kc, p1.qb, s.sp, 2, p1.qg2) <= 227 * 1024   ? 2
            : row1_tc_smem(p1.n_kc, p1.qb, s.sp, 1, p1.qg2) <= 227 * 1024 ? 1
                                                                            : 0;
    p1.Rh = s.Rh;
    p1.g2sum = s.g2sum;
    p1.cnt = s.cnt;
    p1.vbits = s.vbits;
    p1.vwords = s.vwords;
    p1.cf_t0 = s.cf_t0;
    p1.cf_mask = s.cf_mask;
    p1.cf_tau0 = s.cf_tau0;
    p1.cf_tau1 = s.cf_tau1;
    p1.status = s.status;
    return launch_row1_tc(*s.tmA, *s.tmW48, *s.tmR, s.tmG[rt_lt_index(128)], p1, std::min(p1.n_tiles, s.num_sms),
                          st);
  }
  // row update of the step (at most 64 frames: every pair of a lag tile then lies in
  // one 128-row history operand)
  RowTcParams p{};
  p.t0 = s.t0;
  p.b = s.b;
  p.W = s.W;
  p.cap = s.cap;
  p.n_q = s.n_q;
  p.kpad = s.kpad;
  p.n_kc = s.kpad / 64;
  if (!row_update_config(s.n_q, s.kpad, s.b, &p.lt, &p.wst, &p.epi)) return cudaErrorInvalidConfiguration;
  const int li = rt_lt_index(p.lt);
  // lags up to the window, and no further than the step's last frame: a pair (t, t - tau)
  // of this step exists only for tau <= t0 + b - 1, so a young history skips the rest
  p.n_tiles = (int)((std::min<long long>(s.W, s.t0 + s.b) + p.lt - 1) / p.lt);
  p.n_rg = (s.n_q + 35) / 36;
  p.n_mt = w2_mtiles(s.b, s.n_q);
  p.nfb = (s.b + 31) / 32;
  p.npad = stream_npad(s.n_q);
  p.qb = std::min(36, p.npad);
  p.Rh = s.Rh;
  p.vbits = s.vbits;
  p.vwords = s.vwords;
  p.Wp = s.Wp;
  p.qg2 = std::min(36, s.n_q);
  p.sp = s.sp;
  p.status = s.status;
  const int grid = std::min(p.n_tiles * p.n_rg, s.num_sms);
  return launch_row_update_tc(*s.tmA, *s.tmW, *s.tmR, s.tmG[li], s.tmC[li], p, grid, st);
}

// Longest lag tile whose history rows fit one operand and whose layout fits shared memory.
// Steps of at most W2_SMALL_B frames take the small-step epilogue (no diagonal buffers);
// larger steps prefer the skewed-buffer epilogue, then two w stages.
bool row_update_config(int n_q, int kpad, int b, int* lt, int* wst, int* epi) {
  const int n_kc = kpad / 64, qb = std::min(36, stream_npad(n_q)), qg2 = std::min(36, n_q);
  const int small_modes[2][2] = {{2, 2}, {1, 2}};  // {wst, epi}
  const int large_modes[4][2] = {{2, 1}, {1, 1}, {2, 0}, {1, 0}};
  for (int i = 0; i < RT_N_LT; ++i) {
    const int l = RT_LTS[i];
    if (l + b - 1 > 128) continue;
    const int n_modes = b <= W2_SMALL_B ? 2 : 4;
    for (int m = 0; m < n_modes; ++m) {
      const int* c = b <= W2_SMALL_B ? small_modes[m] : large_modes[m];
      if (row_update_tc_smem(n_kc, l, qb, c[0], qg2, c[1]) <= 227 * 1024) {
        *lt = l;
        *wst = c[0];
        *epi = c[1];
        return true;
      }
    }
  }
  return false;
}

}  // namespace xpcs

extern "C" xpcs_status xpcs_stream_row_tile(int n_q, int k, int b, int* lags, int* w_stages, int* epilogue,
                                            int* smem_bytes) {
  if (n_q < 1 || n_q > 1024 || k < 1 || k > 256 || b < 1 || b > 64) return XPCS_EINVAL;
  const int kpad = (k + 63) / 64 * 64;
  if (b >= xpcs::STREAM_GRAM_MIN) {  // the two-time kernel on 128-frame blocks
    if (lags) *lags = 128;
    if (w_stages) *w_stages = 0;
    if (epilogue) *epilogue = 3;
    if (smem_bytes) *smem_bytes = xpcs::gram_smem_bytes();
    return XPCS_OK;
  }
  int lt = 0, wst = 0, epi = 0;
  if (!xpcs::row_update_config(n_q, kpad, b, &lt, &wst, &epi)) return XPCS_ENOTSUP;
  if (lags) *lags = lt;
  if (w_stages) *w_stages = wst;
  if (epilogue) *epilogue = epi;
  if (smem_bytes)
    *smem_bytes = xpcs::row_update_tc_smem(kpad / 64, lt, std::min(36, xpcs::stream_npad(n_q)), wst,
                                           std::min(36, n_q), epi);
  return XPCS_OK;
}

namespace xpcs {

cudaError_t launch_stream_g2(const float2* g2sum, const long long* cnt, int n_q, long long W, long long Wp,
                             double* g2, cudaStream_t st) {
  const long long n = (long long)n_q * W;
  stream_g2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g2sum, cnt, n_q, W, Wp, g2);
  return cudaGetLastError();
}

cudaError_t launch_basis_f32(const double* B, long long n, float* B32, cudaStream_t st) {
  basis_f32_kernel<<<1024, 256, 0, st>>>(B, n, B32);
  return cudaGetLastError();
}

}  // namespace xpcs
