// Ingest, per-frame normalisation factors, operand preparation, pair counts and the g2
// reductions (sm_103a).
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace xpcs {

namespace {


// ---------------------------------------------------------------- raw ingest (ring sums)
// Grid (position chunks of RI_CHUNK ring-sorted positions, groups of RI_F frames).  A CTA
// stages its chunk of the position -> pixel map in shared memory once, then for each of
// its frames gathers the counts into ring-sorted order as bf16 (exact for counts <= 256),
// written as coalesced rows of the operand, and accumulates S_q(t) = sum of counts and the
// sum of squares per ring (Eq. 1 denominators and the exactness bound of the f32 Gram).
// Ring segments start at multiples of 64 positions, so each 64-position group belongs to
// one ring (or its padding): the warp that gathers a group reduces it with shuffles, and at
// the end the CTA adds its groups ring by ring into S and S2 with one 64-bit atomic per
// (ring, frame) it touched (the launch zeroes S and S2).  A warp issues all its gathers of
// a frame (16 per thread) before using any of them.
constexpr int RI_CHUNK = 4096;            // positions per CTA (a multiple of 64)
constexpr int RI_GROUPS = RI_CHUNK / 64;  // 64-position groups per chunk
constexpr int RI_F = 8;                   // frames per CTA
constexpr int RI_J = RI_GROUPS / 8;       // groups per warp (8 warps)

template <int DT>
__global__ void __launch_bounds__(256) raw_ingest_kernel(const RawIngestParams p) {
  __shared__ __align__(16) int sperm[RI_CHUNK];
  __shared__ int sring[RI_GROUPS];
  __shared__ unsigned long long gsum[RI_F][RI_GROUPS];
  __shared__ unsigned long long gsq[RI_F][RI_GROUPS];
  const long long P0 = (long long)blockIdx.x * RI_CHUNK;
  const long long t0 = (long long)blockIdx.y * RI_F;
  const int npos = (int)min((long long)RI_CHUNK, p.Mp - P0);  // a multiple of 64
  const int ngrp = npos / 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < RI_CHUNK; i += blockDim.x) sperm[i] = i < npos ? p.perm[P0 + i] : -1;
  for (int g = threadIdx.x; g < RI_GROUPS; g += blockDim.x) sring[g] = g < ngrp ? p.pos_ring[P0 + 64 * g] : -1;
  __syncthreads();
  bool too_big = false;
  for (int f = 0; f < RI_F; ++f) {
    const long long t = t0 + f;
    if (t >= p.T_pad) break;  // CTA-uniform
    const bool live = t < p.T;
    using Tx = typename std::conditional<DT == 0, uint8_t, uint16_t>::type;
    const Tx* xr = static_cast<const Tx*>(p.X) + t * p.M;
    unsigned a[RI_J], b[RI_J];
#pragma unroll
    for (int j = 0; j < RI_J; ++j) {
      const int o = 64 * (warp + 8 * j) + 2 * lane;
      // the pair of map entries in one 8-byte load (no bank conflicts); -1 for padding and
      // past the chunk
      const int2 sp = *reinterpret_cast<const int2*>(sperm + o);
      a[j] = (live && sp.x >= 0) ? (unsigned)xr[sp.x] : 0u;
      b[j] = (live && sp.y >= 0) ? (unsigned)xr[sp.y] : 0u;
    }
#pragma unroll
    for (int j = 0; j < RI_J; ++j) {
      const int g = warp + 8 * j;
      if (g >= ngrp) break;  // warp-uniform
      const int o = 64 * g + 2 * lane;
      const bool big = (a[j] > 256u) | (b[j] > 256u);
      too_big |= big;
      if (p.Xp) {
        const __nv_bfloat162 v = __floats2bfloat162_rn((float)a[j], (float)b[j]);
        *reinterpret_cast<__nv_bfloat162*>(p.Xp + (p.xp_row0 + t) * p.Mp + P0 + o) = v;
      }
      unsigned long long s1, s2;
      if (!__any_sync(0xffffffffu, big)) {  // squares < 2^17 per lane: 32-bit sums are exact
        s1 = __reduce_add_sync(0xffffffffu, a[j] + b[j]);
        s2 = __reduce_add_sync(0xffffffffu, a[j] * a[j] + b[j] * b[j]);
      } else {
        s1 = (unsigned long long)a[j] + b[j];
        s2 = (unsigned long long)a[j] * a[j] + (unsigned long long)b[j] * b[j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          s1 += __shfl_xor_sync(0xffffffffu, s1, off);
          s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        }
      }
      if (lane == 0) {
        gsum[f][g] = s1;
        gsq[f][g] = s2;
      }
    }
  }
  if (too_big && p.Xp) set_status(p.status, XPCS_DEV_RANGE);
  __syncthreads();
  // groups of one ring are consecutive: one thread per frame walks the chunk's groups and
  // adds each ring's run into S (and S2)
  if (threadIdx.x < RI_F) {
    const int f = threadIdx.x;
    const long long t = t0 + f;
    if (t < p.T) {
      int q = -1;
      unsigned long long r1 = 0, r2 = 0;
      for (int g = 0; g <= ngrp; ++g) {
        const int qg = g < ngrp ? sring[g] : -2;
        if (qg != q) {
          if (q >= 0 && (r1 | r2)) {
            atomicAdd(reinterpret_cast<unsigned long long*>(p.S + (size_t)q * p.T + t), r1);
            if (p.S2) atomicAdd(reinterpret_cast<unsigned long long*>(p.S2 + (size_t)q * p.T + t), r2);
          }
          q = qg;
          r1 = r2 = 0;
        }
        if (g < ngrp && q >= 0) {
          r1 += gsum[f][g];
          r2 += gsq[f][g];
        }
      }
    }
  }
}

// Per-frame operand scale r[q][t], so that C = r(t1) r(t2) N(t1,t2):
//   XPCS_NORM_MEAN  r = sqrt(M_q) / S_q(t)          (Eq. 1), undefined if S_q(t) <= 0
//   XPCS_NORM_FROB  r = 1 / sqrt(sum_p x_{t,p}^2)   (Eq. 2 with Frobenius rows), undefined if 0
//   XPCS_NORM_EQ12  r = sqrt(M_q) / mean_t S_q(t)   (Eq. 12), every frame defined
// Undefined frames get r = 0; blk_bad marks tiles with an undefined frame.
__global__ void raw_scales_kernel(const long long* S, const long long* S2, const double* Sbar, int norm,
                                  const long long* Mq, int n_q, long long T, int T_pad, int nT, float* r,
                                  uint32_t* blk_bad, uint32_t* status) {
  const int q = blockIdx.y, I = blockIdx.x;
  const long long t = (long long)I * TILE + threadIdx.x;
  float v = 0.f;
  bool bad = false;
  // the exactness bound of the f32 Gram: every frame's sum of squares below 2^24
  if (t < T && S2[(size_t)q * T + t] >= (1ll << 24)) set_status(status, XPCS_DEV_RANGE);
  if (t < T) {
    double den;
    if (norm == XPCS_NORM_FROB)
      den = sqrt((double)S2[(size_t)q * T + t]);
    else if (norm == XPCS_NORM_EQ12)
      den = Sbar[q] / sqrt((double)Mq[q]);
    else
      den = (double)S[(size_t)q * T + t] / sqrt((double)Mq[q]);
    if (den > 0.0)
      v = (float)(1.0 / den);
    else
      bad = true;
  }
  r[(size_t)q * T_pad + t] = v;
  const int any = __syncthreads_or(bad);
  if (threadIdx.x == 0) blk_bad[(size_t)q * nT + I] = (uint32_t)any;
}

// Sbar[q] = mean over the T frames of the raw ring sums S_q(t) (FP64, fixed order).
__global__ void __launch_bounds__(256) ring_mean_kernel(const long long* S, long long T, double* Sbar) {
  __shared__ double red[256];
  const int q = blockIdx.x;
  long long acc = 0;  // exact: at most T * M_q * 65535 < 2^63
  for (long long t = threadIdx.x; t < T; t += blockDim.x) acc += S[(size_t)q * T + t];
  red[threadIdx.x] = (double)acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) Sbar[q] = red[0] / (double)T;
}

// Compressed Eq. 12 denominator: S~bar_q = mean_t a_t . s_q = abar . s_q (the ring sum is
// linear in the coefficients), abar = column means of A in FP64.  One block.
__global__ void __launch_bounds__(256) coef_mean_kernel(const float* A, long long T, int k, const double* s64,
                                                        int n_q, double* Sbar) {
  __shared__ double abar[256];
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    double acc = 0.0;
    for (long long t = 0; t < T; ++t) acc += (double)A[t * k + c];
    abar[c] = acc / (double)T;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n_q; q += blockDim.x) {
    double d = 0.0;
    for (int c = 0; c < k; ++c) d += abar[c] * s64[(size_t)q * k + c];
    Sbar[q] = d;
  }
}

// ---------------------------------------------------------------- compressed preparation
template <typename T16>
XPCS_DEV T16 to16(float x);
template <>
XPCS_DEV __half to16<__half>(float x) { return __float2half_rn(x); }
template <>
XPCS_DEV __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

constexpr int PREP_FRAMES = 64;

// Operand rows for one ring and 64 frames: L = r * (a G_q), R = r * a, in the requested
// 16-bit format.  BF16X3 stores [hi | lo] pieces (each padded to a multiple of 64) for
// both, and the two-time kernel forms hi*hi + lo*hi + hi*lo.  W = a G_q is formed in shared
// memory (f32 FMA), then whole rows are written with coalesced 16-byte stores.
template <typename T16, bool SPLIT>
__global__ void __launch_bounds__(256) comp_operands_kernel(const PrepParams p) {
  extern __shared__ float sm[];
  const int k = p.k;
  const int lda = k + 1;
  float* As = sm;                          // [64][k+1]  a
  float* rs = As + PREP_FRAMES * lda;      // [64] r of this block's frames
  float* Ws = rs + PREP_FRAMES;            // [64][k+1]  a G_q
  float* Gs = Ws + PREP_FRAMES * lda;      // [k][64]
  const int q = blockIdx.y;
  const long long t0 = (long long)blockIdx.x * PREP_FRAMES;
  const int tid = threadIdx.x;
  // A rows: 4 rows per pass, 64 columns per row chunk (coalesced, no integer division)
  for (int f = tid >> 6; f < PREP_FRAMES; f += 4) {
    const long long t = t0 + f;
    for (int c = tid & 63; c < k; c += 64) As[f * lda + c] = (t < p.T) ? p.A[t * k + c] : 0.f;
  }
  __syncthreads();
  // ring sums of the decompressed frames S~_q(t) = a_t . s_q: 4 threads per frame, each a
  // compensated f32 dot product (TwoProduct by fma, TwoSum; Ogita, Rump and Oishi, 2005)
  // over a quarter of the coefficients, combined by shuffles with the same transformations.
  // The result carries about twice the f32 precision, so lossy sums near zero keep
  // their sign without the FP64 units.
  {
    const int f = tid >> 2, part = tid & 3;
    const float2* sq = p.s32 + (size_t)q * k;
    const float* arow = As + f * lda;
    float hi = 0.f, lo = 0.f;
    for (int c = part; c < k; c += 4) {
      const float2 sv = sq[c];
      const float x = arow[c];
      const float prod = x * sv.x;
      const float perr = fmaf(x, sv.x, -prod) + x * sv.y;
      const float sum = hi + prod;
      const float z = sum - hi;
      lo += ((hi - (sum - z)) + (prod - z)) + perr;
      hi = sum;
    }
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      const float ohi = __shfl_xor_sync(0xffffffffu, hi, off);
      const float olo = __shfl_xor_sync(0xffffffffu, lo, off);
      const float sum = hi + ohi;
      const float z = sum - hi;
      lo += ((hi - (sum - z)) + (ohi - z)) + olo;
      hi = sum;
    }
    if (part == 0) {
      const long long t = t0 + f;
      float v = 0.f;
      if (t < p.T) {
        // the ring sum of the denominators: a_t s_q (hi + lo; hi alone decides the sign),
        // or the raw frame's exact sum
        const long long* se = p.S_exact ? p.S_exact + (size_t)q * p.T + t : nullptr;
        if (p.St) p.St[(size_t)q * p.T + t] = se ? (double)*se : (double)hi + (double)lo;
        // per-frame scale (xpcs_norm) in f32, the FP64 units being slow on this part (the
        // scale is a float either way); the Frobenius one needs W and is set below
        const float den = p.norm == XPCS_NORM_EQ12 ? (float)p.Sbar[q] : se ? (float)*se : hi + lo;
        if (p.norm != XPCS_NORM_FROB) {
          if (den > 0.f)
            v = sqrtf((float)p.Mq[q]) / den;
          else
            atomicOr(&p.blk_bad[(size_t)q * p.nT + (t >> 7)], 1u);
        }
      }
      if (p.norm != XPCS_NORM_FROB) p.r[(size_t)q * p.T_pad + t] = v;
      rs[f] = v;
    }
  }
  // W = a G_q in 64-column chunks (the scale r is applied when the rows are written):
  // thread (fl, cg) computes frames fl and fl + 32,
  // columns 8 cg .. 8 cg + 7 of the chunk (16 outputs, 4 shared loads per 16 FMAs)
  const int fl = tid & 31, cg = tid >> 5;
  const float* Gq = p.G32 + (size_t)q * k * k;
  for (int j0 = 0; j0 < k; j0 += 64) {
    const int nc = min(64, k - j0);
    __syncthreads();
    for (int c = tid >> 6; c < k; c += 4) {
      const int j = tid & 63;
      Gs[c * 64 + j] = (j < nc) ? Gq[(size_t)c * k + j0 + j] : 0.f;
    }
    __syncthreads();
    float w0[8], w1[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) w0[u] = w1[u] = 0.f;
    const float* a0 = As + fl * lda;
    const float* a1 = As + (fl + 32) * lda;
#pragma unroll 4
    for (int c = 0; c < k; ++c) {
      const float x0 = a0[c], x1 = a1[c];
      const float4 g0 = *reinterpret_cast<const float4*>(Gs + c * 64 + 8 * cg);
      const float4 g1 = *reinterpret_cast<const float4*>(Gs + c * 64 + 8 * cg + 4);
      const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        w0[u] = fmaf(x0, gv[u], w0[u]);
        w1[u] = fmaf(x1, gv[u], w1[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (8 * cg + u < nc) {
        Ws[fl * lda + j0 + 8 * cg + u] = w0[u];
        Ws[(fl + 32) * lda + j0 + 8 * cg + u] = w1[u];
      }
  }
  __syncthreads();
  if (p.norm == XPCS_NORM_FROB) {
    // ||x~_t||^2 over the ring = a_t G_q a_t^T = W_t . a_t, compensated as the ring sums
    const int f = tid >> 2, part = tid & 3;
    const float* wrow = Ws + f * lda;
    const float* arow = As + f * lda;
    float hi = 0.f, lo = 0.f;
    for (int c = part; c < k; c += 4) {
      const float x = wrow[c], y = arow[c];
      const float prod = x * y;
      const float perr = fmaf(x, y, -prod);
      const float sum = hi + prod;
      const float z = sum - hi;
      lo += ((hi - (sum - z)) + (prod - z)) + perr;
      hi = sum;
    }
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      const float ohi = __shfl_xor_sync(0xffffffffu, hi, off);
      const float olo = __shfl_xor_sync(0xffffffffu, lo, off);
      const float sum = hi + ohi;
      const float z = sum - hi;
      lo += ((hi - (sum - z)) + (ohi - z)) + olo;
      hi = sum;
    }
    if (part == 0) {
      const long long t = t0 + f;
      float v = 0.f;
      if (t < p.T) {
        const double n = (double)hi + (double)lo;
        if (n > 0.0)
          v = (float)(1.0 / sqrt(n));
        else
          atomicOr(&p.blk_bad[(size_t)q * p.nT + (t >> 7)], 1u);
      }
      p.r[(size_t)q * p.T_pad + t] = v;
      rs[f] = v;
    }
    __syncthreads();
  }
  // rows out: 8 threads per row, 16-byte vectors, coalesced 128-byte segments
  const int nvec = p.Kc / 8;
  const int piece = SPLIT ? p.Kc / 2 : p.Kc;  // split rows are [hi | lo], each `piece` wide
  uint4* L = reinterpret_cast<uint4*>(static_cast<T16*>(p.L) + ((size_t)q * p.T_pad + t0) * p.Kc);
  uint4* R = reinterpret_cast<uint4*>(static_cast<T16*>(p.R) + ((size_t)q * p.T_pad + t0) * p.Kc);
  for (int ff = tid >> 3; ff < PREP_FRAMES; ff += 32) {
    const float* wrow = Ws + ff * lda;
    const float* arow = As + ff * lda;
    const float rf = rs[ff];
    for (int vv = tid & 7; vv < nvec; vv += 8) {
      // a vector never straddles the hi | lo boundary (piece is a multiple of 64)
      const bool lo = SPLIT && vv * 8 >= piece;
      const int jb = vv * 8 - (lo ? piece : 0);
      alignas(16) T16 lv[8];
      alignas(16) T16 rv[8];
      if (jb + 8 <= k) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float wv = rf * wrow[jb + e], av = rf * arow[jb + e];
          if (!lo) {
            lv[e] = to16<T16>(wv);
            rv[e] = to16<T16>(av);
          } else {
            lv[e] = to16<T16>(wv - (float)to16<T16>(wv));
            rv[e] = to16<T16>(av - (float)to16<T16>(av));
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int j = jb + e;
          const float wv = j < k ? rf * wrow[j] : 0.f, av = j < k ? rf * arow[j] : 0.f;
          if (!lo) {
            lv[e] = to16<T16>(wv);
            rv[e] = to16<T16>(av);
          } else {
            lv[e] = to16<T16>(wv - (float)to16<T16>(wv));
            rv[e] = to16<T16>(av - (float)to16<T16>(av));
          }
        }
      }
      L[(size_t)ff * nvec + vv] = *reinterpret_cast<const uint4*>(lv);
      R[(size_t)ff * nvec + vv] = *reinterpret_cast<const uint4*>(rv);
    }
  }
}

// ---------------------------------------------------------------- tensor-core operand pieces
// Ring sums, scales and R rows of the tensor-core path (L comes from ring_w_tc_kernel;
// not the Frobenius normalisation): a block takes 128 frames and SR_QG rings.  The frames'
// coefficient rows are loaded into shared memory once for all its rings (row pitch = k
// rounded up to 32, plus 2, so the two threads of a frame read distinct banks).  Two
// threads per frame form the compensated ring sum a_t s_q (as in comp_operands_kernel,
// each over every other coefficient, the halves combined in a fixed order so both hold
// the same value), the scale r in f32 (the FP64 units are slow on this part), and write
// the frame's R row (16-byte vectors, the two threads alternating).
constexpr int SR_FRAMES = 128, SR_QG = 4;
template <typename T16, bool SPLIT>
__global__ void __launch_bounds__(256) scales_rows_kernel(const PrepParams p, int lda, int vec) {
  extern __shared__ float sm[];
  const int k = p.k;
  float* As = sm;                                                   // [128][lda]
  float2* Ss = reinterpret_cast<float2*>(As + SR_FRAMES * lda);     // [SR_QG][k]
  const long long t0 = (long long)blockIdx.x * SR_FRAMES;
  const int q0 = blockIdx.y * SR_QG;
  const int qn = min(SR_QG, p.n_q - q0);
  const int tid = threadIdx.x;
  // the tile's rows are 128 k consecutive floats of A (zeros past frame T): 16-byte loads,
  // eight per thread in flight before any is stored, when k is a multiple of 4
  const long long have = (p.T - t0) * k;  // floats of the tile that exist
  if (vec) {
    const float4* A4 = reinterpret_cast<const float4*>(p.A + t0 * k);
    const int n4 = SR_FRAMES * k / 4;
    for (int e0 = tid; e0 < n4; e0 += 8 * 256) {
      float4 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e4 = e0 + u * 256;
        x[u] = (e4 < n4 && 4ll * e4 < have) ? __ldg(A4 + e4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e4 = e0 + u * 256;
        if (e4 < n4) {
          const int f = 4 * e4 / k, c = 4 * e4 - f * k;
          float* d = As + f * lda + c;
          d[0] = x[u].x;
          d[1] = x[u].y;
          d[2] = x[u].z;
          d[3] = x[u].w;
        }
      }
    }
  } else {
    for (int f = tid >> 6; f < SR_FRAMES; f += 4) {
      const long long t = t0 + f;
      for (int c = tid & 63; c < k; c += 64) As[f * lda + c] = (t < p.T) ? p.A[t * k + c] : 0.f;
    }
  }
  for (int e = tid; e < qn * k; e += 256) Ss[e] = p.s32[(size_t)q0 * k + e];
  __syncthreads();
  const int f = tid >> 1, part = tid & 1;
  const long long t = t0 + f;
  const float* arow = As + f * lda;
  const int nvec = p.Kc / 8;                  // 16-byte vectors per row
  const int piece = SPLIT ? p.Kc / 2 : p.Kc;  // split rows are [hi | lo], each `piece` wide
  for (int qi = 0; qi < qn; ++qi) {
    const int q = q0 + qi;
    const float2* sq = Ss + qi * k;
    float hi = 0.f, lo = 0.f;
    for (int c = part; c < k; c += 2) {  // TwoProduct by fma, TwoSum (Ogita, Rump and Oishi)
      const float2 sv = sq[c];
      const float x = arow[c];
      const float prod = x * sv.x;
      const float perr = fmaf(x, sv.x, -prod) + x * sv.y;
      const float sum = hi + prod;
      const float z = sum - hi;
      lo += ((hi - (sum - z)) + (prod - z)) + perr;
      hi = sum;
    }
    {  // both threads combine (half 0, half 1) in the same order
      const float ohi = __shfl_xor_sync(0xffffffffu, hi, 1), olo = __shfl_xor_sync(0xffffffffu, lo, 1);
      const float a = part ? ohi : hi, b = part ? hi : ohi;
      const float la = part ? olo : lo, lb = part ? lo : olo;
      const float sum = a + b;
      const float z = sum - a;
      lo = ((la + ((a - (sum - z)) + (b - z))) + lb);
      hi = sum;
    }
    float v = 0.f;
    if (t < p.T) {
      const long long* se = p.S_exact ? p.S_exact + (size_t)q * p.T + t : nullptr;
      if (p.St && part == 0) p.St[(size_t)q * p.T + t] = se ? (double)*se : (double)hi + (double)lo;
      const float den = p.norm == XPCS_NORM_EQ12 ? (float)p.Sbar[q] : se ? (float)*se : hi + lo;
      if (den > 0.f)
        v = sqrtf((float)p.Mq[q]) / den;
      else if (part == 0)
        atomicOr(&p.blk_bad[(size_t)q * p.nT + (t >> 7)], 1u);
    }
    if (part == 0) p.r[(size_t)q * p.T_pad + t] = v;
    uint4* R = reinterpret_cast<uint4*>(static_cast<T16*>(p.R) + ((size_t)q * p.T_pad + t) * p.Kc);
    for (int vv = part; vv < nvec; vv += 2) {
      // a vector never straddles the hi | lo boundary (piece is a multiple of 64)
      const bool lov = SPLIT && vv * 8 >= piece;
      const int jb = vv * 8 - (lov ? piece : 0);
      alignas(16) T16 rv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = jb + e;
        const float av = j < k ? v * arow[j] : 0.f;
        rv[e] = lov ? to16<T16>(av - (float)to16<T16>(av)) : to16<T16>(av);
      }
      R[vv] = *reinterpret_cast<const uint4*>(rv);
    }
  }
}

__global__ void coef_pieces_kernel(const float* A, long long T, int k, int kq, long long n, __nv_bfloat16* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long t = i / kq;
    const int c = (int)(i - t * kq);
    const float a = (t < T && c < k) ? A[t * k + c] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(a);
    out[t * 2 * kq + c] = hi;
    out[t * 2 * kq + kq + c] = __float2bfloat16_rn(a - __bfloat162float(hi));
  }
}

__global__ void gram_pieces_kernel(const double* G, int n_q, int k, int kq, __nv_bfloat16* out) {
  const long long n = (long long)n_q * kq * kq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / ((long long)kq * kq));
    const int rem = (int)(i - (long long)q * kq * kq);
    const int r = rem / kq, c = rem - r * kq;
    const double g = (r < k && c < k) ? G[((size_t)q * k + r) * k + c] : 0.0;
    const __nv_bfloat16 hi = __double2bfloat16(g);
    const size_t row = ((size_t)q * kq + r) * 2 * kq;
    out[row + c] = hi;
    out[row + kq + c] = __double2bfloat16(g - (double)__bfloat162float(hi));
  }
}

// ---------------------------------------------------------------- pair counts
// Validity bits of every ring (bit t: r_q(t) > 0), and ring_gap[q] != 0 when ring q has an
// undefined frame among t < T (ring_gap zeroed by the launcher).
__global__ void vbits_kernel(const float* r, int n_q, long long T, int T_pad, int words, uint32_t* vbits,
                             uint32_t* ring_gap) {
  const long long gw = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (gw >= (long long)n_q * words) return;
  const int q = (int)(gw / words), w = (int)(gw % words);
  const long long t = (long long)w * 32 + lane;
  const bool v = (t < T_pad) && r[(size_t)q * T_pad + t] > 0.f;
  const uint32_t m = __ballot_sync(0xffffffffu, v);
  const uint32_t real = __ballot_sync(0xffffffffu, t < T);  // frames of the series in this word
  if (lane == 0) {
    vbits[(size_t)q * words + w] = m;
    if ((m & real) != real) atomicOr(&ring_gap[q], 1u);
  }
}

// count_q(tau) = number of t with frames t and t+tau both defined (T - tau when every frame
// of the ring is defined).
__global__ void counts_kernel(const uint32_t* vbits, const uint32_t* ring_gap, int n_q, long long T, int words,
                              long long* count) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n_q * T) return;
  const int q = (int)(gid / T);
  const long long tau = gid % T;
  if (!ring_gap[q]) {
    count[gid] = T - tau;
    return;
  }
  const uint32_t* v = vbits + (size_t)q * words;
  const int ws = (int)(tau >> 5), s = (int)(tau & 31);
  long long c = 0;
  for (int w = 0; w + ws < words; ++w) {
    const uint32_t a = v[w + ws];
    const uint32_t b = (w + ws + 1 < words) ? v[w + ws + 1] : 0u;
    const uint32_t sh = s ? ((a >> s) | (b << (32 - s))) : a;
    c += __popc(v[w] & sh);
  }
  count[gid] = c;
}

// g2_q(tau) from the per-(ring, tile diagonal, chunk) diagonal partial sums.
__global__ void g2_finalize_kernel(const float* partials, const long long* count, int n_q, long long T, int nT,
                                   int maxC, int CH, double* g2) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n_q * T) return;
  const int q = (int)(gid / T);
  const long long tau = gid % T;
  const int d1 = (int)(tau / TILE), e1 = (int)(tau % TILE);
  // two independent chains of compensated f32 sums (hi + lo pairs by TwoSum: about twice
  // the f32 precision, no FP64 arithmetic, which is slow on this part), added in a fixed
  // order; one FP64 division per lag
  float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
  {
    const int nC = (nT - d1 + CH - 1) / CH;
    const float* base = partials + ((size_t)q * nT + d1) * maxC * DIAG_SLOTS;
    for (int c = 0; c < nC; ++c) s1 = f32pair_add(s1, base[(size_t)c * DIAG_SLOTS + TILE + e1]);
  }
  const int d2 = d1 + 1;
  if (d2 < nT) {
    const int nC = (nT - d2 + CH - 1) / CH;
    const float* base = partials + ((size_t)q * nT + d2) * maxC * DIAG_SLOTS;
    for (int c = 0; c < nC; ++c) s2 = f32pair_add(s2, base[(size_t)c * DIAG_SLOTS + e1]);
  }
  s1 = f32pair_add(f32pair_add(s1, s2.x), s2.y);
  const double sum = (double)s1.x + (double)s1.y;
  const long long n = count[gid];
  g2[gid] = n > 0 ? sum / (double)n : __longlong_as_double(0x7ff8000000000000ll);
}

// ---------------------------------------------------------------- g2 over a stored C
// C holds the lower triangle: C[s][s - tau] = C(s - tau, s) for tau >= 0.
// Grid (lag blocks of 128, rings, row splits); 8 warps.  Lane l of every warp owns lags
// L0 + l + 32 m (m = 0..3); the warp walks its rows s four at a time, reading
// C[s][s - L0 - 127 .. s - L0] as 128-byte coalesced segments (16 loads per thread in
// flight).  Undefined (NaN) entries are skipped and counted out.
constexpr int G2C_WARPS = 8;
__global__ void __launch_bounds__(256) g2_from_C_kernel(const float* __restrict__ C, int n_q, long long T,
                                                        double* partial, long long* cnt_partial, int row_splits) {
  __shared__ float ssum[G2C_WARPS][TILE];
  __shared__ int scnt[G2C_WARPS][TILE];
  const long long L0 = (long long)blockIdx.x * TILE;
  const int q = blockIdx.y, split = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nrows = T - L0;
  const long long per = (nrows + row_splits - 1) / row_splits;
  const long long r0 = L0 + (long long)split * per;
  const long long r1 = min(T, r0 + per);
  float s[4] = {0.f, 0.f, 0.f, 0.f};
  int c[4] = {0, 0, 0, 0};
  const float* Cq = C + (size_t)q * T * T;
  // four rows per warp step: their 16 loads per thread are all in flight before any is used
  for (long long row = r0 + 4 * warp; row < r1; row += 4 * G2C_WARPS) {
    float v[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long rr = row + i;
      const long long lim = rr - L0;                       // lags L0 + l with l <= lim
      const float* p = Cq + (size_t)rr * T + (rr - L0);     // element of lag L0
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int l = lane + 32 * m;
        v[i][m] = (rr < r1 && l <= lim) ? __ldcs(p - l) : __int_as_float(0x7fc00000);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m)
        if (v[i][m] == v[i][m]) {  // NaN: undefined pair (or no element)
          s[m] += v[i][m];
          c[m] += 1;
        }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    ssum[warp][lane + 32 * m] = s[m];
    scnt[warp][lane + 32 * m] = c[m];
  }
  __syncthreads();
  if (threadIdx.x < TILE) {
    double a = 0.0;
    long long n = 0;
#pragma unroll
    for (int w = 0; w < G2C_WARPS; ++w) {
      a += (double)ssum[w][threadIdx.x];
      n += scnt[w][threadIdx.x];
    }
    const long long tau = L0 + threadIdx.x;
    if (tau < T) {
      const size_t o = ((size_t)split * n_q + q) * T + tau;
      partial[o] = a;
      cnt_partial[o] = n;
    }
  }
}

__global__ void g2_from_C_reduce_kernel(const double* partial, const long long* cnt_partial, int n_q, long long T,
                                        int row_splits, double* g2, long long* count) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n_q * T) return;
  double a = 0.0;
  long long n = 0;
  for (int s = 0; s < row_splits; ++s) {
    a += partial[(size_t)s * n_q * T + gid];
    n += cnt_partial[(size_t)s * n_q * T + gid];
  }
  g2[gid] = n > 0 ? a / (double)n : __longlong_as_double(0x7ff8000000000000ll);
  if (count) count[gid] = n;
}

}  // namespace

cudaError_t launch_raw_ingest(const RawIngestParams& p, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(p.S, 0, (size_t)p.n_q * p.T * sizeof(long long), st);
  if (e == cudaSuccess && p.S2) e = cudaMemsetAsync(p.S2, 0, (size_t)p.n_q * p.T * sizeof(long long), st);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((p.Mp + RI_CHUNK - 1) / RI_CHUNK), (unsigned)((p.T_pad + RI_F - 1) / RI_F));
  if (p.dtype == 0)
    raw_ingest_kernel<0><<<grid, 256, 0, st>>>(p);
  else
    raw_ingest_kernel<1><<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_raw_scales(const long long* S, const long long* S2, const double* Sbar, int norm,
                              const long long* Mq, int n_q, long long T, int T_pad, int nT, float* r,
                              uint32_t* blk_bad, uint32_t* status, cudaStream_t st) {
  raw_scales_kernel<<<dim3(nT, n_q), TILE, 0, st>>>(S, S2, Sbar, norm, Mq, n_q, T, T_pad, nT, r, blk_bad, status);
  return cudaGetLastError();
}

cudaError_t launch_ring_mean(const long long* S, int n_q, long long T, double* Sbar, cudaStream_t st) {
  ring_mean_kernel<<<n_q, 256, 0, st>>>(S, T, Sbar);
  return cudaGetLastError();
}

cudaError_t launch_coef_mean(const float* A, long long T, int k, const double* s64, int n_q, double* Sbar,
                             cudaStream_t st) {
  coef_mean_kernel<<<1, 256, 0, st>>>(A, T, k, s64, n_q, Sbar);
  return cudaGetLastError();
}

cudaError_t launch_prep_compressed(const PrepParams& p, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(p.blk_bad, 0, (size_t)p.n_q * p.nT * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (p.skip_L) {  // the tensor-core path: ring sums, scales and R rows only
    if (p.norm == XPCS_NORM_FROB) return cudaErrorInvalidValue;
    const int lda = (p.k + 31) / 32 * 32 + 2;
    const int vec = (p.k % 4 == 0 && reinterpret_cast<uintptr_t>(p.A) % 16 == 0) ? 1 : 0;
    const int smem_sr = (SR_FRAMES * lda + SR_QG * p.k * 2) * (int)sizeof(float);
    const dim3 grid_sr(p.T_pad / SR_FRAMES, (p.n_q + SR_QG - 1) / SR_QG);
#define XPCS_SR_LAUNCH(T16, SPLIT)                                                                    \
  do {                                                                                                \
    static int attr_bytes = 0; /* the attribute only ever grows */                                   \
    if (smem_sr > attr_bytes) {                                                                       \
      e = cudaFuncSetAttribute(scales_rows_kernel<T16, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               smem_sr);                                                              \
      if (e != cudaSuccess) return e;                                                                 \
      attr_bytes = smem_sr;                                                                           \
    }                                                                                                 \
    scales_rows_kernel<T16, SPLIT><<<grid_sr, 256, smem_sr, st>>>(p, lda, vec);                       \
  } while (0)
    if (p.prec == XPCS_PREC_FP16)
      XPCS_SR_LAUNCH(__half, false);
    else if (p.prec == XPCS_PREC_BF16)
      XPCS_SR_LAUNCH(__nv_bfloat16, false);
    else
      XPCS_SR_LAUNCH(__nv_bfloat16, true);
#undef XPCS_SR_LAUNCH
    return cudaGetLastError();
  }
  const int smem = (2 * PREP_FRAMES * (p.k + 1) + p.k * 64 + PREP_FRAMES) * (int)sizeof(float);
  const dim3 grid(p.T_pad / PREP_FRAMES, p.n_q);
#define XPCS_PREP_LAUNCH(T16, SPLIT)                                                                  \
  do {                                                                                                \
    static int attr_bytes = 0; /* the attribute only ever grows */                                   \
    if (smem > attr_bytes) {                                                                          \
      e = cudaFuncSetAttribute(comp_operands_kernel<T16, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               smem);                                                                 \
      if (e != cudaSuccess) return e;                                                                 \
      attr_bytes = smem;                                                                              \
    }                                                                                                 \
    comp_operands_kernel<T16, SPLIT><<<grid, 256, smem, st>>>(p);                                     \
  } while (0)
  if (p.prec == XPCS_PREC_FP16)
    XPCS_PREP_LAUNCH(__half, false);
  else if (p.prec == XPCS_PREC_BF16)
    XPCS_PREP_LAUNCH(__nv_bfloat16, false);
  else
    XPCS_PREP_LAUNCH(__nv_bfloat16, true);
#undef XPCS_PREP_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_coef_pieces(const float* A, long long T, int k, int kq, int T_pad, __nv_bfloat16* out,
                               cudaStream_t st) {
  const long long n = (long long)T_pad * kq;
  coef_pieces_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(A, T, k, kq, n, out);
  return cudaGetLastError();
}

cudaError_t launch_gram_pieces(const double* G, int n_q, int k, int kq, __nv_bfloat16* out, cudaStream_t st) {
  const long long n = (long long)n_q * kq * kq;
  gram_pieces_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(G, n_q, k, kq, out);
  return cudaGetLastError();
}

cudaError_t launch_counts(const float* r, int n_q, long long T, int T_pad, uint32_t* vbits, int words,
                          long long* count, cudaStream_t st) {
  const long long nw = (long long)n_q * words;
  uint32_t* ring_gap = vbits + nw;  // n_q flags after the bits
  cudaError_t e = cudaMemsetAsync(ring_gap, 0, (size_t)n_q * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  vbits_kernel<<<(unsigned)((nw + 7) / 8), 256, 0, st>>>(r, n_q, T, T_pad, words, vbits, ring_gap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long n = (long long)n_q * T;
  counts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(vbits, ring_gap, n_q, T, words, count);
  return cudaGetLastError();
}

cudaError_t launch_g2_finalize(const float* partials, const long long* count, int n_q, long long T, int nT,
                               int maxC, int CH, double* g2, cudaStream_t st) {
  const long long n = (long long)n_q * T;
  g2_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(partials, count, n_q, T, nT, maxC, CH, g2);
  return cudaGetLastError();
}

cudaError_t launch_g2_from_C(const float* C, int n_q, long long T, double* partial, int row_splits,
                             long long* cnt_partial, cudaStream_t st) {
  const dim3 grid((unsigned)((T + TILE - 1) / TILE), n_q, row_splits);
  g2_from_C_kernel<<<grid, 256, 0, st>>>(C, n_q, T, partial, cnt_partial, row_splits);
  return cudaGetLastError();
}

cudaError_t launch_g2_from_C_reduce(const double* partial, const long long* cnt_partial, int n_q, long long T,
                                    int row_splits, double* g2, long long* count, cudaStream_t st) {
  const long long n = (long long)n_q * T;
  g2_from_C_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(partial, cnt_partial, n_q, T, row_splits,
                                                                       g2, count);
  return cudaGetLastError();
}

cudaError_t preload_g2_from_C() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, g2_from_C_kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncGetAttributes(&a, g2_from_C_reduce_kernel);
}

}  // namespace xpcs
