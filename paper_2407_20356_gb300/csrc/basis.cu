// Basis fit helpers (Eq. 3-6) and per-ring basis factors, FP64, sm_103a.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace xpcs {

namespace {

// Gf[i][j] = N[i][j] / sqrt(N[i][i] N[j][j]): the Gram of the Frobenius-normalised frames
// (Sec. 2.1) from the exact integer Gram (lower triangle valid).  Zero frames give zero
// rows and columns, which only add zero eigenvalues.
__global__ void gram_normalise_kernel(const long long* N, int n, double* Gf, double* nrm) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n * n) return;
  const int i = (int)(gid / n), j = (int)(gid % n);
  const int a = min(i, j), b = max(i, j);
  const double di = (double)N[(size_t)i * n + i], dj = (double)N[(size_t)j * n + j];
  const double v = (double)N[(size_t)b * n + a];
  Gf[gid] = (di > 0 && dj > 0) ? v / sqrt(di * dj) : 0.0;
  if (j == 0) nrm[i] = sqrt(di);
}

// Z[t][i] = u_t,(n-1-i) / (sigma_i ||x_t||): eigenvalues come ascending from the solver.
__global__ void basis_z_kernel(const double* U, const double* lam, const double* nrm, int n, int k, double* Z) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n * k) return;
  const int t = (int)(gid / k), i = (int)(gid % k);
  const int col = n - 1 - i;
  const double sig = sqrt(fmax(lam[col], 0.0));
  // column-major eigenvectors: U[col * n + t]
  Z[gid] = (nrm[t] > 0 && sig > 0) ? U[(size_t)col * n + t] / (sig * nrm[t]) : 0.0;
}

// B[p][i] = sum_t x_{t,p} Z[t][i] for a 32-wide column tile; zero counts are skipped.
constexpr int BB_T = 64;
__global__ void __launch_bounds__(128) basis_build_kernel(const void* F, int dtype, int n, long long M,
                                                          const double* Z, int k, double* B) {
  __shared__ double Zs[BB_T][32];
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = blockIdx.y * 32;
  const int ni = min(32, k - i0);
  double acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0.0;
  for (int t0 = 0; t0 < n; t0 += BB_T) {
    __syncthreads();
    for (int e = threadIdx.x; e < BB_T * 32; e += blockDim.x) {
      const int tt = e / 32, i = e % 32;
      Zs[tt][i] = (t0 + tt < n && i < ni) ? Z[(size_t)(t0 + tt) * k + i0 + i] : 0.0;
    }
    __syncthreads();
    if (p < M) {
      const int tn = min(BB_T, n - t0);
      for (int tt = 0; tt < tn; ++tt) {
        const size_t o = (size_t)(t0 + tt) * M + p;
        const unsigned x = dtype == 0 ? (unsigned)static_cast<const uint8_t*>(F)[o]
                                      : (unsigned)static_cast<const uint16_t*>(F)[o];
        if (x) {
          const double xd = (double)x;
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] = fma(xd, Zs[tt][i], acc[i]);
        }
      }
    }
  }
  if (p < M)
    for (int i = 0; i < ni; ++i) B[(size_t)p * k + i0 + i] = acc[i];
}

// Sign convention: the entry of largest magnitude of each column is positive
// (first index wins ties).
__global__ void basis_sign_kernel(double* B, long long M, int k) {
  const int i = blockIdx.x;
  __shared__ double sv[256];
  __shared__ long long si[256];
  double best = -1.0;
  long long bi = 0;
  for (long long p = threadIdx.x; p < M; p += blockDim.x) {
    const double a = fabs(B[(size_t)p * k + i]);
    if (a > best) {
      best = a;
      bi = p;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sv[threadIdx.x + s];
      const long long oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const bool flip = B[(size_t)si[0] * k + i] < 0.0;
  if (flip)
    for (long long p = threadIdx.x; p < M; p += blockDim.x) B[(size_t)p * k + i] = -B[(size_t)p * k + i];
}

// Partial ring factors over one split of a ring's pixels:
//   Gpart[q][split] = sum_p B_p^T B_p (32x32 tile), spart[q][split] = sum_p B_p.
// Pixels of ring q are perm[off_q .. off_q + M_q) (ring-sorted plan).
constexpr int RF_P = 32;
__global__ void __launch_bounds__(256) ring_factors_kernel(const double* B, int k, const int* perm, const int* off,
                                                           const long long* Mq, int n_split, double* Gpart,
                                                           double* spart) {
  __shared__ double Bi[RF_P][33];
  __shared__ double Bj[RF_P][33];
  const int q = blockIdx.z / n_split, split = blockIdx.z % n_split;
  const int ti = blockIdx.x, tj = blockIdx.y;
  const int i0 = ti * 32, j0 = tj * 32;
  const long long m = Mq[q];
  const long long per = (m + n_split - 1) / n_split;
  const long long p0 = (long long)split * per, p1 = min(m, p0 + per);
  const int* pix = perm + off[q];
  const int r = threadIdx.x / 8;   // output row in tile 0..31
  const int c4 = threadIdx.x % 8;  // 4 output columns
  double acc[4] = {0, 0, 0, 0};
  double sacc = 0.0;
  for (long long pb = p0; pb < p1; pb += RF_P) {
    __syncthreads();
    for (int e = threadIdx.x; e < RF_P * 32; e += blockDim.x) {
      const int pp = e / 32, c = e % 32;
      const long long pi = pb + pp;
      double vi = 0.0, vj = 0.0;
      if (pi < p1) {
        const size_t row = (size_t)pix[pi] * k;
        if (i0 + c < k) vi = B[row + i0 + c];
        if (j0 + c < k) vj = B[row + j0 + c];
      }
      Bi[pp][c] = vi;
      Bj[pp][c] = vj;
    }
    __syncthreads();
#pragma unroll 4
    for (int pp = 0; pp < RF_P; ++pp) {
      const double a = Bi[pp][r];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(a, Bj[pp][c4 * 4 + u], acc[u]);
    }
    if (tj == 0 && threadIdx.x < 32)
      for (int pp = 0; pp < RF_P; ++pp) sacc += Bi[pp][threadIdx.x];
  }
  double* G = Gpart + ((size_t)q * n_split + split) * k * k;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int gi = i0 + r, gj = j0 + c4 * 4 + u;
    if (gi < k && gj < k) G[(size_t)gi * k + gj] = acc[u];
  }
  if (tj == 0 && threadIdx.x < 32 && i0 + (int)threadIdx.x < k)
    spart[((size_t)q * n_split + split) * k + i0 + threadIdx.x] = sacc;
}

__global__ void ring_factors_reduce_kernel(const double* Gpart, const double* spart, int n_split, int n_q, int k,
                                           double* G, double* s, float* G32, float2* s32) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long kk = (long long)k * k;
  if (gid < (long long)n_q * kk) {
    const int q = (int)(gid / kk);
    const long long e = gid % kk;
    double a = 0.0;
    for (int sp = 0; sp < n_split; ++sp) a += Gpart[((size_t)q * n_split + sp) * kk + e];
    G[gid] = a;
    G32[gid] = (float)a;
  }
  if (gid < (long long)n_q * k) {
    const int q = (int)(gid / k), c = (int)(gid % k);
    double a = 0.0;
    for (int sp = 0; sp < n_split; ++sp) a += spart[((size_t)q * n_split + sp) * k + c];
    s[gid] = a;
    const float hi = (float)a;
    s32[gid] = make_float2(hi, (float)(a - (double)hi));
  }
}

// Bcat (2kp x M_pad, f16, pixel-contiguous rows): rows 0..k-1 = hi = f16(V^T 2^s), rows
// kp..kp+k-1 = lo = f16(V^T 2^s - hi); padded pixels and rows stay zero.  Tiled transpose
// through shared memory.
__global__ void basis_pack_kernel(const double* B, long long M, long long M_pad, int k, int kp, int log2_scale,
                                  __half* Bcat) {
  __shared__ double tile[32][33];
  const long long p0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    const long long p = p0 + yy;
    const int c = c0 + tx;
    tile[yy][tx] = (p < M && c < k) ? ldexp(B[(size_t)p * k + c], log2_scale) : 0.0;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int c = c0 + yy;
    const long long p = p0 + tx;
    if (c < k && p < M_pad) {
      const double v = tile[tx][yy];
      const __half hi = __double2half(v);
      const __half lo = __double2half(v - (double)__half2float(hi));
      Bcat[(size_t)c * M_pad + p] = hi;
      Bcat[(size_t)(kp + c) * M_pad + p] = lo;
    }
  }
}

__global__ void absmax_kernel(const double* B, long long n, double* out) {
  __shared__ double sm[256];
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(B[i]));
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

}  // namespace

cudaError_t launch_gram_normalise(const long long* N, int n, double* Gf, double* nrm, cudaStream_t st) {
  const long long tot = (long long)n * n;
  gram_normalise_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(N, n, Gf, nrm);
  return cudaGetLastError();
}

cudaError_t launch_basis_z(const double* U, const double* lam, const double* nrm, int n, int k, double* Z,
                           cudaStream_t st) {
  const long long tot = (long long)n * k;
  basis_z_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(U, lam, nrm, n, k, Z);
  return cudaGetLastError();
}

cudaError_t launch_basis_build(const void* F, int dtype, int n, long long M, const double* Z, int k, double* B,
                               cudaStream_t st) {
  const dim3 grid((unsigned)((M + 127) / 128), (k + 31) / 32);
  basis_build_kernel<<<grid, 128, 0, st>>>(F, dtype, n, M, Z, k, B);
  return cudaGetLastError();
}

cudaError_t launch_basis_sign(double* B, long long M, int k, cudaStream_t st) {
  basis_sign_kernel<<<k, 256, 0, st>>>(B, M, k);
  return cudaGetLastError();
}

cudaError_t launch_ring_factors2(const double* B, int k, const int* perm, const int* off, const long long* Mq,
                                 int n_q, int n_split, double* Gpart, double* spart, cudaStream_t st) {
  const int nt = (k + 31) / 32;
  const dim3 grid(nt, nt, n_q * n_split);
  ring_factors_kernel<<<grid, 256, 0, st>>>(B, k, perm, off, Mq, n_split, Gpart, spart);
  return cudaGetLastError();
}

cudaError_t launch_ring_factors_reduce(const double* Gpart, const double* spart, int n_chunks, int n_q, int k,
                                       double* G, double* s, float* G32, float2* s32, cudaStream_t st) {
  const long long tot = (long long)n_q * k * k;
  ring_factors_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Gpart, spart, n_chunks, n_q, k, G, s,
                                                                           G32, s32);
  return cudaGetLastError();
}

cudaError_t launch_basis_absmax(const double* B, long long n, double* out, cudaStream_t st) {
  absmax_kernel<<<256, 256, 0, st>>>(B, n, out);
  return cudaGetLastError();
}

cudaError_t launch_basis_pack(const double* B, long long M, long long M_pad, int k, int kp, int log2_scale,
                              __half* Bcat, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(Bcat, 0, (size_t)2 * kp * M_pad * sizeof(__half), st);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((M_pad + 31) / 32), (k + 31) / 32);
  basis_pack_kernel<<<grid, 256, 0, st>>>(B, M, M_pad, k, kp, log2_scale, Bcat);
  return cudaGetLastError();
}

}  // namespace xpcs
