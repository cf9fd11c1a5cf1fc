// Downstream analysis of g2 and of a stored two-time matrix, on the device (Sec. 3).
//
// * Eq. 13 relaxation fit per ring: g2(tau) = B + C exp(-2 tau / t0), unweighted least
//   squares over the defined lags of [tau_lo, tau_hi].  For a fixed t0 the model is
//   linear in (B, C): two sums passes give the 2x2 normal equations and then the residual
//   sum of squares, so the residual is a function of t0 alone.  It is minimised over
//   log t0: a grid of FIT_GRID points over [log t0_min, log t0_max], then golden-section
//   steps inside the grid neighbours of the best point.  One block per ring; per-term
//   arithmetic in f32 (expf), every sum in FP64 with a fixed-order block reduction, so
//   the result is deterministic.
// * Peak visibility (Sec. 3.1): the largest g2 over a peak window of lags minus the mean
//   g2 over a background window (defined lags only), and the detectability flag of
//   Sec. 3.2: visibility > factor x the standard deviation of the TTC.
// * TTC statistics: mean and population standard deviation of the stored lower
//   triangle's off-diagonal defined values (each unordered pair once), per ring; the
//   matrix is read once with coalesced row segments (HBM-bound).
#include <cmath>
#include <string>

#include "handles.h"
#include "internal.h"

using namespace xpcs;

namespace {

constexpr int FIT_THREADS = 256;
constexpr int FIT_GRID = 129;
constexpr int FIT_GOLDEN = 60;
constexpr int STATS_THREADS = 256;
constexpr int STATS_ROWS = 64;  // rows of the lower triangle per block

// Fixed-order sum of one double per thread over the block; every thread gets the total.
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double s = red[0];
  __syncthreads();
  return s;
}

struct FitEval {
  double rss, B, C;
};

// Least-squares (B, C) and the residual sum of squares for t0 = exp(lt).
__device__ FitEval fit_eval(const double* g, long long lo, long long hi, double n, double Sg, double lt,
                            double* red) {
  const float k2 = (float)(2.0 / exp(lt));
  double se = 0.0, see = 0.0, sge = 0.0;
  for (long long t = lo + threadIdx.x; t <= hi; t += blockDim.x) {
    const double gv = g[t];
    if (isnan(gv)) continue;
    const float e = expf(-k2 * (float)t);
    se += e;
    see += (double)e * e;
    sge += gv * e;
  }
  se = block_sum(se, red);
  see = block_sum(see, red);
  sge = block_sum(sge, red);
  const double det = n * see - se * se;
  FitEval r;
  r.C = det > 0.0 ? (n * sge - se * Sg) / det : 0.0;
  r.B = (Sg - r.C * se) / n;
  double rs = 0.0;
  for (long long t = lo + threadIdx.x; t <= hi; t += blockDim.x) {
    const double gv = g[t];
    if (isnan(gv)) continue;
    const float e = expf(-k2 * (float)t);
    const double d = gv - r.B - r.C * (double)e;
    rs += d * d;
  }
  r.rss = block_sum(rs, red);
  return r;
}

__global__ void __launch_bounds__(FIT_THREADS) relaxation_fit_kernel(const double* g2, long long T, long long lo,
                                                                     long long hi, double lt_min, double lt_max,
                                                                     double* out) {
  __shared__ double red[FIT_THREADS];
  const int q = blockIdx.x;
  const double* g = g2 + (size_t)q * T;
  double n = 0.0, sg = 0.0;
  for (long long t = lo + threadIdx.x; t <= hi; t += blockDim.x) {
    const double gv = g[t];
    if (isnan(gv)) continue;
    n += 1.0;
    sg += gv;
  }
  n = block_sum(n, red);
  sg = block_sum(sg, red);
  double* o = out + (size_t)q * 4;
  if (n < 3.0) {
    if (threadIdx.x == 0) o[0] = o[1] = o[2] = o[3] = nan("");
    return;
  }
  // grid over log t0
  const double step = (lt_max - lt_min) / (FIT_GRID - 1);
  int best = 0;
  double best_rss = INFINITY;
  for (int i = 0; i < FIT_GRID; ++i) {
    const FitEval e = fit_eval(g, lo, hi, n, sg, lt_min + step * i, red);
    if (e.rss < best_rss) {
      best_rss = e.rss;
      best = i;
    }
  }
  // golden-section search between the grid neighbours of the best point
  double a = lt_min + step * (best > 0 ? best - 1 : 0);
  double b = lt_min + step * (best < FIT_GRID - 1 ? best + 1 : FIT_GRID - 1);
  const double rg = 0.6180339887498949;  // (sqrt(5) - 1) / 2
  double x1 = b - rg * (b - a), x2 = a + rg * (b - a);
  double f1 = fit_eval(g, lo, hi, n, sg, x1, red).rss, f2 = fit_eval(g, lo, hi, n, sg, x2, red).rss;
  for (int it = 0; it < FIT_GOLDEN; ++it) {
    if (f1 <= f2) {
      b = x2;
      x2 = x1;
      f2 = f1;
      x1 = b - rg * (b - a);
      f1 = fit_eval(g, lo, hi, n, sg, x1, red).rss;
    } else {
      a = x1;
      x1 = x2;
      f1 = f2;
      x2 = a + rg * (b - a);
      f2 = fit_eval(g, lo, hi, n, sg, x2, red).rss;
    }
  }
  double lt = f1 <= f2 ? x1 : x2;
  FitEval e = fit_eval(g, lo, hi, n, sg, lt, red);
  if (e.rss > best_rss) {  // the grid point was better (flat or multi-modal residual)
    lt = lt_min + step * best;
    e = fit_eval(g, lo, hi, n, sg, lt, red);
  }
  if (threadIdx.x == 0) {
    o[0] = e.B;
    o[1] = e.C;
    o[2] = exp(lt);
    o[3] = sqrt(e.rss / n);
  }
}

// Partial sums over rows [row0, row0 + STATS_ROWS) of ring q's lower triangle, strictly
// below the diagonal: element [q][i][j], j < i, is C(j, i).
__global__ void __launch_bounds__(STATS_THREADS) ttc_stats_kernel(const float* C, long long T, int nblk,
                                                                  double* part) {
  __shared__ double red[STATS_THREADS];
  const int q = blockIdx.y;
  const long long row0 = (long long)blockIdx.x * STATS_ROWS;
  double s = 0.0, s2 = 0.0, n = 0.0;
  for (long long i = row0; i < row0 + STATS_ROWS && i < T; ++i) {
    const float* row = C + ((size_t)q * T + i) * T;
    for (long long j = threadIdx.x; j < i; j += blockDim.x) {
      const float v = __ldcs(row + j);
      if (isnan(v)) continue;
      s += v;
      s2 += (double)v * v;
      n += 1.0;
    }
  }
  s = block_sum(s, red);
  s2 = block_sum(s2, red);
  n = block_sum(n, red);
  if (threadIdx.x == 0) {
    double* p = part + ((size_t)q * nblk + blockIdx.x) * 3;
    p[0] = s;
    p[1] = s2;
    p[2] = n;
  }
}

__global__ void ttc_stats_reduce_kernel(const double* part, int nblk, int n_q, double* mean, double* sd) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_q) return;
  double s = 0.0, s2 = 0.0, n = 0.0;
  for (int b = 0; b < nblk; ++b) {  // fixed order
    const double* p = part + ((size_t)q * nblk + b) * 3;
    s += p[0];
    s2 += p[1];
    n += p[2];
  }
  if (n > 0.0) {
    const double m = s / n;
    mean[q] = m;
    if (sd) sd[q] = sqrt(fmax(s2 / n - m * m, 0.0));
  } else {
    mean[q] = nan("");
    if (sd) sd[q] = nan("");
  }
}

__global__ void peak_visibility_kernel(const double* g2, long long T, long long pa, long long pb, long long ba,
                                       long long bb, const double* ttc_sd, double factor, double* vis,
                                       int32_t* flag) {
  __shared__ double red[256];
  __shared__ double mx[256];
  const int q = blockIdx.x;
  const double* g = g2 + (size_t)q * T;
  double m = -INFINITY;
  for (long long t = pa + threadIdx.x; t <= pb; t += blockDim.x)
    if (!isnan(g[t])) m = fmax(m, g[t]);
  mx[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + w]);
    __syncthreads();
  }
  double s = 0.0, n = 0.0;
  for (long long t = ba + threadIdx.x; t <= bb; t += blockDim.x)
    if (!isnan(g[t])) {
      s += g[t];
      n += 1.0;
    }
  s = block_sum(s, red);
  n = block_sum(n, red);
  if (threadIdx.x == 0) {
    const double v = (n > 0.0 && mx[0] > -INFINITY) ? mx[0] - s / n : nan("");
    vis[q] = v;
    if (flag) flag[q] = (ttc_sd && v > factor * ttc_sd[q]) ? 1 : 0;
  }
}

}  // namespace

extern "C" xpcs_status xpcs_fit_relaxation(xpcs_ctx* ctx, const double* g2, int n_q, int64_t T, int64_t tau_lo,
                                           int64_t tau_hi, double t0_min, double t0_max, double* params_out) {
  if (!ctx || !g2 || !params_out || n_q <= 0 || T <= 0 || tau_lo < 0 || tau_hi < tau_lo || tau_hi >= T ||
      !(t0_min > 0.0) || !(t0_max > t0_min))
    return fail(ctx, XPCS_EINVAL, "bad fit_relaxation args");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  XPCS_LAUNCH(ctx, "relaxation_fit", 1, ([&] {
                relaxation_fit_kernel<<<n_q, FIT_THREADS, 0, ctx->stream>>>(g2, T, tau_lo, tau_hi, std::log(t0_min),
                                                                            std::log(t0_max), params_out);
                return cudaGetLastError();
              }()));
  return finish(ctx);
}

extern "C" xpcs_status xpcs_twotime_stats(xpcs_ctx* ctx, const float* C, int n_q, int64_t T, double* mean_out,
                                          double* std_out) {
  if (!ctx || !C || !mean_out || n_q <= 0 || T <= 0) return fail(ctx, XPCS_EINVAL, "bad twotime_stats args");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int nblk = (int)((T + STATS_ROWS - 1) / STATS_ROWS);
  Carve c0;
  c0.take<double>((size_t)n_q * nblk * 3);
  XPCS_TRY(ensure_scratch(ctx, c0.off));
  Carve c1{0, static_cast<char*>(ctx->scratch)};
  double* part = c1.take<double>((size_t)n_q * nblk * 3);
  XPCS_LAUNCH(ctx, "ttc_stats", 2, ([&] {
                ttc_stats_kernel<<<dim3(nblk, n_q), STATS_THREADS, 0, ctx->stream>>>(C, T, nblk, part);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) return e;
                ttc_stats_reduce_kernel<<<(n_q + 127) / 128, 128, 0, ctx->stream>>>(part, nblk, n_q, mean_out,
                                                                                   std_out);
                return cudaGetLastError();
              }()));
  return finish(ctx);
}

extern "C" xpcs_status xpcs_peak_visibility(xpcs_ctx* ctx, const double* g2, int n_q, int64_t T, int64_t peak_lo,
                                            int64_t peak_hi, int64_t bg_lo, int64_t bg_hi, const double* ttc_std,
                                            double factor, double* vis_out, int32_t* flag_out) {
  if (!ctx || !g2 || !vis_out || n_q <= 0 || T <= 0 || peak_lo < 0 || peak_hi < peak_lo || peak_hi >= T ||
      bg_lo < 0 || bg_hi < bg_lo || bg_hi >= T || (flag_out && (!ttc_std || !(factor > 0.0))))
    return fail(ctx, XPCS_EINVAL, "bad peak_visibility args");
  XPCS_CUDA(ctx, cudaSetDevice(ctx->device));
  XPCS_LAUNCH(ctx, "peak_visibility", 1, ([&] {
                peak_visibility_kernel<<<n_q, 256, 0, ctx->stream>>>(g2, T, peak_lo, peak_hi, bg_lo, bg_hi, ttc_std,
                                                                     factor, vis_out, flag_out);
                return cudaGetLastError();
              }()));
  return finish(ctx);
}
