// Stream row update on the tcgen05 tensor cores (sm_103a).
//
// For a step of b <= 64 frames t0 .. t0 + b - 1 and every lag tau < W, ring q:
//     C_q(t, s) = w_q(t) . a_s * r_q(s),  s = t - tau,  w_q(t) = r_q(t) a_t G_q,
// summed into lag bins g2sum_q[tau] (count_q[tau] += 1 for defined pairs).
//
// Work item = (tile of LT consecutive lags tau0 .., group of up to 36 rings).  All its
// pairs use history rows s in [t0 - tau0 - LT + 1, t0 + b - 1 - tau0], fewer than 128
// rows: one 128-row operand.  The other operand holds the (frame, ring) pairs of the
// group, 128 per M-tile, laid out by the frame-factors kernel so that ring q sits in
// TMEM lane quarter q mod 4 (one epilogue warp per quarter): M-tile mt, lane quarter w,
// lane l holds pair idx = 32 mt + l of the list (f, q) with q = q0 + 4 (idx / b) + w,
// f = idx mod b.  One GEMM per M-tile,
//     D[pair][c] = w_q(t0 + f) . a_{s_start + c},   c = 0..127,
// with both operands as bf16 hi/lo pieces of the f32 values (hi.hi + lo.hi + hi.lo,
// f32 accumulation: about 2^-16 relative per product).  In the epilogue a thread owns one
// pair and walks its columns: column c is lag tau0 + tl with tl = f + LT - 1 - c, so the
// thread adds D r_q(s) to bin (q, tl) when 0 <= tl < LT, tau < W, s >= 0 and both r are
// positive.  Lanes of a warp hold distinct pairs and warps hold disjoint rings, so at any
// column the 128 threads update distinct bins: no atomics and no barriers, and every
// bin's additions come in a fixed order.  The bins are added to the FP64 sums once per
// work item.
//
// Warps: 0 TMA producer (history rows + their r values once per item, pair chunks
// through a ring of stages), 1 TMEM owner and MMA issuer (two 128-column accumulators),
// 2..5 epilogue.  Every mbarrier wait is bounded (status word + unwind).
#include "common.cuh"
#include "internal.h"

namespace xpcs {

namespace {

constexpr int RT_ROWS = 128;                   // MMA M (pairs) and N (history rows)
constexpr int RT_CH = 64;                      // K chunk: 64 bf16 = one 128-byte row
constexpr int RT_CHUNK = RT_ROWS * RT_CH * 2;  // 16 KB: one operand chunk
constexpr int RT_THREADS = 192;
constexpr int RT_EPI_BAR = 1;
constexpr int RT_QG = 36;                      // rings per work item (nine per lane quarter)

struct RtLayout {
  int n_kc, lt, qb, wst;
  __host__ __device__ int hist_bytes() const { return 2 * n_kc * RT_CHUNK; }
  __host__ __device__ int w_bytes() const { return wst * 2 * RT_CHUNK; }
  __host__ __device__ int rs_bytes() const { return RT_ROWS * qb * 4; }
  __host__ __device__ int bins_bytes() const { return RT_QG * (lt + 1) * 4; }
  __host__ __device__ int rot_bytes() const { return 4 * 32 * 32 * 4; }  // a 32x32 block per epilogue warp
  __host__ __device__ int smem() const {
    return 1024 + hist_bytes() + w_bytes() + rs_bytes() + bins_bytes() + rot_bytes() + 256;
  }
};

// 64 validity bits of one ring starting at ring slot o (the bit array mirrors its first
// 64 slots after slot cap - 1, so a window never wraps)
XPCS_DEV unsigned long long bits_at(const unsigned long long* vb, long long o) {
  const long long wi = o >> 6;
  const int sh = (int)(o & 63);
  const unsigned long long lo = __ldg(vb + wi);
  return sh ? (lo >> sh) | (__ldg(vb + wi + 1) << (64 - sh)) : lo;
}

__global__ void __launch_bounds__(RT_THREADS, 1)
    row_update_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
                         const __grid_constant__ CUtensorMap tmR, const RowTcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const RtLayout L{p.n_kc, p.lt, p.qb, p.wst};
  uint8_t* hist = smem;                                       // [hi kc..., lo kc...]
  uint8_t* w_st = smem + L.hist_bytes();                      // [stage][hi, lo]
  float* rs = reinterpret_cast<float*>(w_st + L.w_bytes());   // [128][qb] r_q of the history rows
  float* bins = rs + RT_ROWS * p.qb;                          // [36][lt + 1]
  float* rot = bins + RT_QG * (p.lt + 1);                     // [4][32][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(rot) + L.rot_bytes());
  uint64_t* h_full = bars;        // history + r rows landed
  uint64_t* h_empty = bars + 1;   // MMAs done with the history rows
  uint64_t* r_empty = bars + 2;   // epilogue done with the r rows
  uint64_t* w_full = bars + 3;    // [wst <= 4]
  uint64_t* w_empty = bars + 7;   // [wst]
  uint64_t* tfull = bars + 11;    // [2]
  uint64_t* tempty = bars + 13;   // [2]
  uint64_t* mma_done = bars + 15;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 16);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lt = p.lt;
  const int n_items = p.n_tiles * p.n_rg;

  if (threadIdx.x == 0) {
    mbar_init(h_full, 1);
    mbar_init(h_empty, 1);
    mbar_init(r_empty, 4);
    for (int s = 0; s < p.wst; ++s) {
      mbar_init(&w_full[s], 1);
      mbar_init(&w_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(mma_done, 1);
    mbar_fence_init();
    *abort_flag = 0;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 2 * RT_ROWS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmW);
      tma_prefetch_desc(&tmR);
      uint32_t item_i = 0, it = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, ++item_i) {
        const uint32_t par = (item_i & 1) ^ 1;
        if (*abort_flag || !mbar_wait(h_empty, par, p.status) || !mbar_wait(r_empty, par, p.status)) {
          *abort_flag = 1;
          break;
        }
        const int tile = item / p.n_rg, rg = item - tile * p.n_rg;
        const long long tau0 = (long long)tile * lt;
        const long long s_start = p.t0 - tau0 - (lt - 1);
        // before the ring buffer wraps, rows before frame 0 are read as zeros (negative
        // coordinates); afterwards the window is contiguous thanks to the mirrored rows
        const int y = (s_start < 0 && p.t0 + p.b <= p.cap) ? (int)s_start
                                                            : (int)(((s_start % p.cap) + p.cap) % p.cap);
        mbar_arrive_expect_tx(h_full, (uint32_t)(L.hist_bytes() + L.rs_bytes()));
        for (int kc = 0; kc < p.n_kc; ++kc) {
          tma_load_2d(hist + kc * RT_CHUNK, &tmA, h_full, kc * RT_CH, y);
          tma_load_2d(hist + (p.n_kc + kc) * RT_CHUNK, &tmA, h_full, p.kpad + kc * RT_CH, y);
        }
        tma_load_2d(rs, &tmR, h_full, rg * RT_QG, y);
        for (int mt = 0; mt < p.n_mt && ok; ++mt) {
          for (int kc = 0; kc < p.n_kc; ++kc, ++it) {
            const uint32_t s = it % p.wst, ph = (it / p.wst) & 1;
            if (*abort_flag || !mbar_wait(&w_empty[s], ph ^ 1, p.status)) {
              *abort_flag = 1;
              ok = false;
              break;
            }
            uint8_t* dst = w_st + s * 2 * RT_CHUNK;
            const int wy = (rg * p.n_mt + mt) * RT_ROWS;
            mbar_arrive_expect_tx(&w_full[s], 2 * RT_CHUNK);
            tma_load_2d(dst, &tmW, &w_full[s], kc * RT_CH, wy);
            tma_load_2d(dst + RT_CHUNK, &tmW, &w_full[s], p.kpad + kc * RT_CH, wy);
          }
        }
      }
      // never leave the CTA with bulk copies in flight
      if (item_i) mbar_wait(h_full, (item_i - 1) & 1, p.status);
      for (uint32_t j = (it > (uint32_t)p.wst ? it - p.wst : 0); j < it; ++j)
        mbar_wait(&w_full[j % p.wst], (j / p.wst) & 1, p.status);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // history rows used by the step: lt + b - 1 (N a multiple of 16)
      const uint32_t idesc = idesc_f16(1, RT_ROWS, min(RT_ROWS, (lt + p.b - 1 + 15) / 16 * 16));
      uint32_t item_i = 0, it = 0, acc_i = 0;
      bool ok = true, issued = false;
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, ++item_i) {
        if (*abort_flag || !mbar_wait(h_full, item_i & 1, p.status)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        for (int mt = 0; mt < p.n_mt && ok; ++mt, ++acc_i) {
          const uint32_t buf = acc_i & 1;
          if (*abort_flag || !mbar_wait(&tempty[buf], ((acc_i >> 1) & 1) ^ 1, p.status)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + buf * RT_ROWS;
          for (int kc = 0; kc < p.n_kc; ++kc, ++it) {
            const uint32_t s = it % p.wst, ph = (it / p.wst) & 1;
            if (*abort_flag || !mbar_wait(&w_full[s], ph, p.status)) {
              *abort_flag = 1;
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t whi = smem_desc_sw128(w_st + s * 2 * RT_CHUNK);
            const uint64_t wlo = smem_desc_sw128(w_st + s * 2 * RT_CHUNK + RT_CHUNK);
            const uint64_t hhi = smem_desc_sw128(hist + kc * RT_CHUNK);
            const uint64_t hlo = smem_desc_sw128(hist + (p.n_kc + kc) * RT_CHUNK);
#pragma unroll
            for (int kk = 0; kk < RT_CH / 16; ++kk) {  // 16 elements = 32 B per MMA
              tc_mma_f16(d, whi + 2 * kk, hhi + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
              tc_mma_f16(d, wlo + 2 * kk, hhi + 2 * kk, idesc, 1u);
              tc_mma_f16(d, whi + 2 * kk, hlo + 2 * kk, idesc, 1u);
            }
            tc_commit(&w_empty[s]);
            issued = true;
          }
          if (!ok) break;
          tc_commit(&tfull[buf]);
        }
        if (!ok) break;
        tc_commit(h_empty);  // the history rows are free once these MMAs complete
      }
      if (issued) {  // all issued MMAs complete before TMEM is released
        tc_commit(mma_done);
        mbar_wait(mma_done, 0, p.status);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int w = warp & 3;           // TMEM lane quarter = ring residue
    const int et = threadIdx.x - 64;  // 0..127
    const unsigned long long bmask = p.b == 64 ? ~0ull : ((1ull << p.b) - 1);
    const long long o_batch = p.t0 % p.cap;  // validity bits of the step's own frames
    uint32_t item_i = 0, acc_i = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++item_i) {
      const int tile = item / p.n_rg, rg = item - tile * p.n_rg;
      const int q0 = rg * RT_QG;
      const int qn = min(RT_QG, p.n_q - q0);
      const long long tau0 = (long long)tile * lt;
      const long long s_start = p.t0 - tau0 - (lt - 1);
      const int tl_max = (int)min((long long)lt - 1, p.W - 1 - tau0);  // lags that exist
      const int c_min = s_start < 0 ? (int)(-s_start) : 0;              // rows before frame 0
      for (int e = et; e < RT_QG * (lt + 1); e += 128) bins[e] = 0.f;
      named_bar_sync(RT_EPI_BAR, 128);
      bool good = ok && !__any_sync(0xffffffffu, *abort_flag != 0);  // warp-uniform
      if (good) good = mbar_wait_warp(h_full, item_i & 1, p.status);  // r rows landed
      if (!good) {
        *abort_flag = 1;
        ok = false;
      }
      for (int mt = 0; mt < p.n_mt; ++mt, ++acc_i) {
        const uint32_t buf = acc_i & 1;
        good = ok && !__any_sync(0xffffffffu, *abort_flag != 0);
        if (good) good = mbar_wait_warp(&tfull[buf], (acc_i >> 1) & 1, p.status);
        if (!good) {
          *abort_flag = 1;
          ok = false;
        }
        tc_fence_after();
        // Column c of frame f is lag tl = f + lt - 1 - c, kept when 0 <= tl <= tl_max and
        // the row exists (c >= c_min).  Undefined frames contribute zeros (r = 0 in both
        // factors); pair counts come from the validity bits in the fold.
        if (p.b <= W2_SMALL_B) {
          // one frame per M-tile, lane l < 9 holds ring q0 + 4 l + w: the lanes' bins are
          // disjoint, so each thread adds its columns straight into its ring's bins
          const int f = mt, ql = 4 * lane + w;
          const bool pair_ok = lane < 9 && ql < qn;
          const int c_a = max(f + lt - 1 - tl_max, c_min), c_b = min(f + lt - 1, RT_ROWS - 1);
          if (ok && c_a <= c_b && __any_sync(0xffffffffu, pair_ok)) {
            float* brow = bins + (pair_ok ? ql : 0) * (lt + 1) + f + lt - 1;  // bin of column c: brow[-c]
            const float* rcol = rs + (pair_ok ? ql : 0);                      // r of column c: rcol[c qb]
#pragma unroll 1
            for (int c32 = c_a >> 5; c32 <= (c_b >> 5); ++c32) {
              uint32_t v[32];
              tmem_ld32(tmem_base + buf * RT_ROWS + ((uint32_t)(w * 32) << 16) + c32 * 32, v);
              tc_wait_ld();
              if (pair_ok) {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                  const int c = c32 * 32 + jj;
                  if (c >= c_a && c <= c_b) brow[-c] = fmaf(__uint_as_float(v[jj]), rcol[c * p.qb], brow[-c]);
                }
              }
            }
          }
        } else {
        // this warp holds ring q0 + ql for frames f0 .. f0 + 31 (lane = frame offset)
        const int qi = mt / p.nfb, fb = mt - qi * p.nfb;
        const int ql = 4 * qi + w, f0 = 32 * fb, f = f0 + lane;
        const bool pair_ok = ql < qn && f < p.b;
        const int c_a = pair_ok ? max(f + lt - 1 - tl_max, c_min) : RT_ROWS;
        const int c_b = pair_ok ? min(f + lt - 1, RT_ROWS - 1) : -1;
        const int c_lo = __reduce_min_sync(0xffffffffu, c_a);
        const int c_hi = __reduce_max_sync(0xffffffffu, c_b);
        if (ok && c_lo <= c_hi) {
          float* P = rot + w * 1024;
          float* brow = bins + ql * (lt + 1);
#pragma unroll 1
          for (int c32 = c_lo >> 5; c32 <= (c_hi >> 5); ++c32) {
            uint32_t v[32];
            tmem_ld32(tmem_base + buf * RT_ROWS + ((uint32_t)(w * 32) << 16) + c32 * 32, v);
            tc_wait_ld();
            // C(f, c) r_q(s_c) of this 32 x 32 block, zero outside the kept lags, written
            // rotated: P[i][(j - i) mod 32] = x(i, j)
            __syncwarp();  // the previous block's reads of P are done
            {
              float* prow = P + lane * 32;
              int o = (32 - lane) & 31;
#pragma unroll
              for (int jj = 0; jj < 32; ++jj) {
                const int c = c32 * 32 + jj;
                const float x = (c >= c_a && c <= c_b) ? __uint_as_float(v[jj]) * rs[c * p.qb + ql] : 0.f;
                prow[o] = x;
                o = (o + 1) & 31;
              }
            }
            __syncwarp();
            // lane d sums column d: rows i < 32 - d lie on diagonal j - i = d, the others on
            // d - 32; diagonal e is lag offset tl = T0 - e
            float an = 0.f, aw = 0.f;
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
              const float y = P[i * 32 + lane];
              if (i < 32 - lane)
                an += y;
              else
                aw += y;
            }
            const int T0 = f0 + lt - 1 - 32 * c32;
            const int bn = T0 - lane, bw = T0 - lane + 32;
            if (bn >= 0 && bn < lt) brow[bn] += an;
            if (bw >= 0 && bw < lt) brow[bw] += aw;
          }
        }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(r_empty);  // the r rows may be replaced
      named_bar_sync(RT_EPI_BAR, 128);     // all bins of the item are complete
      // fold the item's bins into the FP64 sums (one owner per bin).  Pair count of
      // (q, tau) in this step: frames f < b whose frame t0 + f and history frame
      // t0 + f - tau are both defined, a popcount of two validity-bit windows.
      // Loads of four bins are issued before their stores.
      if (ok) {
        const int n = qn * lt;
        for (int e0 = et; e0 < n; e0 += 4 * 128) {
          double gs[4];
          long long gc[4];
          size_t gi[4];
          int bi[4], cntu[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * 128;
            cntu[u] = 0;
            gi[u] = 0;
            bi[u] = 0;
            if (e < n) {
              const int ql = e / lt, tl = e - ql * lt;
              const long long tau = tau0 + tl;
              if (tl <= tl_max) {
                const unsigned long long* vb = p.vbits + (size_t)(q0 + ql) * p.vwords;
                const unsigned long long mine = bits_at(vb, o_batch) & bmask;
                const long long o_h = (((p.t0 - tau) % p.cap) + p.cap) % p.cap;
                cntu[u] = __popcll(mine & bits_at(vb, o_h));
              }
              bi[u] = ql * (lt + 1) + tl;
              gi[u] = (size_t)(q0 + ql) * p.W + (size_t)(tau0 + tl);
              if (cntu[u]) {
                gs[u] = p.g2sum[gi[u]];
                gc[u] = p.cnt[gi[u]];
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (cntu[u]) {
              p.g2sum[gi[u]] = gs[u] + (double)bins[bi[u]];
              p.cnt[gi[u]] = gc[u] + cntu[u];
            }
        }
      }
      // one decision for all four warps (also orders the fold before the next zeroing)
      if (named_bar_sync_or(RT_EPI_BAR, 128, !ok || *abort_flag)) break;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 2 * RT_ROWS);
  }
}

}  // namespace

int row_update_tc_smem(int n_kc, int lt, int qb, int wst) { return RtLayout{n_kc, lt, qb, wst}.smem(); }

cudaError_t launch_row_update_tc(const CUtensorMap& tmA, const CUtensorMap& tmW, const CUtensorMap& tmR,
                                 const RowTcParams& p, int grid, cudaStream_t st) {
  const int smem = row_update_tc_smem(p.n_kc, p.lt, p.qb, p.wst);
  static int attr_bytes = 0;  // the attribute only ever grows
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(row_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  row_update_tc_kernel<<<grid, RT_THREADS, smem, st>>>(tmA, tmW, tmR, p);
  return cudaGetLastError();
}

}  // namespace xpcs
