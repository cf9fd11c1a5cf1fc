// Stream row update on the tcgen05 tensor cores (sm_103a).
//
// For a step of b <= 64 frames t0 .. t0 + b - 1 and every lag tau < W, ring q:
//     C_q(t, s) = w_q(t) . a_s * r_q(s),  s = t - tau,  w_q(t) = r_q(t) a_t G_q,
// summed into lag bins g2sum_q[tau] (count_q[tau] += 1 for defined pairs).
//
// Work item = (tile of LT consecutive lags tau0 .., group of up to 36 rings).  All its
// pairs use history rows s in [t0 - tau0 - LT + 1, t0 + b - 1 - tau0], at most 128 rows
// (LT + b - 1 <= 128; the host picks the longest such tile that fits shared memory): one
// 128-row operand.  The other operand holds the (frame, ring) pairs of the group, laid out
// by the frame-factors kernel.  Both operands are bf16 hi/lo pieces of the f32 values
// (hi.hi + lo.hi + hi.lo, f32 accumulation: about 2^-16 relative per product).  Column or
// row c of the history operand is lag tau0 + tl with tl = f + LT - 1 - c for frame f; a
// pair adds D r_q(s) to bin (q, tl) when 0 <= tl < LT, tau < W and s >= 0 (undefined
// frames have r = 0).
//
// Large steps (b > 8): M-tiles of 128 pairs, ring q in TMEM lane quarter q mod 4 (one
// epilogue warp per quarter), lane = frame; D[pair][c] = w_q(t0 + f) . a_{s_start + c}.
// A warp sums the diagonals of each 32 x 32 block (through a skewed or rotated buffer)
// into its ring's bins.  Small steps (b <= 8): one frame per M-tile and the history as
// the M operand, D[c][ring] (N = 48 >= 36 rings): the thread holding TMEM lane c owns lag
// tl of every ring, so all 128 lanes work and within a frame no two threads share a bin
// (a barrier separates frames).  Either way every bin's additions come in a fixed order,
// with no atomics, and the bins are added to the running sums once per work item.  The
// sums are f32 pairs (hi, lo) updated by TwoSum: no FP64 arithmetic, which is slow on this
// part, and about 2^-48 relative rounding per addition.
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
constexpr int RT_QROWS = 64, RT_QLD = 36;      // skewed buffer of one epilogue warp (row j - i + 32)

// Epilogue modes: RT_ROT rotates each 32 x 32 block, RT_SKEW sums block diagonals through
// skewed buffers, RT_SMALL serves steps of at most W2_SMALL_B frames only (their pairs go
// straight into the lag bins), so it needs neither buffer and has room for longer lag tiles.
constexpr int RT_ROT = 0, RT_SKEW = 1, RT_SMALL = 2;
constexpr int RT_SMALL_N = 48;  // MMA N of a small step: its 36 ring pairs, rounded up to 16
constexpr int RT_VW = 6;  // validity words per ring: 4 of the history window, 2 of the step

struct RtLayout {
  int n_kc, lt, qb, wst, qg2, epi;
  __host__ __device__ int hist_bytes() const { return 2 * n_kc * RT_CHUNK; }
  __host__ __device__ int w_bytes() const { return wst * 2 * RT_CHUNK; }
  __host__ __device__ int slice_bytes() const { return (qg2 * lt * 8 + 1023) / 1024 * 1024; }  // one of two
  __host__ __device__ int rs_bytes() const { return RT_ROWS * qb * 4; }
  __host__ __device__ int bins_bytes() const { return RT_QG * (lt + 1) * 4; }
  // per epilogue warp: a skewed buffer (64 rows of 36 floats) or a rotated 32x32 block
  __host__ __device__ int rot_bytes() const {
    return epi == RT_SKEW ? 4 * RT_QROWS * RT_QLD * 4 : epi == RT_ROT ? 4 * 32 * 32 * 4 : 0;
  }
  __host__ __device__ int vw_bytes() const { return RT_QG * RT_VW * 8; }
  __host__ __device__ int smem() const {
    return 1024 + hist_bytes() + w_bytes() + 2 * slice_bytes() + rs_bytes() + bins_bytes() + rot_bytes() +
           vw_bytes() + 256;
  }
};

// 64 bits of a little-endian bit string held in 64-bit words, starting at bit o
XPCS_DEV unsigned long long bits64(const unsigned long long* w, int o) {
  const int wi = o >> 6, sh = o & 63;
  return sh ? (w[wi] >> sh) | (w[wi + 1] << (64 - sh)) : w[wi];
}

template <int EPI>
__global__ void __launch_bounds__(RT_THREADS, 1)
    row_update_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
                         const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmG,
                         const __grid_constant__ CUtensorMap tmC, const RowTcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const RtLayout L{p.n_kc, p.lt, p.qb, p.wst, p.qg2, EPI};
  uint8_t* hist = smem;                                       // [hi kc..., lo kc...]
  uint8_t* w_st = smem + L.hist_bytes();                      // [stage][hi, lo]
  double* g2s = reinterpret_cast<double*>(w_st + L.w_bytes());                     // [qg2][lt] g2 sums (f32 pairs)
  long long* cns = reinterpret_cast<long long*>(w_st + L.w_bytes() + L.slice_bytes());  // [qg2][lt] counts
  float* rs = reinterpret_cast<float*>(w_st + L.w_bytes() + 2 * L.slice_bytes());  // [128][qb] r of the rows
  float* bins = rs + RT_ROWS * p.qb;                          // [36][lt + 1]
  float* rot = bins + RT_QG * (p.lt + 1);                     // [4][64][36] skewed, [4][32][32] rotated or none
  unsigned long long* vw = reinterpret_cast<unsigned long long*>(reinterpret_cast<uint8_t*>(rot) + L.rot_bytes());
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(vw) + L.vw_bytes());
  uint64_t* h_full = bars;        // history + r rows landed
  uint64_t* h_empty = bars + 1;   // MMAs done with the history rows
  uint64_t* r_empty = bars + 2;   // epilogue done with the r rows
  uint64_t* w_full = bars + 3;    // [wst <= 4]
  uint64_t* w_empty = bars + 7;   // [wst]
  uint64_t* tfull = bars + 11;    // [2]
  uint64_t* tempty = bars + 13;   // [2]
  uint64_t* mma_done = bars + 15;
  uint64_t* s_full = bars + 16;   // g2sum / cnt slices landed
  uint64_t* s_empty = bars + 17;  // their store has read them
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 18);
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
    mbar_init(s_full, 1);
    mbar_init(s_empty, 1);
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
      tma_prefetch_desc(&tmG);
      tma_prefetch_desc(&tmC);
      uint32_t item_i = 0, it = 0, n_slices = 0;
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
        // single-product rows: the hi pieces only
        mbar_arrive_expect_tx(h_full, (uint32_t)((p.sp ? p.n_kc * RT_CHUNK : L.hist_bytes()) + L.rs_bytes()));
        for (int kc = 0; kc < p.n_kc; ++kc) {
          tma_load_2d(hist + kc * RT_CHUNK, &tmA, h_full, kc * RT_CH, y);
          if (!p.sp) tma_load_2d(hist + (p.n_kc + kc) * RT_CHUNK, &tmA, h_full, p.kpad + kc * RT_CH, y);
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
            mbar_arrive_expect_tx(&w_full[s], (p.sp ? 1 : 2) * RT_CHUNK);
            tma_load_2d(dst, &tmW, &w_full[s], kc * RT_CH, wy);
            if (!p.sp) tma_load_2d(dst + RT_CHUNK, &tmW, &w_full[s], p.kpad + kc * RT_CH, wy);
          }
        }
        // the item's g2 sums and counts, once the previous item's store has read them
        if (ok && (*abort_flag || !mbar_wait(s_empty, par, p.status))) {
          *abort_flag = 1;
          ok = false;
        }
        if (ok) {
          mbar_arrive_expect_tx(s_full, (uint32_t)(2 * p.qg2 * lt * 8));
          tma_load_2d(g2s, &tmG, s_full, (int)tau0, rg * RT_QG);
          tma_load_2d(cns, &tmC, s_full, (int)tau0, rg * RT_QG);
          ++n_slices;
        }
      }
      // never leave the CTA with bulk copies in flight
      if (item_i) mbar_wait(h_full, (item_i - 1) & 1, p.status);
      if (n_slices) mbar_wait(s_full, (n_slices - 1) & 1, p.status);
      for (uint32_t j = (it > (uint32_t)p.wst ? it - p.wst : 0); j < it; ++j)
        mbar_wait(&w_full[j % p.wst], (j / p.wst) & 1, p.status);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // large steps: M = pairs, N = the lt + b - 1 history rows used (a multiple of 16);
      // small steps: M = the 128 history rows, N = the 36 ring pairs of a frame (48)
      // f16 operands (one product) or bf16 pieces (three)
      const int fmt = p.sp ? 0 : 1;
      const uint32_t idesc = EPI == RT_SMALL ? idesc_f16(fmt, RT_ROWS, RT_SMALL_N)
                                             : idesc_f16(fmt, RT_ROWS, min(RT_ROWS, (lt + p.b - 1 + 15) / 16 * 16));
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
            if (p.sp) {
#pragma unroll
              for (int kk = 0; kk < RT_CH / 16; ++kk) {
                if constexpr (EPI == RT_SMALL)
                  tc_mma_f16(d, hhi + 2 * kk, whi + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                else
                  tc_mma_f16(d, whi + 2 * kk, hhi + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
              }
            } else {
#pragma unroll
              for (int kk = 0; kk < RT_CH / 16; ++kk) {  // 16 elements = 32 B per MMA
                if constexpr (EPI == RT_SMALL) {  // D[history row][pair]
                  tc_mma_f16(d, hhi + 2 * kk, whi + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                  tc_mma_f16(d, hhi + 2 * kk, wlo + 2 * kk, idesc, 1u);
                  tc_mma_f16(d, hlo + 2 * kk, whi + 2 * kk, idesc, 1u);
                } else {  // D[pair][history row]
                  tc_mma_f16(d, whi + 2 * kk, hhi + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                  tc_mma_f16(d, wlo + 2 * kk, hhi + 2 * kk, idesc, 1u);
                  tc_mma_f16(d, whi + 2 * kk, hlo + 2 * kk, idesc, 1u);
                }
              }
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
    if constexpr (EPI == RT_SKEW) {  // entries of the skewed buffer no lane writes stay zero
      float* Q = rot + w * (RT_QROWS * RT_QLD);
      for (int x = lane; x < RT_QROWS * RT_QLD; x += 32) Q[x] = 0.f;
      __syncwarp();
    }
    uint32_t item_i = 0, acc_i = 0, stores = 0;
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
      // validity words of the item: for ring ql, words [0, 4) hold the history window
      // starting at bit o_min (the slot of lag tau0 + lt - 1 at frame t0; the fold reads
      // up to bit 63 + lt + 63 < 256), words [4, 6) the step's own frames from bit o_batch
      const long long o_min = (((s_start % p.cap) + p.cap) % p.cap);
      const long long o_batch = p.t0 % p.cap;
      for (int e = et; e < qn * RT_VW; e += 128) {
        const int ql = e / RT_VW, u = e - ql * RT_VW;
        const unsigned long long* vb = p.vbits + (size_t)(q0 + ql) * p.vwords;
        vw[ql * RT_VW + u] = u < 4 ? __ldg(vb + (o_min >> 6) + u) : __ldg(vb + (o_batch >> 6) + (u - 4));
      }
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
        if constexpr (EPI == RT_SMALL) {
          // D[c][ql] = history row c . w_{q0+ql}(t0 + f): the thread holding TMEM lane c
          // owns lag tl = f + lt - 1 - c of every ring, so within a frame no two threads
          // share a bin; it adds D r_q(s_c) for rings ql < qn (r from its own row of rs)
          const int f = mt, c = 32 * w + lane;
          const int c_a = max(f + lt - 1 - tl_max, c_min), c_b = min(f + lt - 1, RT_ROWS - 1);
          const uint32_t tb = tmem_base + buf * RT_ROWS + ((uint32_t)(w * 32) << 16);
          uint32_t v[32], v4[4];
          tmem_ld32(tb, v);
          if (qn > 32) tmem_ld4(tb + 32, v4);  // qn is the same for the whole CTA
          tc_wait_ld();
          if (ok && c >= c_a && c <= c_b) {
            float* bc = bins + (f + lt - 1 - c);  // bin (ql, tl): bc[ql (lt + 1)]
            const float4* r4 = reinterpret_cast<const float4*>(rs + c * p.qb);
            // all bins first, then the products, then all stores (distinct rings' bins
            // never alias, which the compiler cannot prove)
            float bv[RT_QG];
#pragma unroll
            for (int q = 0; q < RT_QG; ++q)
              if (q < qn) bv[q] = bc[q * (lt + 1)];
#pragma unroll
            for (int g = 0; g < RT_QG / 4; ++g) {
              if (4 * g < qn) {
                const float4 r = r4[g];
                const float rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  if (4 * g + u < qn)
                    bv[4 * g + u] = fmaf(__uint_as_float(g < 8 ? v[4 * g + u] : v4[u]), rv[u], bv[4 * g + u]);
              }
            }
#pragma unroll
            for (int q = 0; q < RT_QG; ++q)
              if (q < qn) bc[q * (lt + 1)] = bv[q];
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
          float* brow = bins + ql * (lt + 1);
          if constexpr (EPI == RT_SKEW) {
            // C(f, c) r_q(s_c) of each 32 x 32 block, zero outside the kept lags, stored at
            // row j - i + 32 of the warp's skewed buffer (constant offsets from a per-lane
            // base); row lane then holds block diagonal lane - 32 and row 32 + lane block
            // diagonal lane, summed with 16-byte loads
            float* Q = rot + w * (RT_QROWS * RT_QLD);
            float* qw = Q + (32 - lane) * RT_QLD + lane;
#pragma unroll 1
            for (int c32 = c_lo >> 5; c32 <= (c_hi >> 5); ++c32) {
              uint32_t v[32];
              tmem_ld32(tmem_base + buf * RT_ROWS + ((uint32_t)(w * 32) << 16) + c32 * 32, v);
              tc_wait_ld();
              const int cb = c32 * 32;
              const bool full = __all_sync(0xffffffffu, c_a <= cb && c_b >= cb + 31);  // no lane masks
              const float* rc = rs + (size_t)cb * p.qb + ql;  // r of column cb + jj: rc[jj qb]
              __syncwarp();  // the previous block's row sums are read
              if (full) {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) qw[RT_QLD * jj] = __uint_as_float(v[jj]) * rc[jj * p.qb];
              } else {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                  const int c = cb + jj;
                  qw[RT_QLD * jj] = (c >= c_a && c <= c_b) ? __uint_as_float(v[jj]) * rc[jj * p.qb] : 0.f;
                }
              }
              __syncwarp();
              const float an = skew_row_sum<RT_QLD>(Q, 32 + lane, 0, 32 - lane);
              const float aw = skew_row_sum<RT_QLD>(Q, lane, 32 - lane, 32);
              const int T0 = f0 + lt - 1 - cb;
              const int bn = T0 - lane, bw = T0 - lane + 32;
              if (bn >= 0 && bn < lt) brow[bn] += an;
              if (bw >= 0 && bw < lt) brow[bw] += aw;
            }
          } else {
          float* P = rot + w * 1024;
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
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        // small steps: thread c of frame f and thread c + 1 of frame f + 1 share a bin
        if (EPI == RT_SMALL && mt + 1 < p.n_mt) named_bar_sync(RT_EPI_BAR, 128);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(r_empty);  // the r rows may be replaced
      named_bar_sync(RT_EPI_BAR, 128);     // all bins of the item are complete
      // fold the item's bins into its g2 sums and counts (loaded by TMA, stored back by
      // TMA; one owner per bin).  Pair count of (q, tau) in this step: frames f < b whose
      // frame t0 + f and history frame t0 + f - tau are both defined, a popcount of two
      // windows of the validity bits.
      good = ok && !__any_sync(0xffffffffu, *abort_flag != 0);
      if (good) good = mbar_wait_warp(s_full, item_i & 1, p.status);
      if (!good) {
        *abort_flag = 1;
        ok = false;
      }
      if (ok) {
        // thread et takes lag tl = et mod lt of rings et / lt, et / lt + tpl, ...; the
        // history bits of its lag start at the same offset in every ring's words
        const int sh_b = (int)(o_batch & 63);
        const int tpl = RT_ROWS / lt, tl = et % lt, ql0 = et / lt;
        if (ql0 < tpl && tl <= tl_max) {
          const int o = (int)(o_min & 63) + (lt - 1 - tl);
          float2* g2p = reinterpret_cast<float2*>(g2s);
          int ql = ql0;
          // six rings at a time: all loads, then the sums, then all stores, so the shared
          // memory round trips of the six overlap (the bins, sums and counts of distinct
          // rings never alias, which the compiler cannot prove)
          for (; ql + 5 * tpl < qn; ql += 6 * tpl) {
            int n[6];
            float bv[6];
            float2 acc[6];
            long long cn[6];
#pragma unroll
            for (int u = 0; u < 6; ++u) {
              const int q = ql + u * tpl;
              const unsigned long long* wq = vw + q * RT_VW;
              n[u] = __popcll(bits64(wq + 4, sh_b) & bmask & bits64(wq, o));
              bv[u] = bins[q * (lt + 1) + tl];
              acc[u] = g2p[q * lt + tl];
              cn[u] = cns[q * lt + tl];
            }
#pragma unroll
            for (int u = 0; u < 6; ++u)
              if (n[u]) {
                acc[u] = f32pair_add(acc[u], bv[u]);
                cn[u] += n[u];
              }
#pragma unroll
            for (int u = 0; u < 6; ++u) {
              const int q = ql + u * tpl;
              g2p[q * lt + tl] = acc[u];
              cns[q * lt + tl] = cn[u];
            }
          }
          for (; ql < qn; ql += tpl) {
            const unsigned long long* wq = vw + ql * RT_VW;
            const int n = __popcll(bits64(wq + 4, sh_b) & bmask & bits64(wq, o));
            if (n) {
              g2p[ql * lt + tl] = f32pair_add(g2p[ql * lt + tl], bins[ql * (lt + 1) + tl]);
              cns[ql * lt + tl] += n;
            }
          }
        }
        fence_proxy_async_smem();  // the slice writes, visible to the bulk store
      }
      if (named_bar_sync_or(RT_EPI_BAR, 128, !ok || *abort_flag)) {
        if (et == 0 && stores) bulk_wait_all();
        break;
      }
      if (et == 0) {
        tma_store_2d(&tmG, g2s, (int)tau0, q0);
        tma_store_2d(&tmC, cns, (int)tau0, q0);
        bulk_commit();
        ++stores;
        bulk_wait_read_all();
        mbar_arrive(s_empty);  // the slices may be refilled
      }
      // one decision for all four warps (also orders the fold before the next zeroing)
      if (named_bar_sync_or(RT_EPI_BAR, 128, !ok || *abort_flag)) {
        if (et == 0 && stores) bulk_wait_all();
        break;
      }
    }
    if (et == 0 && stores) bulk_wait_all();  // the sums are in global memory before exit
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 2 * RT_ROWS);
  }
}

}  // namespace

int row_update_tc_smem(int n_kc, int lt, int qb, int wst, int qg2, int epi) {
  return RtLayout{n_kc, lt, qb, wst, qg2, epi}.smem();
}

template <int EPI>
static cudaError_t launch_rt(const CUtensorMap& tmA, const CUtensorMap& tmW, const CUtensorMap& tmR,
                             const CUtensorMap& tmG, const CUtensorMap& tmC, const RowTcParams& p, int grid,
                             cudaStream_t st) {
  const int smem = row_update_tc_smem(p.n_kc, p.lt, p.qb, p.wst, p.qg2, EPI);
  static int attr_bytes = 0;  // the attribute only ever grows
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(row_update_tc_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  row_update_tc_kernel<EPI><<<grid, RT_THREADS, smem, st>>>(tmA, tmW, tmR, tmG, tmC, p);
  return cudaGetLastError();
}

cudaError_t launch_row_update_tc(const CUtensorMap& tmA, const CUtensorMap& tmW, const CUtensorMap& tmR,
                                 const CUtensorMap& tmG, const CUtensorMap& tmC, const RowTcParams& p, int grid,
                                 cudaStream_t st) {
  // the lag tile and the history rows it needs must fit one 128-row operand, and the
  // small-step mode has no buffers for the larger steps' epilogue
  if (p.lt < 2 || (p.lt & 1) || p.lt + p.b - 1 > RT_ROWS || (p.epi == RT_SMALL) != (p.b <= W2_SMALL_B))
    return cudaErrorInvalidValue;
  switch (p.epi) {
    case RT_SKEW:
      return launch_rt<RT_SKEW>(tmA, tmW, tmR, tmG, tmC, p, grid, st);
    case RT_SMALL:
      return launch_rt<RT_SMALL>(tmA, tmW, tmR, tmG, tmC, p, grid, st);
    default:
      return launch_rt<RT_ROT>(tmA, tmW, tmR, tmG, tmC, p, grid, st);
  }
}

// ====================================================================== single frames
// Steps of one frame t (at most 36 rings): for every lag tau < min(W, t + 1), ring q,
//     g2sum_q[tau] += (w_q(t) . a_s) r_q(s),  s = t - tau,
// when r_q(t) > 0 and r_q(s) > 0 (both frames defined).  The pair counts are deferred to
// the frame's count block of 64 frames (a pass over all lags per frame would cost as many
// bytes as the sums); the kernel adds instead one 64th of the lag range of the deferred
// counts of the block before, from the validity bits.  Work item = a tile of 128 lags
// tau0 .. tau0 + 127, history rows s = t - tau0 - 127 + c (c = 0..127): D[c][q] = a_s . w_q
// on the tensor cores (M = the 128 history rows, N = 48 >= 36 ring columns, bf16 hi | lo
// pieces as in the row update kernel, the same products in the same order; or one f16
// product of the hi pieces when the stream computes in f16).  The CTA is
// persistent over its tiles and double-buffers the history rows and their r values, so a
// tile's loads overlap the previous tile's epilogue; the frame's w rows are loaded once.
// Where shared memory allows (two slices for f16 rows, one for bf16 hi | lo rows) the
// producer also loads each tile's running sums (qg2 rings x 128 lags) into a slice as
// soon as the slice is free, so the epilogue reads them without global-load latency.
// Eight epilogue warps (TMEM lane quarter = warp mod 4, rings 18 h .. 18 h + 17 for
// h = (warp - 2) / 4): the thread of lane c adds its lag's product to the running sum (f32
// pair, TwoSum) of each ring and stores it to global memory, 32 consecutive lags per warp
// access.  Each (ring, lag) has one owner: no atomics, the additions of every step in
// stream order.  Every mbarrier wait is bounded.
namespace {

constexpr int R1_EPI_WARPS = 8;
constexpr int R1_THREADS = 64 + 32 * R1_EPI_WARPS;
constexpr int R1_N = 48;                      // MMA N: the 36 ring columns, rounded up to 16
constexpr int R1_WCHUNK = R1_N * RT_CH * 2;   // 6 KB: 48 w rows x 128 B

struct R1Layout {
  int n_kc, qb, np;  // np: pieces per row (2: bf16 hi | lo, 1: f16)
  int sb, qg2;       // sb: staged g2-sum slices (0, 1 or 2) of qg2 rings x 128 lags
  __host__ __device__ int hist_bytes() const { return np * n_kc * RT_CHUNK; }
  __host__ __device__ int w_bytes() const { return np * n_kc * R1_WCHUNK; }
  __host__ __device__ int rs_bytes() const { return (RT_ROWS * qb * 4 + 1023) / 1024 * 1024; }
  __host__ __device__ int sums_bytes() const { return (qg2 * RT_ROWS * 8 + 1023) / 1024 * 1024; }
  __host__ __device__ int smem() const {
    return 1024 + 2 * hist_bytes() + w_bytes() + 2 * rs_bytes() + sb * sums_bytes() + 256;
  }
};

__global__ void __launch_bounds__(R1_THREADS, 1)
    row1_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
                   const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmG,
                   const Row1Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const R1Layout L{p.n_kc, p.qb, p.sp ? 1 : 2, p.sb, p.qg2};
  uint8_t* hist = smem;                                 // [2][hi kc..., lo kc...]
  uint8_t* wbuf = smem + 2 * L.hist_bytes();            // [hi kc..., lo kc...] 48-row chunks
  uint8_t* rsb = wbuf + L.w_bytes();                    // [2][128][qb] r of the rows
  uint8_t* sums = rsb + 2 * L.rs_bytes();               // [sb][qg2][128] staged g2 sums (f32 pairs)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sums + L.sb * L.sums_bytes());
  uint64_t* h_full = bars;       // [2] history rows + their r values landed
  uint64_t* h_empty = bars + 2;  // [2] MMAs and epilogue done with them
  uint64_t* w_full = bars + 4;   // the frame's w rows landed
  uint64_t* tfull = bars + 5;    // [2] accumulator ready
  uint64_t* tempty = bars + 7;   // [2] accumulator read
  uint64_t* mma_done = bars + 9;
  uint64_t* s_full = bars + 10;   // [2] staged sums landed
  uint64_t* s_empty = bars + 12;  // [2] staged sums read
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 14);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long t = p.t;

  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&h_full[b], 1);
      mbar_init(&h_empty[b], 1 + R1_EPI_WARPS);
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], R1_EPI_WARPS);
      mbar_init(&s_full[b], 1);
      mbar_init(&s_empty[b], R1_EPI_WARPS);
    }
    mbar_init(w_full, 1);
    mbar_init(mma_done, 1);
    mbar_fence_init();
    *abort_flag = 0;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 128);
    tmem_relinquish();
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();  // the frame's w, history and r rows

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmW);
      tma_prefetch_desc(&tmR);
      if (p.sb) tma_prefetch_desc(&tmG);
      mbar_arrive_expect_tx(w_full, (uint32_t)L.w_bytes());
      for (int kc = 0; kc < p.n_kc; ++kc) {
        tma_load_2d(wbuf + kc * R1_WCHUNK, &tmW, w_full, kc * RT_CH, 0);
        if (!p.sp) tma_load_2d(wbuf + (p.n_kc + kc) * R1_WCHUNK, &tmW, w_full, p.kpad + kc * RT_CH, 0);
      }
      uint32_t i = 0, ns = 0;  // tiles whose history rows, and whose sums, were loaded
      for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x) {
        const uint32_t bi = i & 1;
        if (*abort_flag || !mbar_wait(&h_empty[bi], ((i >> 1) & 1) ^ 1, p.status)) {
          *abort_flag = 1;
          break;
        }
        const long long s_start = t - (long long)tile * RT_ROWS - (RT_ROWS - 1);
        // before the ring buffer wraps, rows before frame 0 are read as zeros (negative
        // coordinates); afterwards the window is contiguous thanks to the mirrored rows
        const int y = (s_start < 0 && t + 1 <= p.cap) ? (int)s_start : (int)(((s_start % p.cap) + p.cap) % p.cap);
        uint8_t* hb = hist + bi * L.hist_bytes();
        mbar_arrive_expect_tx(&h_full[bi], (uint32_t)(L.hist_bytes() + RT_ROWS * p.qb * 4));
        for (int kc = 0; kc < p.n_kc; ++kc) {
          tma_load_2d(hb + kc * RT_CHUNK, &tmA, &h_full[bi], kc * RT_CH, y);
          if (!p.sp) tma_load_2d(hb + (p.n_kc + kc) * RT_CHUNK, &tmA, &h_full[bi], p.kpad + kc * RT_CH, y);
        }
        tma_load_2d(rsb + bi * L.rs_bytes(), &tmR, &h_full[bi], 0, y);
        ++i;
        if (p.sb) {
          // the tile's running sums (lags tile * 128 .. + 127 of the qg2 rings; lags past
          // the window read as zeros and are not written back), into its slice once the
          // epilogue has read the slice's tile before (two slices: two tiles before)
          const uint32_t sbi = p.sb == 2 ? (ns & 1) : 0u, sph = p.sb == 2 ? ((ns >> 1) & 1) : (ns & 1);
          if (*abort_flag || !mbar_wait(&s_empty[sbi], sph ^ 1, p.status)) {
            *abort_flag = 1;
            break;
          }
          mbar_arrive_expect_tx(&s_full[sbi], (uint32_t)(p.qg2 * RT_ROWS * 8));
          tma_load_2d(sums + sbi * L.sums_bytes(), &tmG, &s_full[sbi], tile * RT_ROWS, 0);
          ++ns;
        }
      }
      // never leave the CTA with bulk copies in flight
      mbar_wait(w_full, 0, p.status);
      for (uint32_t j = (i > 2 ? i - 2 : 0); j < i; ++j) mbar_wait(&h_full[j & 1], (j >> 1) & 1, p.status);
      for (uint32_t j = (ns > (uint32_t)p.sb ? ns - p.sb : 0); j < ns; ++j)
        mbar_wait(&s_full[p.sb == 2 ? (j & 1) : 0u], p.sb == 2 ? ((j >> 1) & 1) : (j & 1), p.status);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(p.sp ? 0 : 1, RT_ROWS, R1_N);
      bool issued = false;
      if (!*abort_flag && mbar_wait(w_full, 0, p.status)) {
        uint32_t i = 0;
        for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++i) {
          const uint32_t bi = i & 1, ph = (i >> 1) & 1;
          if (*abort_flag || !mbar_wait(&tempty[bi], ph ^ 1, p.status) || !mbar_wait(&h_full[bi], ph, p.status)) {
            *abort_flag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + bi * 64;
          const uint8_t* hb = hist + bi * L.hist_bytes();
          for (int kc = 0; kc < p.n_kc; ++kc) {
            const uint64_t hhi = smem_desc_sw128(hb + kc * RT_CHUNK);
            const uint64_t hlo = smem_desc_sw128(hb + (p.n_kc + kc) * RT_CHUNK);
            const uint64_t whi = smem_desc_sw128(wbuf + kc * R1_WCHUNK);
            const uint64_t wlo = smem_desc_sw128(wbuf + (p.n_kc + kc) * R1_WCHUNK);
            if (p.sp) {
#pragma unroll
              for (int kk = 0; kk < RT_CH / 16; ++kk)
                tc_mma_f16(d, hhi + 2 * kk, whi + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            } else {
#pragma unroll
              for (int kk = 0; kk < RT_CH / 16; ++kk) {  // D[history row][ring]
                tc_mma_f16(d, hhi + 2 * kk, whi + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                tc_mma_f16(d, hhi + 2 * kk, wlo + 2 * kk, idesc, 1u);
                tc_mma_f16(d, hlo + 2 * kk, whi + 2 * kk, idesc, 1u);
              }
            }
          }
          tc_commit(&h_empty[bi]);  // the history rows are free once these MMAs complete
          tc_commit(&tfull[bi]);
          issued = true;
        }
      } else {
        *abort_flag = 1;
      }
      if (issued) {  // all issued MMAs complete before TMEM is released
        tc_commit(mma_done);
        mbar_wait(mma_done, 0, p.status);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..9)
    const int quarter = warp & 3, h = (warp - 2) >> 2;
    const int c = quarter * 32 + lane;  // history row = TMEM lane
    const int q0 = 18 * h, qn = max(0, min(18, p.n_q - q0));
    // r of the new frame for this warp's rings
    const long long slot_t = t % p.cap;
    float rt[18];
#pragma unroll
    for (int u = 0; u < 18; ++u) rt[u] = u < qn ? p.Rh[slot_t * p.npad + q0 + u] : 0.f;
    // deferred pair counts (ring, lag) of the block before, spread over the epilogue threads
    // of all CTAs while the first tiles load
    if (p.cf_mask) {
      const long long nl = p.cf_tau1 - p.cf_tau0;
      const long long n = (long long)p.n_q * nl;
      const int nth = R1_EPI_WARPS * 32;
      for (long long e = (long long)blockIdx.x * nth + (threadIdx.x - 64); e < n; e += (long long)gridDim.x * nth) {
        const int q = (int)(e / nl);
        const long long tau = p.cf_tau0 + (e - (long long)q * nl);
        const long long m = masked_pair_count(p.vbits + (size_t)q * p.vwords, p.cap, p.cf_t0, p.cf_mask, tau);
        if (m) p.cnt[(size_t)q * p.Wp + tau] += m;
      }
    }
    uint32_t i = 0;
    for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++i) {
      const uint32_t bi = i & 1, ph = (i >> 1) & 1;
      const bool good = !__any_sync(0xffffffffu, *abort_flag != 0) && mbar_wait_warp(&tfull[bi], ph, p.status) &&
                        mbar_wait_warp(&h_full[bi], ph, p.status);  // warp-uniform outcome
      if (!good) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      uint32_t v[32];  // columns q0 - 16 h .. : ring q0 + u is v[u + 2 h]
      tmem_ld32(tmem_base + bi * 64 + 16 * h + ((uint32_t)(quarter * 32) << 16), v);
      const float* rrow = reinterpret_cast<const float*>(rsb + bi * L.rs_bytes()) + (size_t)c * p.qb + q0;
      float rs[18];
#pragma unroll
      for (int u = 0; u < 18; ++u) rs[u] = u < qn ? rrow[u] : 0.f;
      tc_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&tempty[bi]);
        mbar_arrive(&h_empty[bi]);
      }
      const long long tau = (long long)tile * RT_ROWS + (RT_ROWS - 1 - c);
      const bool live = !(tau >= p.W || tau > t || qn == 0);
      float2* gs = p.g2sum + (size_t)q0 * p.Wp + tau;
      if (p.sb) {
        // the running sums come from the staged slice (ring q0 + u, lag 127 - c of the
        // tile): no load latency in the loop, only the stores of the new sums
        const uint32_t sbi = p.sb == 2 ? bi : 0u, sph = p.sb == 2 ? ph : (i & 1);
        if (!mbar_wait_warp(&s_full[sbi], sph, p.status)) {
          *abort_flag = 1;
          break;
        }
        const float2* ss = reinterpret_cast<const float2*>(sums + sbi * L.sums_bytes()) + (size_t)q0 * RT_ROWS +
                           (RT_ROWS - 1 - c);
        if (live) {
#pragma unroll
          for (int u = 0; u < 18; ++u) {
            if (u < qn && rt[u] > 0.f && rs[u] > 0.f) {
              const float d = __uint_as_float(h ? v[u + 2] : v[u]);  // compile-time register indices
              gs[(size_t)u * p.Wp] = f32pair_add(ss[(size_t)u * RT_ROWS], d * rs[u]);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[sbi]);
        continue;
      }
      if (!live) continue;
      // two batches of nine rings: loads of a batch in flight together, then the adds
#pragma unroll
      for (int u0 = 0; u0 < 18; u0 += 9) {
        bool pr[9];
        float2 acc[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          const int u = u0 + e;
          pr[e] = u < qn && rt[u] > 0.f && rs[u] > 0.f;
          if (pr[e]) acc[e] = gs[(size_t)u * p.Wp];
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          const int u = u0 + e;
          if (pr[e]) {
            const float d = __uint_as_float(h ? v[u + 2] : v[u]);  // compile-time register indices
            gs[(size_t)u * p.Wp] = f32pair_add(acc[e], d * rs[u]);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 128);
  }
}

}  // namespace

int row1_tc_smem(int n_kc, int qb, int sp, int sb, int qg2) { return R1Layout{n_kc, qb, sp ? 1 : 2, sb, qg2}.smem(); }

cudaError_t launch_row1_tc(const CUtensorMap& tmA, const CUtensorMap& tmW, const CUtensorMap& tmR,
                           const CUtensorMap& tmG, const Row1Params& p, int grid, cudaStream_t st) {
  // at most 256 elements of the history rows' pieces (two 64-wide chunks of hi | lo, or four
  // of f16)
  if (p.n_q < 1 || p.n_q > 36 || p.qb < p.n_q || p.n_kc < 1 || p.n_kc > (p.sp ? 4 : 2) ||
      p.sb < 0 || p.sb > 2 || p.qg2 != std::min(36, p.n_q))
    return cudaErrorInvalidValue;
  const int smem = row1_tc_smem(p.n_kc, p.qb, p.sp, p.sb, p.qg2);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  static int attr_bytes = 0;  // the attribute only ever grows
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(row1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  return launch_pdl(row1_tc_kernel, dim3(grid), dim3(R1_THREADS), (size_t)smem, st, tmA, tmW, tmR, tmG, p);
}

}  // namespace xpcs
