// Two-time correlation tile kernel (raw exact path and compressed path), sm_103a.
//
// For every ring q and every output tile (I, J = I + delta) of the upper triangle of
// the T x T two-time matrix it computes the ring Gram tile
//     acc(t1, t2) = sum_k L_q(t1, k) R_q(t2, k)
// on the tcgen05 tensor cores (Eq. 2 for raw counts, Eq. 10 for coefficients), then in
// the epilogue forms C_q (Eq. 1), optionally stores it, and reduces it along its
// diagonals into per-lag partial sums for g2.
//
// Raw mode: L = R = ring-sorted counts in bf16 (exact integers <= 256); the f32
// accumulator is exact while every partial sum stays below 2^24, which the ingest step
// proves per ring from max_t sum_p x^2 (all terms are non-negative, so every partial
// sum of N(t1,t2) is bounded by sqrt(N(t1,t1) N(t2,t2))).  C = acc * r(t1) * r(t2)
// with r = sqrt(M_q)/S_q.
// Compressed mode: the rows of L and R already carry r(t), so acc is C itself.
//
// Structure (one CTA per SM, persistent over work items):
//   warp 0      TMA producer: 64-wide K chunks of the L and R row blocks, NSTAGE ring
//   warp 1      TMEM allocator and MMA issuer: 128x128 f32 accumulator, 2 TMEM buffers
//   warps 2..9  epilogue: TMEM -> registers -> skewed shared tile -> (C store, diagonal sums)
//
// Work item = (q, delta, I0, I1): the tiles (I, I+delta) for I in [I0, I1) of one tile
// diagonal.  Its diagonal sums go to one partial slot; no atomics, deterministic.
//
// Skewed tile: element (i, j) of the tile is written to shared row i, column
// 128 - i + j.  Column c then holds the tile diagonal j - i = c - 128 (c >= 128: upper
// diagonals 0..127; c < 128: lower diagonals -128..-1).  Cells a row never writes stay
// zero, so summing a column over a warp-uniform row range gives the diagonal sum.
#include "common.cuh"
#include "internal.h"

namespace xpcs {

namespace {

constexpr int NSTAGE = 2;
constexpr int CHUNK_BYTES = TILE * KCH * 2;        // one operand chunk: 128 rows x 128 B
constexpr int STAGE_BYTES = 2 * CHUNK_BYTES;       // L + R
constexpr int SKEW_LD = 258;                       // floats per skewed row (257 = 1 mod 32)
constexpr int SKEW_BYTES = TILE * SKEW_LD * 4;
constexpr int N_EPI_WARPS = 8;
constexpr int N_EPI_THREADS = 32 * N_EPI_WARPS;
constexpr int GRAM_THREADS = 64 + N_EPI_THREADS;
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES = 1024 + NSTAGE * STAGE_BYTES + SKEW_BYTES + BAR_BYTES;
constexpr uint32_t TMEM_COLS = 256;                // two 128-column accumulators
constexpr int EPI_BAR = 1;                         // named barrier id for the epilogue warps

__global__ void __launch_bounds__(GRAM_THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmR,
               const GramParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  float* skew = reinterpret_cast<float*>(smem + NSTAGE * STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES + SKEW_BYTES);
  uint64_t* full = bars;                    // [NSTAGE]
  uint64_t* empty = bars + NSTAGE;          // [NSTAGE]
  uint64_t* tfull = bars + 2 * NSTAGE;      // [2]
  uint64_t* tempty = bars + 2 * NSTAGE + 2; // [2]
  uint64_t* mma_done = bars + 2 * NSTAGE + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSTAGE + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], N_EPI_WARPS);
    }
    mbar_init(mma_done, 1);
    mbar_fence_init();
    *abort_flag = 0;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  for (int i = threadIdx.x; i < TILE * SKEW_LD; i += blockDim.x) skew[i] = 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmL);
      tma_prefetch_desc(&tmR);
      uint32_t it = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const int4 w = p.items[item];
        const int q = w.x, delta = w.y;
        const int nk = p.k_chunks[q];
        const int koff = p.k_off[q];
        const int rowbase = q * p.ring_rows;
        for (int I = w.z; I < w.w && ok; ++I) {
          const int J = I + delta;
          for (int c = 0; c < nk; ++c, ++it) {
            const uint32_t s = it % NSTAGE, ph = (it / NSTAGE) & 1;
            if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1, p.status)) {
              *abort_flag = 1;
              ok = false;
              break;
            }
            uint8_t* st = stages + s * STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(st, &tmL, &full[s], koff + c * KCH, rowbase + I * TILE);
            tma_load_2d(st + CHUNK_BYTES, &tmR, &full[s], koff + c * KCH, rowbase + J * TILE);
          }
        }
      }
      // drain: never leave the CTA with bulk copies in flight
      for (uint32_t j = (it > NSTAGE ? it - NSTAGE : 0); j < it; ++j)
        mbar_wait(&full[j % NSTAGE], (j / NSTAGE) & 1, p.status);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(p.fmt, TILE, TILE);
      uint32_t it = 0, tile = 0;
      bool ok = true, issued = false;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const int4 w = p.items[item];
        const int nk = p.k_chunks[w.x];
        for (int I = w.z; I < w.w && ok; ++I, ++tile) {
          const uint32_t b = tile & 1, tph = (tile >> 1) & 1;
          if (*abort_flag || !mbar_wait(&tempty[b], tph ^ 1, p.status)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + b * TILE;
          for (int c = 0; c < nk; ++c, ++it) {
            const uint32_t s = it % NSTAGE, ph = (it / NSTAGE) & 1;
            if (*abort_flag || !mbar_wait(&full[s], ph, p.status)) {
              *abort_flag = 1;
              ok = false;
              break;
            }
            tc_fence_after();
            const uint8_t* st = stages + s * STAGE_BYTES;
            const uint64_t ad = smem_desc_sw128(st);
            const uint64_t bd = smem_desc_sw128(st + CHUNK_BYTES);
#pragma unroll
            for (int kk = 0; kk < KCH / 16; ++kk)  // 16 elements = 32 B per MMA
              tc_mma_f16(d, ad + 2 * kk, bd + 2 * kk, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            issued = true;
            tc_commit(&empty[s]);
          }
          if (!ok) break;
          tc_commit(&tfull[b]);
        }
      }
      if (issued) {  // all issued MMAs complete before TMEM is released
        tc_commit(mma_done);
        mbar_wait(mma_done, 0, p.status);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;              // 0..7
    const int quarter = warp & 3;         // TMEM lane quarter this warp may access
    const int h = ew >> 2;                // column half of the tile
    const int e = ew * 32 + lane;         // skew column owned in the diagonal pass
    const int i_row = quarter * 32 + lane;  // tile row owned when draining TMEM
    const int dlo = (ew >= 4) ? 0 : 97 - 32 * ew;
    const int dhi = (ew >= 4) ? 256 - 32 * ew : TILE;
    const long long T = p.T;
    uint32_t tile = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
      const int4 w = p.items[item];
      const int q = w.x, delta = w.y;
      const float* rq = p.r + (size_t)q * p.T_pad;
      float acc = 0.f;
      for (int I = w.z; I < w.w; ++I, ++tile) {
        const int J = I + delta;
        const uint32_t b = tile & 1, tph = (tile >> 1) & 1;
        if (!mbar_wait(&tfull[b], tph, p.status)) *abort_flag = 1;
        named_bar_sync(EPI_BAR, N_EPI_THREADS);
        if (*abort_flag) {
          ok = false;
          break;
        }
        tc_fence_after();
        const long long t1 = (long long)I * TILE + i_row;
        const float ri = p.raw ? rq[t1] : 1.f;
        float* dst_row = skew + i_row * SKEW_LD + TILE - i_row;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int col0 = 64 * h + 32 * cc;
          uint32_t v[32];
          tmem_ld32(tmem_base + b * TILE + ((uint32_t)(quarter * 32) << 16) + col0, v);
          tc_wait_ld();
          if (p.raw) {
            const float* rj = rq + (size_t)J * TILE + col0;
            if (p.Nout && t1 < T) {
              long long* nrow = p.Nout + ((size_t)q * T + t1) * T + (size_t)J * TILE + col0;
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if ((long long)J * TILE + col0 + j < T) nrow[j] = (long long)__uint_as_float(v[j]);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) dst_row[col0 + j] = (__uint_as_float(v[j]) * ri) * __ldg(rj + j);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) dst_row[col0 + j] = __uint_as_float(v[j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
        named_bar_sync(EPI_BAR, N_EPI_THREADS);

        // diagonal sums of this tile: column e over the warp's row range
        {
          float s0 = 0.f, s1 = 0.f;
          const float* col = skew + e;
          int i = dlo;
          for (; i + 1 < dhi; i += 2) {
            s0 += col[i * SKEW_LD];
            s1 += col[(i + 1) * SKEW_LD];
          }
          if (i < dhi) s0 += col[i * SKEW_LD];
          acc += s0 + s1;
        }

        // C store: rows of the tile, coalesced along t2, NaN for undefined pairs
        if (p.C) {
          const bool bad = p.blk_bad[(size_t)q * p.nT + I] | p.blk_bad[(size_t)q * p.nT + J];
          for (int rr = 0; rr < TILE / N_EPI_WARPS; ++rr) {
            const int i = ew * (TILE / N_EPI_WARPS) + rr;
            const long long tt1 = (long long)I * TILE + i;
            if (tt1 >= T) break;
            const float* src = skew + i * SKEW_LD + TILE - i;
            float* crow = p.C + ((size_t)q * T + tt1) * T + (size_t)J * TILE;
            const bool row_ok = !bad || rq[tt1] > 0.f;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              const int j = lane + 32 * m;
              const long long tt2 = (long long)J * TILE + j;
              if (tt2 < T) {
                float val = src[j];
                if (bad && !(row_ok && rq[tt2] > 0.f)) val = __int_as_float(0x7fc00000);
                __stcs(crow + j, val);
              }
            }
          }
        }
        named_bar_sync(EPI_BAR, N_EPI_THREADS);
      }
      if (!ok) break;
      if (p.partials) {
        const int chunk = w.z / p.CH;
        p.partials[(((size_t)q * p.nT + delta) * p.maxC + chunk) * DIAG_SLOTS + e] = acc;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

}  // namespace

int gram_smem_bytes() { return SMEM_BYTES; }

cudaError_t launch_gram(const CUtensorMap& tmL, const CUtensorMap& tmR, const GramParams& p, int grid,
                        cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  gram_tc_kernel<<<grid, GRAM_THREADS, SMEM_BYTES, st>>>(tmL, tmR, p);
  return cudaGetLastError();
}

}  // namespace xpcs
