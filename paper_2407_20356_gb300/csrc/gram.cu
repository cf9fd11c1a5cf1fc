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
//   warp 1      TMEM allocator and MMA issuer: two f32 tile accumulators in TMEM (128
//               columns each, 256 for tile pairs; single tiles add a merge accumulator)
//   warps 2..5  drain: TMEM -> registers -> C store
//   warps 6..13 TMEM -> registers -> warp shuffles -> diagonal sums
// Any warp may read the TMEM lanes of its quarter (warp id mod 4), so both groups read
// the accumulator independently; they meet only at the TMEM full/empty barriers, and the
// C stores of one tile overlap the diagonal pass of another.
//
// Tile pairs (NP = 2): one MMA of N = 256 multiplies the 128 L rows of block I with the
// 256 R rows of blocks J and J + 1, so one L chunk in shared memory serves two tiles and a
// stage carries 1.5 operand panels per tile instead of 2; the accumulator holds tile
// (I, J) in columns 0..127 and tile (I, J + 1) in columns 128..255.  A work item then runs
// along two neighbouring tile diagonals, delta (even) and delta + 1; where J + 1 is past
// the last tile block the MMA is issued with N = 128 and the second half is not used.
//
// Work item = (q, delta, I0, I1): the tiles (I, I+delta) (and (I, I+delta+1) for pairs)
// for I in [I0, I1).  The diagonal sums of each tile diagonal of an item go to one partial
// slot; no atomics, deterministic.
//
// Merged items (compressed path): every tile of an item lies on one tile diagonal, and
// element (i, j) of each of them belongs to lag 128 delta + j - i, so the diagonal sums of
// the item are the diagonal sums of the SUM of its tiles (the compressed operand rows
// carry both scales, so each accumulator is C itself).  For g2 only (C not stored) the
// MMAs of all its tiles accumulate into one TMEM accumulator.  When C is stored (single
// tiles), the diagonal warps add each tile, as they read it, into a running sum in a
// merge accumulator (TMEM load, f32 add, TMEM store) and shuffle-reduce only the item's
// last sum: one diagonal pass per item instead of one per tile.
//
// C store: C is symmetric, so tile (I, J >= I) is written transposed into the lower
// triangle, straight from registers and fully coalesced.
//
// Diagonal sums: a diagonal warp holds 32 tile rows (its lane quarter) x 64 columns (a
// strip) of the accumulator, lane i = row i.  For strip column c, lane l takes the element
// of row (c + l) mod 32 with one shuffle (source lane (c + l) mod 32, the same register
// c in every lane), so every element a lane receives lies on strip diagonal c - i = -l,
// 32 - l or 64 - l, whichever the wrap of (c + l) says: three per-lane sums per tile
// diagonal, no shared memory.  The eight warps' per-lane sums meet once per work item in
// shared memory and are added in a fixed order.

#include "common.cuh"
#include "internal.h"

namespace xpcs {

namespace {

constexpr int N_DIAG_WARPS = 8;
constexpr int GRAM_THREADS = 64 + 4 * 32 + N_DIAG_WARPS * 32;  // producer, MMA, 4 drain, 8 diagonal warps
constexpr int BAR_BYTES = 256;
constexpr int SMEM_MAX = 227 * 1024;
constexpr int DIAG_BAR = 1;
constexpr int MAX_STAGE = 4;  // deeper rings measured slower for the C-storing calls                        // named barrier of the eight diagonal warps

// Shared-memory layout, pipeline depth and accumulators of one configuration: NP = tiles
// per accumulator (1, or 2 for tile pairs).  As many operand stages as fit, at most
// MAX_STAGE; two TMEM tile accumulators, and for single tiles a merge accumulator of 128
// columns beside them.
template <int NP>
struct GramCfg {
  static constexpr int red_floats = NP * N_DIAG_WARPS * 3 * 32;  // per-warp sums of a work item
  static constexpr int diag_bytes = red_floats * 4;
  static constexpr int chunk_l = TILE * KCH * 2;       // L chunk: 128 rows x 128 B
  static constexpr int chunk_r = NP * TILE * KCH * 2;  // R chunk: 128 NP rows x 128 B
  static constexpr int stage_bytes = chunk_l + chunk_r;
  static constexpr int fixed = 1024 + diag_bytes + BAR_BYTES;
  static constexpr int fit = (SMEM_MAX - fixed) / stage_bytes;
  static constexpr int nstage = fit > MAX_STAGE ? MAX_STAGE : fit;
  static constexpr int bytes = fixed + nstage * stage_bytes;
  static constexpr int nacc = 2;                        // tile accumulators of NP x 128 columns
  static constexpr uint32_t macc_col = nacc * NP * TILE;  // merge accumulator (single tiles)
  static constexpr uint32_t tmem_cols = 512;
  static_assert(nstage >= 3, "at least three operand stages");
  static_assert(bytes <= SMEM_MAX, "shared memory of one CTA");
  static_assert(NP == 2 || macc_col + TILE <= tmem_cols, "the merge accumulator fits the TMEM");
  static_assert(2 * MAX_STAGE + 2 * 4 + 1 <= BAR_BYTES / 8 - 1, "barriers and the TMEM slot fit");
};

// Stores one 32-column chunk of a tile row: element (i, j) of tile (I, J) is C(t1, t2)
// with t1 = 128 I + i, t2 = 128 J + j, written transposed at [t2][t1] (lower triangle) so
// that for a fixed j the warp's 32 lanes write 32 consecutive values.  Raw mode also
// writes the exact integer Gram N and scales the accumulator by r(t1) r(t2).
__device__ __forceinline__ void store_chunk(const GramParams& p, uint32_t (&v)[32], int q, int J, int col0,
                                            long long t1, float ri, const float* rq, bool bad, bool interior) {
  const long long T = p.T;
  const float* rj = rq + (size_t)J * TILE + col0;
  const size_t obase = ((size_t)q * T + (size_t)J * TILE + col0) * T + (size_t)t1;
  if (p.raw) {
    if (p.Nout) {
      if (interior) {
#pragma unroll
        for (int j = 0; j < 32; ++j) p.Nout[obase + (size_t)j * T] = (long long)__uint_as_float(v[j]);
      } else if (t1 < T) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if ((long long)J * TILE + col0 + j < T) p.Nout[obase + (size_t)j * T] = (long long)__uint_as_float(v[j]);
      }
    }
    if (!p.C) return;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __float_as_uint((__uint_as_float(v[j]) * ri) * __ldg(rj + j));
  }
  if (interior) {
#pragma unroll
    for (int j = 0; j < 32; ++j) __stcs(p.C + obase + (size_t)j * T, __uint_as_float(v[j]));
  } else if (t1 < T) {
    const bool row_ok = ri > 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if ((long long)J * TILE + col0 + j < T) {
        float val = __uint_as_float(v[j]);
        if (bad && !(row_ok && __ldg(rj + j) > 0.f)) val = __int_as_float(0x7fc00000);
        __stcs(p.C + obase + (size_t)j * T, val);
      }
    }
  }
}

// Tiles of work item w that share one accumulator ("unit" u): one tile (pair) per unit,
// or the whole item when merged.
struct UnitRange {
  int I_begin, I_end;
};
__device__ __forceinline__ UnitRange unit_range(const GramParams& p, const int4& w, int u) {
  return p.merge ? UnitRange{w.z, w.w} : UnitRange{w.z + u, w.z + u + 1};
}
__device__ __forceinline__ int units_of(const GramParams& p, const int4& w) { return p.merge ? 1 : w.w - w.z; }

// Work item i: from the list, or computed for a stream's raw row update (a ring of blocks)
__device__ __forceinline__ int4 item_at(const GramParams& p, int i) {
  if (p.items) return p.items[i];
  const int qi = i / p.ring_nd, d = i - qi * p.ring_nd;
  const int q = (p.sm && p.pairs) ? 2 * qi : qi;  // ring pairs of a stream step
  const int I = ((p.ring_J - d) % p.ring_nb + p.ring_nb) % p.ring_nb;
  return make_int4(q, d, I, I + 1);
}
// Whether the second half of a tile pair exists: tile (I, I + delta + 1) offline, ring q + 1
// in a stream step
template <int NP>
__device__ __forceinline__ bool second_half(const GramParams& p, int q, int I, int delta) {
  return (NP == 2 && p.sm) ? q + 1 < p.sm_nq : I + delta + 1 < p.nT;
}
// Column block of tile (I, I + delta): wraps around the ring of a stream's history
__device__ __forceinline__ int col_block(const GramParams& p, int I, int delta) {
  const int J = I + delta;
  return p.ring_nb ? J % p.ring_nb : J;
}

template <int NP>
__global__ void __launch_bounds__(GRAM_THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmR,
               const GramParams p) {
  using CF = GramCfg<NP>;
  constexpr int NSTAGE = CF::nstage;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  float* diag_smem = reinterpret_cast<float*>(smem + NSTAGE * CF::stage_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * CF::stage_bytes + CF::diag_bytes);
  uint64_t* full = bars;                    // [NSTAGE]
  uint64_t* empty = bars + NSTAGE;          // [NSTAGE]
  uint64_t* tfull = bars + 2 * NSTAGE;                // [nacc]
  uint64_t* tempty = bars + 2 * NSTAGE + CF::nacc;    // [nacc]
  uint64_t* mma_done = bars + 2 * NSTAGE + 2 * CF::nacc;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < CF::nacc; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], p.partials ? 4 + N_DIAG_WARPS : 4);  // drain (+ diagonal) warps
    }
    mbar_init(mma_done, 1);
    mbar_fence_init();
    *abort_flag = 0;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, CF::tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const bool sm = NP == 2 && p.sm;        // stream steps always run as ring pairs
  const bool rm = NP == 1 && p.rmerge;    // per-item running sum of the tiles in TMEM

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmL);
      tma_prefetch_desc(&tmR);
      uint32_t it = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const int4 w = item_at(p, item);
        const int q = w.x, delta = w.y;
        const int nk = sm ? p.sm_nk : p.k_chunks[q];
        const int nc = p.split ? 2 * nk : nk;  // chunks per tile
        const int koff = sm ? 0 : p.k_off[q];
        const int rowbase = sm ? 0 : q * p.ring_rows;
        for (int I = w.z; I < w.w && ok; ++I) {
          const int J = col_block(p, I, delta);
          const int rrow = sm ? q * TILE : rowbase + J * TILE;  // first row of the R box
          for (int c = 0; c < nc; ++c, ++it) {
            const uint32_t s = it % NSTAGE, ph = (it / NSTAGE) & 1;
            if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1, p.status)) {
              *abort_flag = 1;
              ok = false;
              break;
            }
            // split: chunk 2 kc holds the hi pieces of K-block kc, chunk 2 kc + 1 the lo pieces
            const int x = koff + (p.split ? ((c & 1) * nk + (c >> 1)) * KCH : c * KCH);
            uint8_t* st = stages + s * CF::stage_bytes;
            mbar_arrive_expect_tx(&full[s], CF::stage_bytes);
            tma_load_2d(st, &tmL, &full[s], x, rowbase + I * TILE);
            // NP x 128 rows of R (rows past the matrix are filled with zeros)
            tma_load_2d(st + CF::chunk_l, &tmR, &full[s], x, rrow);
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
      const uint32_t idesc1 = idesc_f16(p.fmt, TILE, TILE);
      const uint32_t idesc2 = idesc_f16(p.fmt, TILE, NP * TILE);
      uint32_t it = 0, unit = 0;
      bool ok = true, issued = false;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const int4 w = item_at(p, item);
        const int nk = sm ? p.sm_nk : p.k_chunks[w.x];
        const int nc = p.split ? 2 * nk : nk;
        const int n_units = units_of(p, w);
        for (int u = 0; u < n_units && ok; ++u, ++unit) {
          const uint32_t b = unit % CF::nacc, tph = (unit / CF::nacc) & 1;
          if (*abort_flag || !mbar_wait(&tempty[b], tph ^ 1, p.status)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + b * (NP * TILE);
          const UnitRange ur = unit_range(p, w, u);
          bool first = true;  // the unit's first MMA overwrites the accumulator
          for (int I = ur.I_begin; I < ur.I_end && ok; ++I) {
            // tile pair when the second tile exists, else N = 128 (first half only)
            const uint32_t idesc = (NP == 2 && second_half<NP>(p, w.x, I, w.y)) ? idesc2 : idesc1;
            for (int c = 0; c < nc; ++c, ++it) {
              const uint32_t s = it % NSTAGE, ph = (it / NSTAGE) & 1;
              if (*abort_flag || !mbar_wait(&full[s], ph, p.status)) {
                *abort_flag = 1;
                ok = false;
                break;
              }
              tc_fence_after();
              const uint8_t* st = stages + s * CF::stage_bytes;
              const uint64_t ad = smem_desc_sw128(st);
              const uint64_t bd = smem_desc_sw128(st + CF::chunk_l);
              if (!p.split) {
#pragma unroll
                for (int kk = 0; kk < KCH / 16; ++kk)  // 16 elements = 32 B per MMA
                  tc_mma_f16(d, ad + 2 * kk, bd + 2 * kk, idesc, (first && kk == 0) ? 0u : 1u);
                tc_commit(&empty[s]);
              } else if ((c & 1) == 0) {
                // hi pieces: L_hi R_hi now; the stage stays until the lo pieces arrive
#pragma unroll
                for (int kk = 0; kk < KCH / 16; ++kk)
                  tc_mma_f16(d, ad + 2 * kk, bd + 2 * kk, idesc, (first && kk == 0) ? 0u : 1u);
              } else {
                // lo pieces: L_lo R_hi and L_hi R_lo with the previous stage's hi pieces
                const uint32_t sp = (it - 1) % NSTAGE;
                const uint8_t* sth = stages + sp * CF::stage_bytes;
                const uint64_t adh = smem_desc_sw128(sth);
                const uint64_t bdh = smem_desc_sw128(sth + CF::chunk_l);
#pragma unroll
                for (int kk = 0; kk < KCH / 16; ++kk) {
                  tc_mma_f16(d, ad + 2 * kk, bdh + 2 * kk, idesc, 1u);
                  tc_mma_f16(d, adh + 2 * kk, bd + 2 * kk, idesc, 1u);
                }
                tc_commit(&empty[sp]);
                tc_commit(&empty[s]);
              }
              first = false;
              issued = true;
            }
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
  } else if (warp < 6) {
    // ------------------------------------------------------------ drain warps (2..5)
    // One warp per TMEM lane quarter: thread = tile row i.  TMEM -> registers -> C store,
    // transposed into the lower triangle: for a fixed column j the warp's 32 lanes write
    // 32 consecutive floats of output row t2.  (Merged units store no C: nothing to do.)
    const int quarter = warp & 3;
    const int i_row = quarter * 32 + lane;
    const long long T = p.T;
    const bool work = (p.C || p.Nout) && !p.merge;
    uint32_t unit = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
      const int4 w = item_at(p, item);
      const int q = w.x, delta = w.y;
      const float* rq = p.r + (size_t)q * p.T_pad;
      const int n_units = units_of(p, w);
      for (int u = 0; u < n_units; ++u, ++unit) {
        const int I = unit_range(p, w, u).I_begin;
        const uint32_t b = unit % CF::nacc, tph = (unit / CF::nacc) & 1;
        // per-tile metadata first, so its load latency overlaps the wait for the MMA
        const long long t1 = (long long)I * TILE + i_row;
        const float ri = work ? rq[t1] : 0.f;
        const int nh = (NP == 2 && I + delta + 1 < p.nT) ? 2 : 1;
        bool bad[NP], interior[NP];
#pragma unroll
        for (int h2 = 0; h2 < NP; ++h2) {
          const int J = I + delta + h2;
          bad[h2] = work && h2 < nh && (p.blk_bad[(size_t)q * p.nT + I] | p.blk_bad[(size_t)q * p.nT + J]);
          interior[h2] = !bad[h2] && (long long)(I + 1) * TILE <= T && (long long)(J + 1) * TILE <= T;
        }
        if (!mbar_wait_warp(&tfull[b], tph, p.status)) {  // warp-uniform outcome
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        if (work) {
#pragma unroll
          for (int h2 = 0; h2 < NP; ++h2) {
            if (h2 >= nh) break;
            const int J = I + delta + h2;
            const uint32_t tbase = tmem_base + b * (NP * TILE) + h2 * TILE + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
            for (int cc = 0; cc < 4; cc += 2) {
              uint32_t v0[32], v1[32];
              tmem_ld32(tbase + 32 * cc, v0);
              tmem_ld32(tbase + 32 * cc + 32, v1);
              tc_wait_ld();
              store_chunk(p, v0, q, J, 32 * cc, t1, ri, rq, bad[h2], interior[h2]);
              store_chunk(p, v1, q, J, 32 * cc + 32, t1, ri, rq, bad[h2], interior[h2]);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
    }
  } else if (p.partials) {
    // ------------------------------------------------------------ diagonal warps (6..13)
    // Warp dw (0..7) covers TMEM lane quarter r = warp mod 4 (tile rows 32 r ..) and
    // column half h = dw / 4 (strip columns 64 h .. 64 h + 63) of each tile of the
    // accumulator.  Lane l gathers, for every strip column c, the element of row
    // (c + l) mod 32 (a shuffle per column), which lies on strip diagonal c - i = 32 m - l
    // for m = 0, 1 or 2; it keeps one sum per m and tile diagonal of the item.  Strip
    // diagonal 32 m - l is diagonal 32 (e - 1) + (32 - l) of the slot layout below.
    const int dw = warp - 6;
    const int r = warp & 3;
    const int h = dw >> 2;
    float* red = diag_smem;  // [half][warp][k][lane]: strip diagonal 32 (k - 1) + lane
    const int i_row = r * 32 + lane;
    uint32_t unit = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
      const int4 w = item_at(p, item);
      const int q = w.x, delta = w.y;
      const float* rq = p.r + (size_t)q * p.T_pad;
      // the item's second tile diagonal (pairs; in a stream step the second ring) holds tiles
      const bool has2 = NP == 2 && second_half<NP>(p, q, w.z, delta);
      float acc[NP][3];
#pragma unroll
      for (int h2 = 0; h2 < NP; ++h2) acc[h2][0] = acc[h2][1] = acc[h2][2] = 0.f;
      const int n_units = units_of(p, w);
      for (int u = 0; u < n_units && ok; ++u, ++unit) {
        const int I = unit_range(p, w, u).I_begin;
        const uint32_t b = unit % CF::nacc, tph = (unit / CF::nacc) & 1;
        const float ri = !p.raw ? 1.f
                         : sm ? p.r[((size_t)I * TILE + i_row) * p.r_ld + q]
                                : rq[(size_t)I * TILE + i_row];
        // a stream step's second half is ring q + 1, with its own row scale
        const float ri2 = (NP == 2 && sm && has2) ? p.r[((size_t)I * TILE + i_row) * p.r_ld + q + 1] : ri;
        if (*abort_flag || !mbar_wait_warp(&tfull[b], tph, p.status)) {  // warp-uniform outcome
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const int nh = (NP == 2 && (p.merge || sm ? has2 : I + delta + 1 < p.nT)) ? 2 : 1;
#pragma unroll
        for (int h2 = 0; h2 < NP; ++h2) {
          if (h2 >= nh) break;
          const bool last = h2 == nh - 1;  // TMEM is released after the unit's last load
          // a stream step's w block is zero outside the step's frames: a strip without any
          // of them adds nothing
          if (sm && !(p.sm_c0 < 64 * h + 64 && p.sm_c1 > 64 * h)) {
            if (last) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&tempty[b]);
            }
            continue;
          }
          const uint32_t tbase =
              tmem_base + b * (NP * TILE) + h2 * TILE + ((uint32_t)(r * 32) << 16) + 64 * h;
          const float* rj = sm ? nullptr
                                 : (p.rc ? p.rc + (size_t)q * p.T_pad : rq) +
                                       (size_t)col_block(p, I, delta + h2) * TILE + 64 * h;
          uint32_t v0[32], v1[32];
          tmem_ld32(tbase, v0);
          tmem_ld32(tbase + 32, v1);
          tc_wait_ld();
          if (last) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
          }
          if (rm) {
            // compressed tiles with C stored: add the strip to the item's running sum in the
            // merge accumulator (the operand rows carry both scales, so each tile is C
            // itself); the item's last tile reduces the sum along its diagonals
            const uint32_t mbase = tmem_base + CF::macc_col + ((uint32_t)(r * 32) << 16) + 64 * h;
            if (u > 0) {
              uint32_t m[32];
              tmem_ld32(mbase, m);
              tc_wait_ld();
#pragma unroll
              for (int j = 0; j < 32; ++j) v0[j] = __float_as_uint(__uint_as_float(m[j]) + __uint_as_float(v0[j]));
              tmem_ld32(mbase + 32, m);
              tc_wait_ld();
#pragma unroll
              for (int j = 0; j < 32; ++j) v1[j] = __float_as_uint(__uint_as_float(m[j]) + __uint_as_float(v1[j]));
            }
            if (u < n_units - 1) {
              tmem_st32(mbase, v0);
              tmem_st32(mbase + 32, v1);
              tc_wait_st();  // written before the next tile reads it (and before v0, v1 are reused)
              continue;
            }
          } else if (sm) {  // stream step: the w columns carry their own scale
            const float s = h2 ? ri2 : ri;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              v0[j] = __float_as_uint(__uint_as_float(v0[j]) * s);
              v1[j] = __float_as_uint(__uint_as_float(v1[j]) * s);
            }
          } else if (p.raw) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              v0[j] = __float_as_uint((__uint_as_float(v0[j]) * ri) * __ldg(rj + j));
              v1[j] = __float_as_uint((__uint_as_float(v1[j]) * ri) * __ldg(rj + 32 + j));
            }
          }
          // column c of the strip from row (c + lane) mod 32: strip diagonal 32 m - lane
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int src = (lane + j) & 31;
            const float x0 = __shfl_sync(0xffffffffu, __uint_as_float(v0[j]), src);
            const float x1 = __shfl_sync(0xffffffffu, __uint_as_float(v1[j]), src);
            if (lane + j >= 32) {
              acc[h2][1] += x0;
              acc[h2][2] += x1;
            } else {
              acc[h2][0] += x0;
              acc[h2][1] += x1;
            }
          }
        }
      }
      // lane l > 0 holds strip diagonals 32 (k - 1) + (32 - l); lane 0 holds 0 and 32 (k = 1,
      // 2), and strip diagonal -32 (k = 0, lane 0) has no element
      const int lp = (32 - lane) & 31;
#pragma unroll
      for (int h2 = 0; h2 < NP; ++h2)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          red[((h2 * N_DIAG_WARPS + dw) * 3 + k) * 32 + lp] = lane ? acc[h2][k] : (k ? acc[h2][k - 1] : 0.f);
      named_bar_sync(DIAG_BAR, N_DIAG_WARPS * 32);
      if (ok && !*abort_flag) {
        // warp dw finishes diagonals 32 (dw - 4) + lane of each tile diagonal, adding the
        // warps in a fixed order
        const int e = dw - 4;
        const int chunk = w.z / p.CH;
#pragma unroll
        for (int h2 = 0; h2 < NP; ++h2) {
          if (h2 == 1 && !has2) break;
          const float* rh = red + h2 * N_DIAG_WARPS * 3 * 32;
          float sum = 0.f;
#pragma unroll
          for (int u = 0; u < N_DIAG_WARPS; ++u) {
            const int k = e - (2 * (u >> 2) - ((u + 6) & 3) - 1);
            if (k >= 0 && k < 3) sum += rh[(u * 3 + k) * 32 + lane];
          }
          // offline: tile diagonal delta + h2 of ring q; stream step: ring q + h2, diagonal delta
          const int sq = sm ? q + h2 : q, sd = sm ? delta : delta + h2;
          float* slot = p.partials + (((size_t)sq * p.nT + sd) * p.maxC + chunk) * DIAG_SLOTS;
          slot[32 * dw + lane] = sum;
        }
      }
      named_bar_sync(DIAG_BAR, N_DIAG_WARPS * 32);  // red is free again
      if (!ok || *abort_flag) break;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, CF::tmem_cols);
  }
}

}  // namespace

int gram_smem_bytes() { return GramCfg<1>::bytes > GramCfg<2>::bytes ? GramCfg<1>::bytes : GramCfg<2>::bytes; }

template <int NP>
static cudaError_t launch_gram_t(const CUtensorMap& tmL, const CUtensorMap& tmR, const GramParams& p, int grid,
                                 cudaStream_t st) {
  constexpr int smem = GramCfg<NP>::bytes;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  gram_tc_kernel<NP><<<grid, GRAM_THREADS, smem, st>>>(tmL, tmR, p);
  return cudaGetLastError();
}

// The tile pairing is a parameter of the call (autotuned per workload shape).
cudaError_t launch_gram(const CUtensorMap& tmL, const CUtensorMap& tmR, const GramParams& p, int grid,
                        cudaStream_t st) {
  return p.pairs ? launch_gram_t<2>(tmL, tmR, p, grid, st) : launch_gram_t<1>(tmL, tmR, p, grid, st);
}

}  // namespace xpcs
