// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <utility>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/xpcs.h"

namespace xpcs {

// status-word codes written by kernels (the host maps them to xpcs_status)
enum : uint32_t {
  XPCS_DEV_OK = 0,
  XPCS_DEV_TIMEOUT = 1,  // a bounded wait expired
  XPCS_DEV_RANGE = 2,    // input outside the exact range of the chosen path
};

constexpr int TILE = 128;        // frames per tile side
constexpr int KCH = 64;          // 16-bit K elements per pipeline chunk (128 bytes)
constexpr int DIAG_SLOTS = 256;  // local diagonal slots per (ring, tile-diagonal, chunk)
constexpr int CHUNK_TILES = 8;   // default tiles per work item along a tile diagonal

// ------------------------------------------------------------------ Gram kernel

// Launch of a kernel with programmatic stream serialization (its threads call pdl_wait
// before they read what the kernel ahead of it wrote).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

struct GramParams {
  int T;                   // frames
  int nT;                  // ceil(T / 128)
  int T_pad;               // nT * 128, rows per ring in r[] (and per ring block of operands)
  int maxC;                // chunk slots per (ring, tile diagonal)
  int CH;                  // tiles per chunk
  int n_items;
  const int4* items;       // (q, delta, I0, I1)
  const int* k_off;        // per ring: K offset (elements) into the operand matrices
  const int* k_chunks;     // per ring: number of 64-wide K chunks, >= 1
  int ring_rows;           // operand row offset between rings (0 when rings share rows)
  int fmt;                 // 0 = f16, 1 = bf16
  int split;               // 1: operand rows are [hi | lo] pieces of k_chunks chunks each;
                           //    C = L_hi R_hi + L_lo R_hi + L_hi R_lo
  int raw;                 // 1: C = acc * r(t1) * r(t2); 0: operands already scaled
  int pairs;               // 1: tile pairs (I, J), (I, J + 1) per accumulator (N = 256 MMA);
                           //    items then cover the tile diagonals delta (even) and delta + 1
  int merge;               // 1: the tiles of an item accumulate into one accumulator (compressed
                           //    path, g2 only, no C store); the diagonal pass runs once per item
  int rmerge;              // 1 (single tiles, compressed, C and g2): C stored per tile, the tiles of
                           //    an item summed in a TMEM accumulator for one diagonal pass per item
  // raw row update of a stream (items == nullptr): row blocks live in a ring of ring_nb
  // blocks, column block J = (I + delta) mod ring_nb, and item i is (q, delta, I, I + 1)
  // with q = i / ring_nd, delta = i mod ring_nd, I = (ring_J - delta) mod ring_nb
  int ring_nb, ring_nd, ring_J;
  const float* rc;         // nullable [n_q][T_pad] column scales (default: r)
  // compressed stream step (sm = 1, with the ring fields above): L = the coefficient history
  // shared by all rings (rows I*128 ..), R = the step's block of 128 w rows of ring q (rows
  // q*128 .., zero except the step's frames, which carry their scale r_q(t)), sm_nk
  // 64-wide chunks per piece, row scale r[slot * r_ld + q], no column scale
  int sm, sm_nk, r_ld;
  int sm_c0, sm_c1;        // stream step: the step's frames are rows [sm_c0, sm_c1) of each w block
  int sm_nq;               // stream step: rings; with pairs, the two halves of an accumulator are
                           // rings q and q + 1 (item q = 2 (i / ring_nd)) of one tile diagonal
  const float* r;          // [n_q][T_pad] sqrt(M_q)/S_q(t); 0 where undefined
  const uint32_t* blk_bad;  // [n_q][nT] block holds an undefined frame (< T)
  float* C;                // nullable [n_q][T][T]
  long long* Nout;         // nullable, raw only [n_q][T][T]
  float* partials;         // nullable [n_q][nT][maxC][256]
  uint32_t* status;
};

cudaError_t launch_gram(const CUtensorMap& tmL, const CUtensorMap& tmR, const GramParams& p, int grid,
                        cudaStream_t st);
int gram_smem_bytes();

// ------------------------------------------------------------------ ingest / prep / g2

struct RawIngestParams {
  const void* X;           // [T][M] u8 or u16
  int dtype;               // 0 u8, 1 u16
  long long T, M;
  int T_pad;
  long long Mp;            // permuted row length (elements)
  const int* perm;         // [Mp] source pixel or -1
  const int* pos_ring;     // [Mp] ring of position or -1
  int n_q;
  __nv_bfloat16* Xp;       // [T_pad][Mp] (nullable when only sums are wanted)
  long long xp_row0;       // row of Xp that frame 0 goes to (a stream's ring slot; else 0)
  long long* S;            // [n_q][T] (accumulated with atomics; the launch zeroes it)
  long long* S2;           // nullable [n_q][T] per-frame sum of squared counts (likewise)
  uint32_t* status;
};
cudaError_t launch_raw_ingest(const RawIngestParams& p, cudaStream_t st);

// r[q][t] for the chosen normalisation (xpcs_norm) from the raw int64 sums S, the
// per-frame sums of squares S2 (FROB) or the ring means Sbar (EQ12), and block flags
// (also flags XPCS_DEV_RANGE when a frame's sum of squares over a ring reaches 2^24)
cudaError_t launch_raw_scales(const long long* S, const long long* S2, const double* Sbar, int norm,
                              const long long* Mq, int n_q, long long T, int T_pad, int nT, float* r,
                              uint32_t* blk_bad, uint32_t* status, cudaStream_t st);
// Sbar[q] = mean over T frames of S[q][t]
cudaError_t launch_ring_mean(const long long* S, int n_q, long long T, double* Sbar, cudaStream_t st);
// Sbar[q] = (column means of A) . s_q, the compressed ring sum averaged over T frames
cudaError_t launch_coef_mean(const float* A, long long T, int k, const double* s64, int n_q, double* Sbar,
                             cudaStream_t st);

struct PrepParams {
  const float* A;          // [T][k]
  long long T;
  int k;
  int n_q;
  int T_pad, nT;
  const float* G32;        // [n_q][k][k]
  const double* s64;       // [n_q][k]
  const float2* s32;       // [n_q][k] (hi, lo) f32 pieces of s64
  const long long* Mq;     // [n_q]
  int prec;                // xpcs_precision
  int Kc;                  // operand row length (elements, multiple of 64)
  void* L;                 // [n_q][T_pad][Kc] 16-bit
  void* R;                 // [n_q][T_pad][Kc] 16-bit
  float* r;                // [n_q][T_pad]
  uint32_t* blk_bad;        // [n_q][nT]
  double* St;              // nullable [n_q][T] compressed ring sums
  int norm;                // xpcs_norm
  const double* Sbar;      // [n_q] mean compressed ring sums (XPCS_NORM_EQ12)
  const long long* S_exact;  // nullable [n_q][T] exact raw ring sums (XPCS_QMEAN_EXACT_RAW)
  int skip_L;              // 1: ring sums, scales and R rows only (L from the tensor-core kernel)
};

// Tensor-core left operand L_q(t) = r_q(t) a_t G_q (comp_tc.cu), kq = k rounded up to 64
// (64 or 128).  A pieces: [T_pad][2 kq] bf16 ([hi | lo]); G pieces: [n_q kq][2 kq] bf16,
// row (q, n) holding G_q[n][:] as [hi | lo].
struct CompTcParams {
  const float* r;          // [n_q][T_pad] scales from the CUDA-core operand pass
  void* L;                 // [n_q][T_pad][Kc] 16-bit operand rows
  int T_pad, Kc, kq;
  uint32_t* status;
};
int comp_tc_smem(int kq);
cudaError_t launch_ring_w_tc(const CUtensorMap& tmA, const CUtensorMap& tmG, const CompTcParams& p, int n_q,
                             int n_tiles, int prec, cudaStream_t st);
// [T_pad][2 kq] bf16 hi/lo pieces of the coefficient rows (zero beyond T and k)
cudaError_t launch_coef_pieces(const float* A, long long T, int k, int kq, int T_pad, __nv_bfloat16* out,
                               cudaStream_t st);
// [n_q kq][2 kq] bf16 hi/lo pieces of the ring factors G_q (FP64), zero beyond k
cudaError_t launch_gram_pieces(const double* G, int n_q, int k, int kq, __nv_bfloat16* out, cudaStream_t st);
cudaError_t launch_prep_compressed(const PrepParams& p, cudaStream_t st);

// validity bits (vbits: n_q x words, followed by n_q per-ring flags) and pair counts
cudaError_t launch_counts(const float* r, int n_q, long long T, int T_pad, uint32_t* vbits, int words,
                          long long* count, cudaStream_t st);
cudaError_t launch_g2_finalize(const float* partials, const long long* count, int n_q, long long T, int nT,
                               int maxC, int CH, double* g2, cudaStream_t st);
// Row splits of the g2-over-C kernel: enough CTAs for about 8 per SM, and no CTA walking
// more than about 1024 rows (its rows are a serial chain of loads), at most 64.
inline int g2_from_C_splits(long long T, int n_q, int num_sms) {
  const long long blocks = (T + TILE - 1) / TILE * n_q;
  const long long by_sms = (8LL * num_sms + blocks - 1) / blocks;
  const long long by_rows = (T + 1023) / 1024;
  const long long s = by_sms > by_rows ? by_sms : by_rows;
  return (int)(s < 1 ? 1 : (s > 64 ? 64 : s));
}
cudaError_t launch_g2_from_C(const float* C, int n_q, long long T, double* partial, int row_splits,
                             long long* cnt_partial, cudaStream_t st);
cudaError_t launch_g2_from_C_reduce(const double* partial, const long long* cnt_partial, int n_q, long long T,
                                    int row_splits, double* g2, long long* count, cudaStream_t st);
// Loads the two g2-over-C kernels into the current device's context (lazy module
// loading would otherwise do it, and may allocate, at their first launch).
cudaError_t preload_g2_from_C();

// ------------------------------------------------------------------ encode

struct EncodeParams {
  long long T, M;
  int k;
  int dtype;             // 0 u8, 1 u16
  int n_split;           // pixel splits
  long long px_per_split;  // multiple of 64
  float* partials;       // [n_split][T_pad][k]
  int T_pad;
  uint32_t* status;
};
cudaError_t launch_encode(const CUtensorMap& tmX, const CUtensorMap& tmB, const EncodeParams& p, int grid,
                          cudaStream_t st);
int encode_smem_bytes(int k);
int encode_frame_blocks(int k);  // 128-frame blocks sharing each basis tile
cudaError_t launch_encode_reduce(const float* partials, int n_split, long long T, int T_pad, int k, float scale,
                                 float* A, cudaStream_t st);

// ------------------------------------------------------------------ stream

struct StreamStep {
  const void* X;           // b x M counts (device)
  int dtype;               // 0 u8, 1 u16
  int vec16;               // X and its rows are 16-byte aligned (vector loads allowed)
  long long M;
  int k, n_q, b;
  long long t0;            // index of the first frame of the batch
  long long W, cap;
  long long Wp;            // row pitch of g2sum / cnt
  int nblk;
  const float* B32;        // M x k
  const float* G32;        // n_q x k x k
  const double* s64;       // n_q x k
  const long long* Mq;     // n_q
  const int* qmap;         // nullable M ring labels: with Sx, exact ring sums of the frames
  long long* Sx;           // nullable b x n_q exact ring sums (zeroed by the step launch)
  float* part;             // b x nblk x k
  float* a;                // b x k
  unsigned* se_done;       // b slice blocks finished per frame (the last adds the partials)
  __nv_bfloat16* W2;       // (max_batch n_q) x 2 kpad: w_q(t) rows, bf16 hi | lo
  __nv_bfloat16* A2;       // (cap + 128) x 2 kpad: coefficient history, bf16 hi | lo;
                           // rows cap .. cap + 127 mirror rows 0 .. 127
  int kpad;                // k rounded up to 64
  long long w2_rows;       // rows allocated in W2
  float* Rh;               // (cap + 128) x npad, rows cap .. cap + 127 mirror rows 0 .. 127
  unsigned long long* vbits;  // n_q x vwords: bit s of ring q = r_q(slot s) > 0, slots
                              // cap .. cap + 127 mirror slots 0 .. 127
  long long vwords;
  float2* g2sum;           // n_q x Wp (W rounded up to 64): running sums as f32 pairs (hi, lo)
  long long* cnt;          // n_q x Wp
  uint32_t* status;
  int num_sms;
  const CUtensorMap* tmA;  // host copies of the tensor maps of A2, W2, Rh, g2sum, cnt
  const CUtensorMap* tmW;
  const CUtensorMap* tmR;
  const CUtensorMap* tmG;  // [RT_N_LT]: one per lag tile of RT_LTS
  const CUtensorMap* tmC;  // [RT_N_LT]
  // steps of at least STREAM_GRAM_MIN frames (all in one 128-frame block) run on the
  // two-time kernel: w rows of the block per ring, diagonal partials
  __nv_bfloat16* Wg;       // n_q x 128 x 2 kpad: w_q(t) of the step's frames, row t mod 128,
                           // zero rows elsewhere (the fold clears the step's rows)
  float* gpart;            // n_q x nd x 256 diagonal partial sums
  int nd;                  // tile diagonals that can hold a lag < W
  const CUtensorMap* tmWg;  // boxes of 128 w rows (one ring)
  const CUtensorMap* tmWg2; // boxes of 256 w rows (two rings)
  const CUtensorMap* tmW48; // W2 in boxes of 48 rows (single-frame steps)
  int pre_encoded;         // 1: a already holds the step's coefficients (tensor-core encode)
  int sp;                  // 1: coefficient rows in f16, one product (the hi halves of the rows
                           //    only); 0: bf16 hi | lo pieces, three products
  // single-frame steps: the deferred pair counts this step adds (frames cf_t0 + f of
  // cf_mask, lags cf_tau0 .. cf_tau1 - 1; none when cf_mask is 0)
  long long cf_t0;
  unsigned long long cf_mask;
  int cf_tau0, cf_tau1;
};
// Single-frame steps leave their pair counts to count blocks of 64 frames (block of frame
// t: t / 64).  The deferred counts of a block are added in 64 parts of the lag range, part
// j by the single-frame step at position j of the next block, or by launch_count_flush.
__host__ __device__ inline long long cf_part_len(long long W) { return (W + 63) / 64; }
bool stream_step_row1(const StreamStep& s);
cudaError_t launch_count_flush(const unsigned long long* vbits, long long vwords, long long cap, int n_q,
                               long long W, long long Wp, long long* cnt, long long t0, unsigned long long mask,
                               unsigned long long done, cudaStream_t st);
// Smallest step (frames) that runs on the two-time kernel; smaller steps take the row
// update kernel.  Steps never cross a 128-frame block when they may take the former.
constexpr int STREAM_GRAM_MIN = 32;
// tile diagonals of the history that can hold a lag < W
inline int stream_nd(long long W) { return (int)((W + 126) / 128 + 1); }
cudaError_t launch_stream_step(const StreamStep& s, cudaStream_t st);

// Row update of a step of at most 64 frames on the tensor cores (see stream_tc.cu).
// W2 holds the step's w rows in pair order, per ring group rg (36 rings from q0 = 36 rg)
// n_mt M-tiles of 128 rows starting at row rg n_mt 128; within M-tile mt:
//   small steps (b <= 8): mt = f, row ql = q - q0 (rows 0..35): one frame per tile, its
//     36 rings as the N operand of an MMA whose M operand is the history;
//   larger steps: mt = qi nfb + fb (nfb = ceil(b / 32)), lane quarter w = ring residue
//     q mod 4, lane l: ring q = q0 + 4 qi + w, frame f = 32 fb + l: a warp holds 32
//     consecutive frames of one ring.
constexpr int W2_SMALL_B = 8;
struct RowTcParams {
  long long t0, W, cap;
  int b, n_q, kpad, n_kc, lt, wst, n_tiles;
  int epi;                 // epilogue: 0 rotated blocks, 1 skewed buffers, 2 steps of <= W2_SMALL_B frames
  int n_rg;  // ring groups of 36
  int n_mt;  // M-tiles per ring group
  int nfb;   // 32-frame blocks of the step
  int npad;  // Rh row pitch (n_q rounded up to 4)
  int qb;    // r values per history row loaded per item (min(36, npad))
  const float* Rh;
  const unsigned long long* vbits;  // n_q x vwords validity bits of the ring slots (+ 128 mirrored)
  long long vwords;
  long long Wp;  // row pitch (elements) of g2sum and cnt: W rounded up to 64
  int qg2;       // ring rows per g2sum / cnt box: min(36, n_q)
  int sp;        // 1: f16 rows, one product (hi halves only)
  uint32_t* status;
};
int row_update_tc_smem(int n_kc, int lt, int qb, int wst, int qg2, int epi);
// Single-frame steps (b = 1, n_q <= 36) on the tensor cores (stream_tc.cu): frame t
struct Row1Params {
  long long t, W, cap;
  int n_q, kpad, n_kc, npad, qb, n_tiles;  // qb = npad (r values per history row)
  long long Wp;            // row pitch of g2sum / cnt
  int sp;                  // 1: f16 rows, one product (hi halves only)
  int sb, qg2;             // sb = 2 (1): each tile's g2 sums (qg2 = min(36, n_q) rings x 128
                           // lags) staged in shared memory by TMA in two slices, one tile ahead
                           // (in one slice); 0: read in place
  const float* Rh;         // (cap + 128) x npad
  float2* g2sum;           // n_q x Wp
  long long* cnt;          // n_q x Wp (only the deferred counts below)
  const unsigned long long* vbits;
  long long vwords;
  long long cf_t0;         // deferred counts to add: frames cf_t0 + f of cf_mask, lags
  unsigned long long cf_mask;  // cf_tau0 .. cf_tau1 - 1
  int cf_tau0, cf_tau1;
  uint32_t* status;
};
int row1_tc_smem(int n_kc, int qb, int sp, int sb, int qg2);
// tensor maps: A2 history (64 x 128 boxes), W2 (64 x 48 boxes), Rh (qb x 128 boxes),
// g2sum (128 x qg2 boxes)
cudaError_t launch_row1_tc(const CUtensorMap& tmA, const CUtensorMap& tmW, const CUtensorMap& tmR,
                           const CUtensorMap& tmG, const Row1Params& p, int grid, cudaStream_t st);
// tensor maps: A2 history, W2 pairs, Rh r values, g2sum and cnt (lt x qg2 boxes)
cudaError_t launch_row_update_tc(const CUtensorMap& tmA, const CUtensorMap& tmW, const CUtensorMap& tmR,
                                 const CUtensorMap& tmG, const CUtensorMap& tmC, const RowTcParams& p, int grid,
                                 cudaStream_t st);
// M-tiles per ring group for a step of b frames
__host__ __device__ inline int w2_mtiles(int b, int n_q) {
  if (b <= W2_SMALL_B) return b;
  const int nq4 = ((n_q < 36 ? n_q : 36) + 3) / 4;
  return nq4 * ((b + 31) / 32);
}
// pair-order row of (frame f, ring q) in W2 for a step of b frames
__host__ __device__ inline int w2_pair_row(int f, int q, int b, int n_q) {
  const int rg = q / 36, ql = q - 36 * rg;
  const int base = rg * w2_mtiles(b, n_q) * 128;
  if (b <= W2_SMALL_B) return base + f * 128 + ql;
  const int nfb = (b + 31) / 32;
  return base + (ql % 4) * 32 + ((ql / 4) * nfb + f / 32) * 128 + f % 32;
}
// 64-bit words per ring of the validity bits: cap + 128 bits and two spare words
inline long long stream_vwords(long long cap) { return (cap + 128 + 63) / 64 + 2; }
// Rh row pitch: n_q rounded up to 4 (16-byte rows for the tensor map)
__host__ __device__ inline int stream_npad(int n_q) { return (n_q + 3) / 4 * 4; }
// Lag tiles of the row update: a step of b frames takes the longest tile with
// lt + b - 1 <= 128 (its history rows fit one operand) that fits shared memory, so a
// single-frame step covers 128 lags per work item.  One g2-sum / count tensor map per tile.
constexpr int RT_N_LT = 5;
constexpr int RT_LTS[RT_N_LT] = {128, 120, 96, 64, 32};
inline int rt_lt_index(int lt) {
  for (int i = 0; i < RT_N_LT; ++i)
    if (RT_LTS[i] == lt) return i;
  return -1;
}
// lag tile, w stages (2 or 1) and epilogue mode of the row update for steps of b frames;
// false if nothing fits shared memory
bool row_update_config(int n_q, int kpad, int b, int* lt, int* wst, int* epi);
cudaError_t launch_stream_g2(const float2* g2sum, const long long* cnt, int n_q, long long W, long long Wp,
                             double* g2, cudaStream_t st);
cudaError_t launch_basis_f32(const double* B, long long n, float* B32, cudaStream_t st);

// ------------------------------------------------------------------ basis

cudaError_t launch_gram_normalise(const long long* N, int n, double* Gf, double* nrm, cudaStream_t st);
cudaError_t launch_basis_z(const double* U, const double* lam, const double* nrm, int n, int k, double* Z,
                           cudaStream_t st);
cudaError_t launch_basis_build(const void* F, int dtype, int n, long long M, const double* Z, int k, double* B,
                               cudaStream_t st);
cudaError_t launch_basis_sign(double* B, long long M, int k, cudaStream_t st);
cudaError_t launch_ring_factors2(const double* B, int k, const int* perm, const int* off, const long long* Mq,
                                 int n_q, int n_split, double* Gpart, double* spart, cudaStream_t st);
cudaError_t launch_ring_factors_reduce(const double* Gpart, const double* spart, int n_chunks, int n_q, int k,
                                       double* G, double* s, float* G32, float2* s32, cudaStream_t st);
cudaError_t launch_basis_absmax(const double* B, long long n, double* out, cudaStream_t st);
cudaError_t launch_basis_pack(const double* B, long long M, long long M_pad, int k, int kp, int log2_scale,
                              __half* Bcat, cudaStream_t st);

}  // namespace xpcs
