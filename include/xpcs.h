/*
 * xpcs.h -- C ABI of the GB300 (sm_103a) library for XPCS two-time correlation on raw
 * photon-count frames and on SVD-compressed frames, after arXiv 2407.20356,
 * "Homomorphic data compression for real time photon correlation analysis".
 *
 * Conventions for every entry point:
 *  - Pointers are DEVICE pointers (memory of the context's GPU) unless the parameter
 *    name ends in `_host`, in which case they are host pointers.
 *  - The caller owns every data buffer.  The library owns the opaque handles it creates
 *    (context, ring plan, basis, stream) and frees them in the matching destroy/close.
 *    Destroy every handle before the context it was created on.
 *  - Matrices are dense row-major.  X is T x M (frame t, pixel p), one frame per row.
 *  - Work is enqueued on the context's CUDA stream.  Unless the context is in
 *    asynchronous mode (xpcs_set_async), each call waits for its work and returns any
 *    error it raised; in asynchronous mode errors surface at xpcs_synchronize().
 *  - Functions return an xpcs_status; nothing throws or aborts across the ABI.  The text
 *    of the last error of a context is available from xpcs_last_error().
 *  - The two-time matrix is symmetric; outputs hold its lower triangle: C[q][t1][t2]
 *    (and N[q][t1][t2]) for t1 >= t2, n_q x T x T row-major, float32 (int64 for N).
 *    Entries above the diagonal are left untouched.  Undefined pairs (a ring sum <= 0)
 *    are NaN.  g2 and count arrays are n_q x T, indexed by lag tau = 0..T-1; g2 is NaN
 *    where count is 0.
 */
#ifndef XPCS_GB300_H
#define XPCS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum xpcs_status {
  XPCS_OK = 0,
  XPCS_EINVAL = 1,   /* bad argument, shape or handle */
  XPCS_ENOMEM = 2,   /* device allocation failed or the HBM budget would be exceeded */
  XPCS_ECUDA = 3,    /* a CUDA runtime/driver/library call failed */
  XPCS_ETIMEOUT = 4, /* a bounded device-side wait expired; the context stays usable */
  XPCS_EBUSY = 5,    /* the request does not fit the HBM budget now; retry later */
  XPCS_ERANGE = 6,   /* input outside the exact range of the requested path */
  XPCS_ENOTSUP = 7   /* shape or option not supported by this build */
} xpcs_status;

typedef enum xpcs_dtype { XPCS_U8 = 0, XPCS_U16 = 1 } xpcs_dtype;

/* Arithmetic of the compressed two-time Gram (tensor cores, f32 accumulation). */
typedef enum xpcs_precision {
  XPCS_PREC_FP16 = 0,  /* coefficients in f16 (unit roundoff 2^-11) */
  XPCS_PREC_BF16 = 1,  /* coefficients in bf16 (unit roundoff 2^-8) */
  XPCS_PREC_BF16X3 = 2 /* hi/lo bf16 split, three products: about 2^-16 */
} xpcs_precision;

/* Normalisation of the two-time correlation, as a per-frame scale r_q(t) with
 * C_q(t1,t2) = r_q(t1) r_q(t2) N_q(t1,t2) and g2_q(tau) the mean of C_q over the defined
 * pairs of the tau-th diagonal:
 *   XPCS_NORM_MEAN  Eq. 1: r = sqrt(M_q) / S_q(t) (per-frame ring mean); frames with
 *                   S_q(t) <= 0 are undefined (the default of xpcs_twotime{,_raw});
 *   XPCS_NORM_FROB  Eq. 2 with rows normalised by their Frobenius norm (Sec. 2.1):
 *                   r = 1 / sqrt(N_q(t,t)), C is the cosine similarity of the ring's
 *                   frames; frames with N_q(t,t) = 0 are undefined;
 *   XPCS_NORM_EQ12  Eq. 12 literally: r = sqrt(M_q) / Sbar_q with Sbar_q the mean of
 *                   S_q(t) over the T frames, so g2 = <I(t) I(t+tau)> / <I>^2 with both
 *                   averages over frames and ring pixels; every frame is defined.
 * On the compressed path N~ and S~ take the place of N and S (N~_q(t,t) = a_t G_q a_t^T,
 * Sbar~_q = abar s_q with abar the mean coefficient row). */
typedef enum xpcs_norm { XPCS_NORM_MEAN = 0, XPCS_NORM_FROB = 1, XPCS_NORM_EQ12 = 2 } xpcs_norm;

/* Per-frame ring sums in the denominators of the compressed path (Eq. 1 read with the
 * compressed Gram of Eq. 10 in the numerator):
 *   XPCS_QMEAN_COMPRESSED  S~_q(t) = a_t s_q, the ring sum of the decompressed frame
 *                          (consistent with Eq. 8; the default); lossy bases can make it
 *                          <= 0, which leaves the frame undefined;
 *   XPCS_QMEAN_EXACT_RAW   S_q(t), the exact ring sum of the raw frame, captured when the
 *                          frames are encoded (xpcs_encode_sums, or a stream opened with
 *                          this option); only frames without photons in a ring are then
 *                          undefined there. */
typedef enum xpcs_qmean { XPCS_QMEAN_COMPRESSED = 0, XPCS_QMEAN_EXACT_RAW = 1 } xpcs_qmean;

/* Options of the compressed calls.  Zero-initialised it is { XPCS_PREC_FP16,
 * XPCS_NORM_MEAN, XPCS_QMEAN_COMPRESSED }. */
typedef struct xpcs_options {
  int precision; /* xpcs_precision */
  int norm;      /* xpcs_norm */
  int qmean;     /* xpcs_qmean */
} xpcs_options;

typedef struct xpcs_ctx xpcs_ctx;
typedef struct xpcs_rings xpcs_rings;
typedef struct xpcs_basis xpcs_basis;
typedef struct xpcs_stream xpcs_stream;
typedef struct xpcs_server xpcs_server;
typedef struct xpcs_graph xpcs_graph;

/* ------------------------------------------------------------------ context */

/* Library version (major*10000 + minor*100 + patch). */
int xpcs_version(void);

/* Create a context on `device` that enqueues on `cuda_stream` (a cudaStream_t, or NULL
 * for a stream the library creates).  `hbm_budget_bytes` caps the device memory the
 * library itself allocates (scratch and handles); 0 means no cap. */
xpcs_status xpcs_create(int device, size_t hbm_budget_bytes, void* cuda_stream, xpcs_ctx** out);
xpcs_status xpcs_destroy(xpcs_ctx* ctx);
/* Text of the last error of this context ("" if none).  Valid until the next call. */
const char* xpcs_last_error(const xpcs_ctx* ctx);
/* async != 0: calls return once their work is enqueued; errors surface at synchronize. */
xpcs_status xpcs_set_async(xpcs_ctx* ctx, int async);
/* Wait for all enqueued work and report any device-side error. */
xpcs_status xpcs_synchronize(xpcs_ctx* ctx);
/* Bytes the library currently holds on the device for this context and its handles. */
size_t xpcs_device_bytes(const xpcs_ctx* ctx);
/* Number of CUDA kernels the library has launched on this context so far. */
uint64_t xpcs_launch_count(const xpcs_ctx* ctx);

/* Per-kernel timing: when enabled, CUDA events on the context's stream bracket every
 * launch site; entries accumulate per site name.  Enabling (or disabling) clears them.
 * xpcs_profile_get waits for the stream, then reports entry i: name (NUL-terminated,
 * truncated to name_cap), total milliseconds and number of timed launches. */
xpcs_status xpcs_profile_enable(xpcs_ctx* ctx, int on);
int xpcs_profile_count(const xpcs_ctx* ctx);
xpcs_status xpcs_profile_get(xpcs_ctx* ctx, int i, char* name_host, size_t name_cap, double* ms_host,
                             int64_t* launches_host);

/* Failure-detection self test (no counterpart in the paper).  Every device-side wait of
 * the library is bounded: past its limit the kernel records a timeout and unwinds, and
 * the host sees XPCS_ETIMEOUT with the context still usable.  This call runs one such
 * wait that nothing satisfies, for limit_ms (1..1000) milliseconds, or with limit_ms = 0
 * through the library's own bounded wait with the context's limit (xpcs_set_timeout; at
 * most 10 s for this call), and returns what a real expired wait returns: XPCS_ETIMEOUT
 * (at once in synchronous mode, else from xpcs_synchronize).  XPCS_EINVAL for a limit
 * out of range. */
xpcs_status xpcs_selftest_timeout(xpcs_ctx* ctx, int limit_ms);
/* Limit of the bounded device-side waits (no counterpart in the paper) of the kernels this
 * context launches, and of the streams opened on it after this
 * call (a stream keeps the limit it was opened with): 1..600000 ms, or 0 for the default
 * of 2000 ms.  A wait that runs past it ends its kernel with XPCS_ETIMEOUT.  Waits for the
 * context's queued work first; XPCS_EBUSY during a capture. */
xpcs_status xpcs_set_timeout(xpcs_ctx* ctx, int timeout_ms);
/* The context's current limit in milliseconds (-1 for a null context). */
int xpcs_get_timeout(const xpcs_ctx* ctx);

/* ------------------------------------------------------------------ q-rings (Sec. 2.2)
 * A ring plan fixes which pixels form each q-ring: qmap[p] in [0, n_q) is the ring of
 * pixel p, -1 leaves the pixel out (the q-subsets of Sec. 2.2).  `qmap` is a device
 * int32 array of length M, read once; the plan keeps its own copy. */
xpcs_status xpcs_rings_create(xpcs_ctx* ctx, const int32_t* qmap, int64_t M, int n_q, xpcs_rings** out);
xpcs_status xpcs_rings_destroy(xpcs_rings* rings);
/* M_q, the pixel count of every ring (host array of n_q). */
xpcs_status xpcs_rings_sizes(const xpcs_rings* rings, int64_t* Mq_host);

/* Ring sums S_q(t) = sum over p in ring q of X[t][p] (M_q times the pixel average in the
 * denominator of Eq. 1).  X: T x M counts of `dtype`.  S_out: n_q x T int64. */
xpcs_status xpcs_ring_sums(xpcs_ctx* ctx, const xpcs_rings* rings, const void* X, xpcs_dtype dtype, int64_t T,
                           int64_t* S_out);

/* ------------------------------------------------------------------ raw path (Eq. 1, 2)
 * Exact two-time correlation of raw counts, per ring:
 *   N_q = X_q X_q^T (Eq. 2 on the ring's pixels), C_q = M_q N_q / (S_q(t1) S_q(t2)) (Eq. 1),
 *   g2_q(tau) = mean over t of C_q(t, t+tau) over defined pairs.
 * The integer Gram is computed exactly on the tensor cores (bf16 operands, f32
 * accumulation kept below 2^24); counts above 256, or a ring whose largest per-frame
 * sum of squared counts reaches 2^24, return XPCS_ERANGE.
 * Outputs (all nullable): C_out n_q x T x T f32 (lower triangle), N_out n_q x T x T
 * int64 (lower triangle), g2_out n_q x T f64, count_out n_q x T int64. */
xpcs_status xpcs_twotime_raw(xpcs_ctx* ctx, const xpcs_rings* rings, const void* X, xpcs_dtype dtype, int64_t T,
                             float* C_out, int64_t* N_out, double* g2_out, int64_t* count_out);
/* xpcs_twotime_raw with a chosen normalisation (xpcs_norm); norm = XPCS_NORM_MEAN is
 * xpcs_twotime_raw.  N_out is the integer Gram in every mode. */
xpcs_status xpcs_twotime_raw_norm(xpcs_ctx* ctx, const xpcs_rings* rings, const void* X, xpcs_dtype dtype,
                                  int64_t T, xpcs_norm norm, float* C_out, int64_t* N_out, double* g2_out,
                                  int64_t* count_out);

/* ------------------------------------------------------------------ basis (Eq. 3-6)
 * Fit the encoding matrix V_K (M x k) on n_fit frames F (T x M layout, n_fit rows):
 * rows are divided by their Frobenius norm (Sec. 2.1), the n_fit x n_fit Gram is
 * eigendecomposed in FP64, and V_K = F^T U_k Sigma_k^-1 keeps the k largest singular
 * values (Eq. 6).  Ring factors G_q = B_q^T B_q and s_q = B_q^T 1 are formed in FP64.
 * sigma_host (nullable): all n_fit singular values, descending.  k above the numerical
 * rank returns XPCS_EINVAL. */
xpcs_status xpcs_fit_basis(xpcs_ctx* ctx, const xpcs_rings* rings, const void* F, xpcs_dtype dtype, int64_t n_fit,
                           int k, xpcs_basis** out, double* sigma_host);
/* Use an external encoding matrix (the paper's option of a basis fit on other data):
 * B_host is M x k FP64 row-major. */
xpcs_status xpcs_basis_import(xpcs_ctx* ctx, const xpcs_rings* rings, const double* B_host, int k,
                              xpcs_basis** out);
/* Copy basis data to the host (each pointer nullable): B M x k, G n_q x k x k, s n_q x k. */
xpcs_status xpcs_basis_export(xpcs_ctx* ctx, const xpcs_basis* basis, double* B_host, double* G_host,
                              double* s_host);
xpcs_status xpcs_basis_rank(const xpcs_basis* basis, int* k);
/* Rank choice from a fitted spectrum (Sec. 3.1, offline lossy compression): the number of
 * components whose value in the spectrum is at least `factor` times its smallest value
 * (the paper's rule uses factor 2).  sigma_host: n values in descending order, as
 * xpcs_fit_basis returns them; values at or below the numerical-rank cutoff
 * (sigma^2 <= n * eps * sigma_max^2) are left out, so the minimum is taken over the
 * numerical rank.  Host-side, no context needed.  Returns K >= 0, or -1 for a null
 * pointer, n <= 0, factor <= 0 or a spectrum that is not descending. */
int xpcs_rank_from_spectrum(const double* sigma_host, int n, double factor);
xpcs_status xpcs_basis_destroy(xpcs_basis* basis);

/* ------------------------------------------------------------------ encode (Eq. 7)
 * Coefficients Y_K = X V_K: A_out is T x k float32.  X: T x M counts (M a multiple of 8
 * for u16, 16 for u8).  Tensor cores: counts as f16 (exact up to 1023, else
 * XPCS_ERANGE), V_K as a power-of-two-scaled hi/lo f16 pair, f32 accumulation. */
xpcs_status xpcs_encode(xpcs_ctx* ctx, const xpcs_basis* basis, const void* X, xpcs_dtype dtype, int64_t T,
                        float* A_out);

/* xpcs_encode of frames in HOST memory (X_host, T x M counts, best pinned), with the
 * host-to-device copy overlapped with the encode: the frames move in blocks of about 256 MB
 * through three device staging buffers (context scratch), the copies alternating between
 * two copy streams, and each block is encoded on the context's stream as soon as it has
 * landed.  A_out is a device T x k float32 array as for xpcs_encode.  Returns once the
 * encode is done (unless the context is asynchronous; the host buffer must then stay
 * unchanged until xpcs_synchronize).  XPCS_EBUSY during a capture. */
xpcs_status xpcs_encode_host(xpcs_ctx* ctx, const xpcs_basis* basis, const void* X_host, xpcs_dtype dtype, int64_t T,
                             float* A_out);
/* xpcs_encode that also captures the exact ring sums of the raw frames for the option
 * XPCS_QMEAN_EXACT_RAW: S_out n_q x T int64 (device), S_q(t) = sum of X[t][p] over the
 * pixels p of ring q of the basis's ring plan (as xpcs_ring_sums; one more pass over X). */
xpcs_status xpcs_encode_sums(xpcs_ctx* ctx, const xpcs_basis* basis, const void* X, xpcs_dtype dtype, int64_t T,
                             float* A_out, int64_t* S_out);

/* ------------------------------------------------------------------ compressed path (Eq. 8-10)
 * Two-time correlation from coefficients only (no decompression):
 *   N~_q = A G_q A^T, S~_q(t) = a_t s_q, C~_q = M_q N~_q / (S~_q(t1) S~_q(t2)),
 * g2 as for the raw path.  A: T x k float32 (from xpcs_encode or the caller).
 * Outputs nullable as for xpcs_twotime_raw. */
xpcs_status xpcs_twotime(xpcs_ctx* ctx, const xpcs_basis* basis, const float* A, int64_t T, xpcs_precision prec,
                         float* C_out, double* g2_out, int64_t* count_out);
/* Autotuner of xpcs_twotime for one workload shape (rings, frames, precision, whether C
 * is stored): times each candidate configuration of the two-time kernel on these very
 * arguments, `reps` timed calls each after one untimed call, keeps the fastest in the
 * context for later calls of that shape, and runs it once more so the outputs are its
 * own.  Candidates: tiles per work item (1, 2, 4, 8, 16 or 32 along a tile diagonal) x schedule
 * (0: single tiles, one N = 128 MMA per tile; 1: tile pairs, one N = 256 MMA for tiles
 * (I, J) and (I, J + 1)).  The default stays unless another candidate is at least 3 %
 * faster: 8 single tiles when C is stored; 4 tiles with tile pairs for g2 only (C not
 * stored, where all tiles of a work item accumulate into one accumulator).
 * tiles_out, sched_out, ms_out (host, nullable): the choice and its time per call.  Not
 * during a capture. */
xpcs_status xpcs_autotune_twotime(xpcs_ctx* ctx, const xpcs_basis* basis, const float* A, int64_t T,
                                  xpcs_precision prec, float* C_out, double* g2_out, int64_t* count_out, int reps,
                                  int* tiles_out, int* sched_out, double* ms_out);
/* Fix the two-time configuration of this context's calls (xpcs_twotime*, xpcs_twotime_raw*)
 * instead of the tuned or default one: `tiles` per work item (1..64) and `schedule` (0 or 1
 * as for the autotuner).  tiles = 0 returns to the automatic choice.  The results of
 * every configuration agree up to the f32 rounding order of the g2 partial sums (the raw
 * integer Gram and C are bit-identical).  XPCS_EINVAL for values out of range. */
xpcs_status xpcs_twotime_config(xpcs_ctx* ctx, int tiles, int schedule);
/* The same autotuner for xpcs_twotime_raw (arguments as that call's); the raw default is
 * tile pairs, one per work item, or the fewest tiles per item (a power of two) that keep
 * the g2 partial slots (1 KB per ring, tile diagonal and item chunk) within 512 MB. */
xpcs_status xpcs_autotune_twotime_raw(xpcs_ctx* ctx, const xpcs_rings* rings, const void* X, xpcs_dtype dtype,
                                      int64_t T, float* C_out, int64_t* N_out, double* g2_out, int64_t* count_out,
                                      int reps, int* tiles_out, int* sched_out, double* ms_out);
/* xpcs_twotime with a chosen normalisation (xpcs_norm); norm = XPCS_NORM_MEAN is
 * xpcs_twotime. */
xpcs_status xpcs_twotime_norm(xpcs_ctx* ctx, const xpcs_basis* basis, const float* A, int64_t T,
                              xpcs_precision prec, xpcs_norm norm, float* C_out, double* g2_out,
                              int64_t* count_out);

/* xpcs_twotime with every option: opt (host, NULL = defaults) gives the precision, the
 * normalisation and the ring sums of the denominators.  With qmean = XPCS_QMEAN_EXACT_RAW,
 * S_raw (device, n_q x T int64: the exact ring sums of the raw frames of A, from
 * xpcs_encode_sums or xpcs_ring_sums) replaces a_t s_q in Eq. 1 (and its mean in Eq. 12);
 * otherwise S_raw is not read and may be NULL.  XPCS_EINVAL for EXACT_RAW without S_raw or
 * with the Frobenius normalisation (which uses no ring sums). */
xpcs_status xpcs_twotime_opts(xpcs_ctx* ctx, const xpcs_basis* basis, const float* A, int64_t T,
                              const xpcs_options* opt, const int64_t* S_raw, float* C_out, double* g2_out,
                              int64_t* count_out);

/* ------------------------------------------------------------------ g2 over a stored C
 * g2_q(tau) = mean over t of C[q][t+tau][t], NaN entries skipped, from the lower
 * triangle of C (n_q x T x T float32).  g2_out n_q x T f64, count_out nullable.
 * n_q above XPCS_G2_MAX_RINGS returns XPCS_ERANGE. */
#define XPCS_G2_MAX_RINGS 65535
xpcs_status xpcs_g2(xpcs_ctx* ctx, const float* C, int n_q, int64_t T, double* g2_out, int64_t* count_out);

/* ------------------------------------------------------------------ g2 over a stored C, no allocation
 * The paper has no counterpart to this call: it is a library convenience.
 * Same arguments, layout and result as xpcs_g2 (up to the order of the f64 partial
 * sums), but it allocates no device memory while it runs: its partial sums live in one
 * fixed array of XPCS_G2_NOALLOC_MAX_CELLS x 16 bytes (16 MiB) per device, part of the
 * library's image, instead of the context's scratch, which xpcs_g2 grows with cudaMalloc.
 * For callers that must not allocate while they run, e.g. a loop whose HBM is all
 * handed out under a budget, or one that cannot take the device-wide synchronisation a
 * cudaFree may imply.
 *   - n_q * T must not exceed XPCS_G2_NOALLOC_MAX_CELLS, nor n_q XPCS_G2_MAX_RINGS;
 *     larger calls return XPCS_ERANGE (with a message in xpcs_last_error) and launch
 *     nothing.
 *   - The first call on each device does a one-time set-up (finds the array's device
 *     address and loads the kernels, which the CUDA runtime may do by allocating):
 *     make it at start-up, before any stream capture and before the caller's
 *     no-allocation region.  Later calls only launch two kernels on the context's stream.
 *     The array's address found at set-up belongs to the device's primary context and is
 *     kept for the life of the process: after cudaDeviceReset, or from a context other
 *     than the primary one, do not call this entry point.
 *   - Nothing needs to start at zero: every call overwrites the partial sums it reads.
 *   - The array is shared by every call on a device: calls that can run at the same time
 *     (on different CUDA streams or contexts of one device) race on it and give wrong
 *     results.  Calls on one CUDA stream are ordered and safe. */
#define XPCS_G2_NOALLOC_MAX_CELLS (1 << 20)
xpcs_status xpcs_g2_noalloc(xpcs_ctx* ctx, const float* C, int n_q, int64_t T, double* g2_out,
                            int64_t* count_out);

/* ------------------------------------------------------------------ downstream analysis (Sec. 3)
 * Eq. 13 relaxation fit per ring: g2(tau) = B + C exp(-2 tau / t0), unweighted least
 * squares over the defined lags tau_lo..tau_hi of g2 (n_q x T f64, device; NaN lags are
 * skipped), t0 searched over [t0_min, t0_max] (variable projection: (B, C) solved for
 * each t0, the residual minimised over log t0 by a grid and golden-section refinement).
 * params_out (device, n_q x 4 f64): B, C, t0, rms residual; NaN for a ring with fewer
 * than three defined lags.  Requires 0 <= tau_lo <= tau_hi < T, 0 < t0_min < t0_max. */
xpcs_status xpcs_fit_relaxation(xpcs_ctx* ctx, const double* g2, int n_q, int64_t T, int64_t tau_lo,
                                int64_t tau_hi, double t0_min, double t0_max, double* params_out);
/* Mean and population standard deviation of a stored two-time matrix per ring (the
 * spread that Sec. 3.2 takes as the TTC's background level): over the defined values of
 * the lower triangle strictly below the diagonal, i.e. every unordered pair t1 != t2
 * once.  C: n_q x T x T f32 as written by the two-time calls; mean_out, std_out (nullable)
 * device n_q f64; NaN for a ring without defined pairs. */
xpcs_status xpcs_twotime_stats(xpcs_ctx* ctx, const float* C, int n_q, int64_t T, double* mean_out,
                               double* std_out);
/* Peak visibility (Sec. 3.1) per ring: the largest g2 over lags peak_lo..peak_hi minus the
 * mean g2 over lags bg_lo..bg_hi (defined lags only; NaN if either window has none).
 * flag_out (nullable, needs ttc_std): 1 when the visibility exceeds factor x ttc_std[q]
 * (Sec. 3.2's detectability test, factor 2), else 0.  All arrays device, length n_q. */
xpcs_status xpcs_peak_visibility(xpcs_ctx* ctx, const double* g2, int n_q, int64_t T, int64_t peak_lo,
                                 int64_t peak_hi, int64_t bg_lo, int64_t bg_hi, const double* ttc_std,
                                 double factor, double* vis_out, int32_t* flag_out);

/* ------------------------------------------------------------------ CUDA-graph capture
 * xpcs_capture_begin records the following library calls made on ctx (encode, two-time,
 * g2, analysis: everything that runs on the context's stream) instead of running them;
 * xpcs_capture_end instantiates them as one graph that xpcs_graph_launch replays with a
 * single launch on the context's stream (asynchronously if the context is, else waiting
 * for it).  During the capture the context runs asynchronously and profiling must be off.
 * The graph refers to the buffers the captured calls used, so while any graph of the
 * context exists, calls that would move or rewrite the context's scratch, its cached
 * two-time work items or a basis's first-use copies fail with XPCS_EBUSY: run each call
 * once, at its largest size, before capturing it.  Streams and servers are not captured.
 * A failed capture leaves the context usable and returns XPCS_ECUDA (or the failing
 * call's status). */
xpcs_status xpcs_capture_begin(xpcs_ctx* ctx);
xpcs_status xpcs_capture_end(xpcs_ctx* ctx, xpcs_graph** out);
xpcs_status xpcs_graph_launch(xpcs_ctx* ctx, const xpcs_graph* graph);
/* Library kernels in the graph (added to xpcs_launch_count at every launch). */
uint64_t xpcs_graph_kernels(const xpcs_graph* graph);
xpcs_status xpcs_graph_destroy(xpcs_graph* graph);

/* ------------------------------------------------------------------ online stream (Sec. 2.2, Fig. 1c)
 * Online compression with a basis fit before acquisition: every pushed frame is encoded
 * (a_t = x_t V_K: in steps of fewer than 32 frames sparse, only nonzero pixels reading
 * their f32 basis row; steps of 32 or more, on 16-byte aligned frame rows and without
 * exact ring sums, take the tensor-core encode of xpcs_encode, whose counts must stay
 * below 1024 — larger ones are flagged XPCS_ERANGE as there), appended to a
 * device ring buffer of the last `history` coefficient rows, and its two-time row
 * C_q(t, s) for s in (t - history, t] is folded into running sums over lags
 * tau = 0 .. history-1 (C itself is not stored).  xpcs_stream_read_g2 returns
 * g2_q(tau) = mean over t of C_q(t, t - tau) for every pushed frame t, and the pair count.
 * Work runs on the stream's own CUDA stream, so several streams overlap on the device.
 * Push only while the basis is alive; destroy streams before their context (closing a
 * stream does not read its basis, and a basis does not read its ring plan). */

/* Open a stream on `basis` for frames of `dtype`, keeping `history` lags, with batches
 * of up to `max_batch` frames.  XPCS_EBUSY if its device memory does not fit the
 * context's budget now (retry once other streams close); XPCS_ENOTSUP if no row-update
 * lag tile for 64-frame steps fits shared memory at this k and ring count.  `basis` must
 * stay alive while frames are pushed; closing the stream does not read it. */
xpcs_status xpcs_stream_open(xpcs_ctx* ctx, const xpcs_basis* basis, int64_t history, int max_batch,
                             xpcs_dtype dtype, xpcs_stream** out);
/* xpcs_stream_open with options: of opt (host, NULL = xpcs_stream_open's defaults) qmean
 * and precision are used.  precision XPCS_PREC_BF16X3 (xpcs_stream_open's) keeps the
 * coefficient history and the w_q(t) rows of Eq. 1 as bf16 hi | lo pieces (three
 * products, about 2^-16 relative); XPCS_PREC_FP16 (a zero-initialised opt) keeps them as
 * one f16 piece (one product, half the history bytes, about 2^-11 relative: the same
 * error as the offline f16 path), each history row scaled by a power of two that its
 * ring factors take out again; XPCS_PREC_BF16 is refused (XPCS_EINVAL).  With
 * XPCS_QMEAN_EXACT_RAW every pushed frame's exact ring sums, added up from its nonzero
 * pixels during the sparse encode, replace a_t s_q in the denominators. */
xpcs_status xpcs_stream_open_opts(xpcs_ctx* ctx, const xpcs_basis* basis, int64_t history, int max_batch,
                                  xpcs_dtype dtype, const xpcs_options* opt, xpcs_stream** out);
/* The row-update configuration a stream step of b frames takes for n_q rings and a k-term
 * basis (host-side, no context or device needed).  Steps of 32 frames or more (cut so that
 * they stay within one 128-frame block) run on the two-time kernel: *epilogue = 3, *lags =
 * 128 (one tile diagonal per work item), *w_stages = 0, *smem_bytes = that kernel's.
 * Smaller steps take the row update kernel: *lags = the lag tile (the longest of 128, 120,
 * 96, 64, 32 with lags + b - 1 <= 128 whose layout fits shared memory), *w_stages =
 * pair-operand stages (1 or 2), *epilogue = 0 rotated blocks, 1 skewed buffers, 2 the
 * small-step form (exactly when b <= 8), *smem_bytes = dynamic shared memory of the
 * launch.  Outputs are nullable.  XPCS_EINVAL unless 1 <= n_q <= 1024, 1 <= k <= 256 and
 * 1 <= b <= 64; XPCS_ENOTSUP if nothing fits. */
xpcs_status xpcs_stream_row_tile(int n_q, int k, int b, int* lags, int* w_stages, int* epilogue, int* smem_bytes);
/* Push n frames (n x M counts in host memory).  The frames are copied before the call
 * returns, so the caller may reuse its buffer.  *ticket (nullable) = frames pushed so far;
 * pass it to xpcs_stream_poll. */
xpcs_status xpcs_stream_push(xpcs_stream* s, const void* frames_host, int64_t n_frames, uint64_t* ticket);
/* Push n frames already in device memory (the buffer must stay valid until the ticket
 * completes). */
xpcs_status xpcs_stream_push_device(xpcs_stream* s, const void* frames, int64_t n_frames, uint64_t* ticket);
/* As xpcs_stream_push_device, with each frame's arrival time: arrive_ns_host holds
 * n_frames values of xpcs_clock_ns (e.g. when the detector delivered the frame), and the
 * latency statistics count from there instead of from the call. */
xpcs_status xpcs_stream_push_device_at(xpcs_stream* s, const void* frames, int64_t n_frames,
                                       const int64_t* arrive_ns_host, uint64_t* ticket);
/* The host steady clock of the latency statistics, in nanoseconds. */
int64_t xpcs_clock_ns(void);
/* XPCS_OK once every frame up to `ticket` is folded into the sums; XPCS_EBUSY if not
 * within timeout_ms (0 = just check). */
xpcs_status xpcs_stream_poll(xpcs_stream* s, uint64_t ticket, int timeout_ms);
/* g2_host (nullable): n_q x history f64; count_host (nullable): n_q x history int64.
 * Waits for the stream's pending work.  The running sums behind g2 are f32 pairs
 * (hi + lo, about 2^-48 relative rounding per addition), divided by the count in FP64. */
xpcs_status xpcs_stream_read_g2(xpcs_stream* s, double* g2_host, int64_t* count_host);
/* Frames pushed so far. */
int64_t xpcs_stream_frames(const xpcs_stream* s);
/* Checkpoint / resume of a stream's state: the coefficient history, ring-factor rows,
 * validity bits, g2 sums, pair counts and frame count (everything else is per-step
 * scratch), after a header with the stream's shape and a hash of the basis's ring
 * factors.  xpcs_stream_checkpoint waits for the stream's queued batches and copies the
 * state into host_buf (at least xpcs_stream_checkpoint_size bytes).  xpcs_stream_restore
 * takes a checkpoint into a stream opened with the same basis, history, max_batch and
 * dtype to which no frame has been pushed yet, which then continues where the
 * checkpointed one stopped; other shapes or bases give XPCS_EINVAL, as do checkpoints of
 * format version 1 (FP64 sums; this build writes version 2).  Latency records are not
 * part of the state. */
xpcs_status xpcs_stream_checkpoint_size(const xpcs_stream* stream, size_t* bytes);
xpcs_status xpcs_stream_checkpoint(xpcs_stream* stream, void* host_buf, size_t bytes);
xpcs_status xpcs_stream_restore(xpcs_stream* stream, const void* host_buf, size_t bytes);
/* Per-frame latency of completed frames, in microseconds (host steady clock): from the
 * frame's arrival (entering xpcs_stream_push, or its submission to a server) to the end of
 * its batch's device work.  *n_frames = frames measured.  reset != 0 forgets them. */
xpcs_status xpcs_stream_latency(xpcs_stream* s, int reset, double* p50_us, double* p99_us, double* max_us,
                                int64_t* n_frames);
xpcs_status xpcs_stream_close(xpcs_stream* s);

/* ------------------------------------------------------------------ online stream on raw frames
 * The raw-path counterpart of the online stream (Sec. 2.2 online mode, against which Sec.
 * 3.2 times the compressed path): every pushed frame's exact two-time row against the last
 * `history` frames, C_q(t, s) = M_q N_q(t, s) / (S_q(t) S_q(s)) with the integer Gram of
 * Eq. 2 on the tensor cores (bf16 counts, exact below the raw path's bounds: counts <= 256
 * and every frame's sum of squared counts per ring below 2^24, else XPCS_ERANGE), folded
 * into running FP64 sums per lag.  The frames are kept in ring-sorted bf16 rows (128 x
 * ceil(history / 128) + 256 rows of the ring plan's padded length), so every push reads the
 * whole window once.  Work runs on the context's stream; the ring plan must stay alive
 * while frames are pushed. */
typedef struct xpcs_raw_stream xpcs_raw_stream;
xpcs_status xpcs_raw_stream_open(xpcs_ctx* ctx, const xpcs_rings* rings, int64_t history, xpcs_dtype dtype,
                                 xpcs_raw_stream** out);
/* Push n frames already in device memory (n x M counts of the stream's dtype), processed in
 * steps that do not cross a 128-frame block.  Returns once they are
 * folded in (unless the context is asynchronous). */
xpcs_status xpcs_raw_stream_push_device(xpcs_raw_stream* rs, const void* frames, int64_t n);
/* g2_host (nullable): n_q x history f64, NaN without pairs; count_host (nullable): n_q x
 * history int64.  Waits for the context's stream. */
xpcs_status xpcs_raw_stream_read_g2(xpcs_raw_stream* rs, double* g2_host, int64_t* count_host);
/* Frames pushed so far (-1 for a null handle). */
int64_t xpcs_raw_stream_frames(const xpcs_raw_stream* rs);
xpcs_status xpcs_raw_stream_close(xpcs_raw_stream* rs);

/* ------------------------------------------------------------------ serving several streams
 * A server owns a scheduler thread for streams opened through it.  xpcs_server_submit
 * copies frames into the stream's host queue and returns at once; the scheduler takes,
 * for each stream whose staging buffer is free, every frame that has arrived (up to the
 * stream's max_batch) and enqueues it on the stream's own CUDA stream, so streams of
 * different detector sizes overlap on the device and a batch grows while the previous one
 * runs.  Streams are admitted against the context's device-memory budget.  A stream's
 * results depend only on its own frames (alone or in a mix they agree up to the f32
 * rounding of per-batch partial sums).  Streams of a server are used only through the
 * xpcs_server_* calls; all of them are thread-safe. */
xpcs_status xpcs_server_create(xpcs_ctx* ctx, xpcs_server** out);
/* Open a stream (arguments as xpcs_stream_open).  If it does not fit the budget, wait up
 * to wait_ms for streams to close (0: fail at once); XPCS_EBUSY if it still does not fit. */
xpcs_status xpcs_server_open(xpcs_server* server, const xpcs_basis* basis, int64_t history, int max_batch,
                             xpcs_dtype dtype, int wait_ms, xpcs_stream** out);
/* Queue n host frames; *ticket (nullable) = frames submitted to this stream so far. */
xpcs_status xpcs_server_submit(xpcs_server* server, xpcs_stream* s, const void* frames_host, int64_t n,
                               uint64_t* ticket);
/* Queue n frames that are already in device memory (a detector feeding the GPU
 * directly).  Nothing is copied: the stream's kernels read the frames in place, so the
 * caller keeps them unchanged until the ticket has completed (xpcs_server_poll).  Batches
 * are taken from one submitted block at a time. */
xpcs_status xpcs_server_submit_device(xpcs_server* server, xpcs_stream* s, const void* frames_dev, int64_t n,
                                      uint64_t* ticket);
/* XPCS_OK once every frame up to `ticket` is folded in; XPCS_EBUSY after timeout_ms. */
xpcs_status xpcs_server_poll(xpcs_server* server, xpcs_stream* s, uint64_t ticket, int timeout_ms);
xpcs_status xpcs_server_read_g2(xpcs_server* server, xpcs_stream* s, double* g2_host, int64_t* count_host);
xpcs_status xpcs_server_latency(xpcs_server* server, xpcs_stream* s, int reset, double* p50_us, double* p99_us,
                                double* max_us, int64_t* n_frames);
/* Finish the stream's queued frames, close it and release its memory to waiting opens. */
xpcs_status xpcs_server_close(xpcs_server* server, xpcs_stream* s);
/* Batches the scheduler has enqueued so far. */
uint64_t xpcs_server_batches(const xpcs_server* server);
/* Stop the scheduler and close the remaining streams. */
xpcs_status xpcs_server_destroy(xpcs_server* server);

#ifdef __cplusplus
}
#endif
#endif /* XPCS_GB300_H */
