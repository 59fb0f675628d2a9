/*
 * hos.h -- C ABI of the GB300 higher-order-spectra library.
 *
 * The library estimates the smoothed sample bispectrum and trispectrum of a
 * real series X(1..n) (paper: Problem Statement, "compute smoothed sample
 * bispectrum and trispectrum") by the indirect method the paper names in
 * "Direct Method for HOS" (the Fourier transform of the third cumulant):
 *
 *   1. per-part mean removal in FP64          (Algorithm DBS steps 1-2);
 *   2. sample cumulant c3 over the lag square, or c4 over the lag cube
 *      (Problem Statement: moments m_k, cumulants, time averages);
 *   3. lag window, and average over parts      (Algorithm DBS step 6);
 *   4. 2-D / 3-D DFT onto the frequency grid   (Problem Statement; sign of
 *      Algorithm DBS step 3).
 *
 * Definitions (the paper is silent on these; the library's readings):
 *   c3(w1,w2)    = (1/n) sum_i y(i) y(i+w1) y(i+w2), samples outside the
 *                  series are zero (biased estimator);
 *   c4(w1,w2,w3) = m4(w1,w2,w3) - c2(w1)c2(w3-w2) - c2(w2)c2(w3-w1)
 *                  - c2(w3)c2(w2-w1), with m4, c2 the same time averages;
 *   Parzen d(u), u = |w|/L: 1-6u^2+6u^3 (u<=1/2), 2(1-u)^3 (u<=1), 0 beyond;
 *   B(k1,k2)     = (2 pi)^-2 sum_w W(w) c3(w) exp(-i 2 pi (k1 w1 + k2 w2)/N),
 *   T(k1,k2,k3)  = (2 pi)^-3 sum_w W(w) c4(w) exp(-i 2 pi k.w / N),
 *                  k = 0..N-1 (unshifted), N = nfft (default 2L).
 * Every window used has W = 0 at |w| = L, so the lag range computed is
 * [-L, L-1] on each axis (2L lags) and no lag aliases on an N >= 2L grid.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* and every array argument are DEVICE pointers on the
 *     current CUDA device, owned by the caller.  The library never allocates
 *     or frees device memory: scratch lives in the caller's workspace `ws`
 *     (size from hos_workspace_size, 256-byte aligned).
 *   - All work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and the call returns without synchronising.
 *   - Argument errors return synchronously and enqueue nothing.  A launch
 *     failure returns HOS_ERR_CUDA.  Failures detected on the device (a wait
 *     that ran past its time limit) are written to a status word in `ws`;
 *     read it with hos_get_device_status after the stream completes.
 *   - Complex outputs are interleaved float pairs (re, im), i.e. complex64.
 *   - A workspace may be reused by consecutive calls on one stream; calls
 *     that overlap in time need separate workspaces.
 */
#ifndef HOS_H
#define HOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* hos_stream_t; /* identical to cudaStream_t */

typedef enum {
    HOS_OK = 0,
    HOS_ERR_INVALID_ARG = 1,  /* bad size, null pointer, bad enum value */
    HOS_ERR_UNSUPPORTED = 2,  /* valid but not implemented (e.g. L too large for a path) */
    HOS_ERR_WORKSPACE = 3,    /* ws too small or misaligned */
    HOS_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed */
    HOS_ERR_TIMEOUT = 5,      /* device status: a wait inside a kernel hit its limit */
    HOS_ERR_DEVICE_FAULT = 6  /* device status: an internal consistency check failed */
} hos_status;

typedef enum { HOS_F32 = 0, HOS_F64 = 1 } hos_dtype;

/* Arithmetic of the cumulant contraction (the dominant step).
 *   FP32        : 3xTF32 split products on the tensor cores (tcgen05 kind::tf32),
 *                 FP32 accumulation, FP64-class cross-tile reduction (~1e-6);
 *   SPLIT_BF16  : x = hi + lo in bf16, three products on the tensor cores
 *                 (tcgen05 kind::f16), FP32 accumulation, FP64-class
 *                 reduction (~1e-5);
 *   TF32        : one plain TF32 product per term (tcgen05 kind::tf32, the
 *                 factors rounded to 10 mantissa bits), FP32 accumulation:
 *                 about 1e-4 to 1e-3, for comparison only (no accuracy
 *                 target); the adjoint runs it on the CUDA cores;
 *   SIMT_FP32   : plain FP32 FFMA on the CUDA cores (cross-check path);
 *   SPLIT_FP16  : FP32-class like FP32 at the speed of SPLIT_BF16: each
 *                 series is scaled by a power of two (exact) that puts its
 *                 largest |y| at 2^7 (2^4 for the fourth order), then
 *                 x = hi + lo in FP16 (11 + 11 significant bits), three
 *                 products on the tensor cores (tcgen05 kind::f16, F16
 *                 operands), FP32 accumulation over half as many MMA steps
 *                 as 3xTF32; the scale is divided out in the FP64-class
 *                 reduction.  The adjoint runs it on the CUDA cores.
 * Mean removal is FP64.  The cross-chunk reduction and c2 are FP64-class in
 * every mode: double-float sums (two floats, TwoSum / FMA, about 44-48
 * significant bits) on the FP32 pipes, since GB300 issues FP64 at about 1/64
 * of its FP32 rate.                                                        */
typedef enum {
    HOS_PREC_FP32 = 0,
    HOS_PREC_SPLIT_BF16 = 1,
    HOS_PREC_TF32 = 2,
    HOS_PREC_SIMT_FP32 = 3,
    HOS_PREC_SPLIT_FP16 = 4
} hos_precision;

/* Lag windows.  PARZEN: d(w1)d(w2)[d(w3)] (separable).  PARZEN_SYM (bispectrum
 * only): d(w1)d(w2)d(w1-w2), which keeps c3's six-fold symmetry.  RECT: 1 for
 * every |w| <= L-1.                                                        */
typedef enum { HOS_WIN_PARZEN = 0, HOS_WIN_PARZEN_SYM = 1, HOS_WIN_RECT = 2 } hos_window;

typedef enum {
    HOS_OP_BISPECTRUM = 0,
    HOS_OP_TRISPECTRUM = 1,
    HOS_OP_BISPECTRUM_BATCHED = 2,
    HOS_OP_BISPECTRUM_BACKWARD = 3,
    HOS_OP_CUMULANT3 = 4,
    HOS_OP_CUMULANT4 = 5,
    HOS_OP_SERIES_SUM = 6,
    HOS_OP_CUMULANT3_SLICE = 7,
    HOS_OP_BISPECTRUM_FROM_C3 = 8,
    HOS_OP_TRISPECTRUM_BATCHED = 9,
    HOS_OP_TRISPECTRUM_BACKWARD = 10,
    HOS_OP_MOMENTS4_SLICE = 11,
    HOS_OP_TRISPECTRUM_FROM_MOMENTS = 12
} hos_op;

typedef struct {
    int32_t L;            /* maximum lag, 1 <= L <= 1024 (trispectrum: L <= 64) */
    int32_t nfft;         /* grid points per axis; 0 -> 2L; otherwise >= 2L    */
    int32_t precision;    /* hos_precision                                      */
    int32_t window;       /* hos_window                                         */
    int32_t remove_mean;  /* nonzero: subtract each part's mean (FP64)          */
    int32_t segment_len;  /* 0: one part (K = 1); else parts of this many
                             samples (the last may be shorter), each part's
                             cumulant uses its own length, estimates averaged
                             (Algorithm DBS steps 1, 2, 6)                      */
    int32_t tile_n;       /* 0: automatic; else 128 or 256: width of the lag
                             tile one CTA accumulates (tuning knob)             */
    int32_t flush_chunks; /* 0: automatic; else the most 1024-sample chunks one
                             tile accumulates in FP32 before its partial sum is
                             handed to the cross-chunk reduction (tuning knob)  */
    int32_t segment_overlap; /* 0: parts do not overlap.  Else 1 <= overlap <
                             segment_len: parts of exactly segment_len samples
                             start every segment_len - overlap samples, K =
                             floor((n - segment_len) / (segment_len - overlap))
                             + 1 of them; samples past the last whole part are
                             not used; n <= segment_len gives one part.  The
                             parts are copied one after another into the
                             workspace (K * segment_len samples, counted by
                             hos_workspace_size) and averaged as above.  Only
                             hos_bispectrum, hos_trispectrum, hos_cumulant3,
                             hos_cumulant4 (and the no-allocation entry)
                             accept it; the others return
                             HOS_ERR_INVALID_ARG for a nonzero value.         */
    int32_t chunk_len;    /* 0: automatic; else samples of the time index one
                             contraction step covers before moving on (a
                             multiple of 64, at most 1024; tuning knob: a
                             shorter chunk makes shorter FP32 sums per partial
                             and more partials to reduce)                      */
} hos_params;

/* Bytes of workspace an operation needs.
 *   op        : hos_op
 *   n_total   : samples (batched: total over all series)
 *   n_series  : number of series (1 unless batched)
 *   max_len   : longest series (batched), else n_total
 * Returns HOS_ERR_INVALID_ARG for bad params.                              */
hos_status hos_workspace_size(int32_t op, int64_t n_total, int32_t n_series, int64_t max_len,
                              const hos_params* params, size_t* bytes);

/* Smoothed sample bispectrum of one series.
 *   d_x : n samples (dtype float32 or float64)
 *   d_B : nfft*nfft complex64, row-major [k1][k2]
 * c3 of a zero-padded series (or part) takes one value at the six lag pairs
 * (w1, w2), (w2, w1), (-w1, w2 - w1) and their swaps; where that needs
 * fewer tiles than the swap symmetry alone (L >= 128 with the default tile
 * width), the contraction computes one pair of each six (w1 in [0, L), w2 in
 * [w1, w1 + L)) and the grid takes every lag pair's value from it.  The
 * result equals the window
 * and transform of hos_cumulant3's c3 (hos_bispectrum_from_cumulant) within
 * the precision's target; with the environment variable HOS_TILE_SCHEME=swap
 * both contract the same lag pairs and agree bit for bit.                  */
hos_status hos_bispectrum(const void* d_x, int32_t dtype, int64_t n, const hos_params* params, void* d_B,
                          void* ws, size_t ws_bytes, hos_stream_t stream);

/* Smoothed sample trispectrum of one series.
 *   d_T : nfft^3 complex64, row-major [k1][k2][k3]                         */
hos_status hos_trispectrum(const void* d_x, int32_t dtype, int64_t n, const hos_params* params, void* d_T,
                           void* ws, size_t ws_bytes, hos_stream_t stream);

/* Bispectra of S independent series of uneven length in one pass.
 *   d_x       : concatenated samples, n_total of them
 *   d_offsets : S+1 int64, series s is d_x[offsets[s] .. offsets[s+1]),
 *               nondecreasing, offsets[0] = 0, offsets[S] = n_total
 *   max_len   : an upper bound on any series length (sizes the workspace)
 *   d_B       : S * nfft^2 complex64, series-major
 * A series of length 0 yields B = 0.  segment_len must be 0.              */
hos_status hos_bispectrum_batched(const void* d_x, int32_t dtype, const int64_t* d_offsets, int32_t S,
                                  int64_t n_total, int64_t max_len, const hos_params* params, void* d_B, void* ws,
                                  size_t ws_bytes, hos_stream_t stream);

/* Trispectra of S independent series of uneven length in one pass (the
 * fourth-order counterpart of hos_bispectrum_batched; tensor-core precisions
 * only, SIMT_FP32 returns HOS_ERR_UNSUPPORTED).
 *   d_offsets, max_len : as hos_bispectrum_batched
 *   d_T       : S * nfft^3 complex64, series-major, each [k1][k2][k3]
 * A series of length 0 yields T = 0.  segment_len must be 0.              */
hos_status hos_trispectrum_batched(const void* d_x, int32_t dtype, const int64_t* d_offsets, int32_t S,
                                   int64_t n_total, int64_t max_len, const hos_params* params, void* d_T, void* ws,
                                   size_t ws_bytes, hos_stream_t stream);

/* ---- fourth order over time slices ----------------------------------------
 * The trispectrum's m4 and c2 are sums over time too: rank r sums over its
 * own samples i in [a_r, b_r), reading up to L samples before the slice and
 * 2L - 1 after it (the c2 lags reach 2L - 1) as lags only.  After FP64 sum
 * all-reduces of the series' total (hos_series_sum), then of m4 and c2,
 * hos_trispectrum_from_moments forms c4 = m4 - (three c2 c2 products) and
 * transforms it, in the same FP32 arithmetic as hos_trispectrum.
 *
 * hos_moments4_slice (op HOS_OP_MOMENTS4_SLICE; tensor-core precisions,
 * L <= 64, segment_len = 0):
 *   d_x        : halo_before + n_slice + halo_after samples (this slice with
 *                its neighbours' samples around it)
 *   halo_before <= L, halo_after <= 2L (fewer at the series' ends)
 *   d_sum      : 1 double, the whole series' sum (all slices added)
 *   n_total    : length of the whole series (the 1/n of the time average)
 *   d_m4       : (2L)^3 doubles [w1+L][w2+L][w3+L]: (1/n_total) sum over the
 *                slice's i of y(i) y(i+w1) y(i+w2) y(i+w3), y = x - mean
 *   d_c2       : 4L - 1 doubles, index t + 2L - 1: (1/n_total) sum over the
 *                slice's i of y(i) y(i+|t|) (c2 is even in t once joined)
 * hos_trispectrum_from_moments (op HOS_OP_TRISPECTRUM_FROM_MOMENTS):
 *   d_m4, d_c2 : the joined sums; d_T: nfft^3 complex64 as hos_trispectrum.  */
hos_status hos_moments4_slice(const void* d_x, int32_t dtype, int64_t n_slice, int64_t halo_before, int64_t halo_after,
                              const double* d_sum, int64_t n_total, const hos_params* params, double* d_m4,
                              double* d_c2, void* ws, size_t ws_bytes, hos_stream_t stream);
hos_status hos_trispectrum_from_moments(const double* d_m4, const double* d_c2, const hos_params* params, void* d_T,
                                        void* ws, size_t ws_bytes, hos_stream_t stream);

/* Adjoint of hos_bispectrum (one part only, segment_len = 0): the gradient of a
 * real loss l through B.
 *   d_dB : nfft^2 complex64 holding dl/dRe B + i dl/dIm B
 *   d_dx : n values, same dtype as d_x, receives dl/dx (overwritten)
 * Steps: adjoint transform and window, symmetrised; the two contractions of
 * the triple-product loop's derivative; the mean-removal adjoint.          */
hos_status hos_bispectrum_backward(const void* d_x, int32_t dtype, int64_t n, const hos_params* params,
                                   const void* d_dB, void* d_dx, void* ws, size_t ws_bytes, hos_stream_t stream);

/* Adjoint of hos_trispectrum (one part only, segment_len = 0; L <= 64;
 * window PARZEN or RECT; precision SPLIT_BF16 or SPLIT_FP16 -- anything else
 * returns HOS_ERR_UNSUPPORTED): the gradient of a real loss l through T.
 *   d_dT : nfft^3 complex64 holding dl/dRe T + i dl/dIm T, [k1][k2][k3]
 *   d_dx : n values, same dtype as d_x, receives dl/dx (overwritten)
 * Steps, the chain rule in reverse through the forward (the Problem
 * Statement's trispectrum as the transform of the windowed c4): adjoint
 * 3-D transform and window, symmetrised over the six orders of the lags;
 * through c4 = m4 - (three c2 c2 products), dl/dc2; the fourth-moment
 * loop's derivative as one tensor-core contraction
 * D[u, (w1, w2)] = sum_w3 y(u + w3) Gs(w1, w2, w3) whose epilogue forms
 * E(u, w1) = sum_w2 D y(u + w2) and the two gradient terms; the c2 loop's
 * derivative; the mean-removal adjoint.  Workspace grows as
 * ((2L)^2 / 128) * n * 4 bytes for the per-block row partials.            */
hos_status hos_trispectrum_backward(const void* d_x, int32_t dtype, int64_t n, const hos_params* params,
                                    const void* d_dT, void* d_dx, void* ws, size_t ws_bytes, hos_stream_t stream);

/* Third-order sample cumulant, unwindowed, FP64.
 *   d_c3 : (2L)*(2L) doubles, row-major [w1+L][w2+L], w in [-L, L-1]
 * With segment_len > 0 it is the average of the parts' cumulants.          */
hos_status hos_cumulant3(const void* d_x, int32_t dtype, int64_t n, const hos_params* params, double* d_c3,
                         void* ws, size_t ws_bytes, hos_stream_t stream);

/* Fourth-order sample cumulant, unwindowed, FP64.
 *   d_c4 : (2L)^3 doubles, row-major [w1+L][w2+L][w3+L], w in [-L, L-1]    */
hos_status hos_cumulant4(const void* d_x, int32_t dtype, int64_t n, const hos_params* params, double* d_c4,
                         void* ws, size_t ws_bytes, hos_stream_t stream);

/* ---- One long series cut into time slices (one slice per GPU) -----------
 * The time average c3(w1,w2) = (1/n) sum_i y(i)y(i+w1)y(i+w2) (Problem
 * Statement) is a sum over i, so cutting i into slices [a_r, b_r) gives
 * c3 = sum_r c3_r, where c3_r sums only the slice's i.  A slice needs its own
 * samples, up to L samples on each side (its neighbours' halo) and the
 * series' mean.  Per rank:
 *   1. hos_series_sum over the slice's own samples; sum the ranks' sums
 *      (FP64 all-reduce): the series' total;
 *   2. hos_cumulant3_slice with that total;
 *   3. sum the ranks' c3 (FP64 all-reduce of (2L)^2 doubles);
 *   4. hos_bispectrum_from_cumulant on the summed c3.
 * Up to FP64 rounding the result equals one hos_cumulant3 / hos_bispectrum
 * call over the whole series.                                              */

/* FP64 sum of d_x[0..n) into d_sum[0] (device), in a fixed order.
 * Workspace: hos_workspace_size(HOS_OP_SERIES_SUM, n, 1, n, params, ...)
 * (params may be NULL there).                                              */
hos_status hos_series_sum(const void* d_x, int32_t dtype, int64_t n, double* d_sum, void* ws, size_t ws_bytes,
                          hos_stream_t stream);

/* One slice's share of c3 of a longer series.
 *   d_x         : halo_before + n_slice + halo_after samples: the slice
 *                 [a, a + n_slice) preceded by samples [a - halo_before, a)
 *                 and followed by [a + n_slice, a + n_slice + halo_after);
 *                 0 <= halo_* <= L, fewer than L only at the series' ends
 *                 (outside the series the samples are zero)
 *   d_sum       : device pointer to the FP64 sum of the whole series; the
 *                 mean removed is *d_sum / n_total when params->remove_mean
 *   n_total     : length of the whole series (the estimator's 1/n)
 *   d_c3        : (2L)^2 doubles in hos_cumulant3's layout, receives
 *                 (1/n_total) sum over i in the slice of y(i)y(i+w1)y(i+w2)
 * segment_len must be 0.  Workspace: as hos_cumulant3 for n_slice samples
 * (hos_workspace_size(HOS_OP_CUMULANT3_SLICE, n_slice, 1, n_slice, ...)).   */
hos_status hos_cumulant3_slice(const void* d_x, int32_t dtype, int64_t n_slice, int64_t halo_before,
                               int64_t halo_after, const double* d_sum, int64_t n_total, const hos_params* params,
                               double* d_c3, void* ws, size_t ws_bytes, hos_stream_t stream);

/* The last steps of hos_bispectrum from a given c3 (hos_cumulant3's layout):
 * lag window, (2 pi)^-2, wrap onto the nfft grid, 2-D DFT into d_B (as
 * hos_bispectrum).  The window and scale use the same FP32 arithmetic as
 * hos_bispectrum's swap plan, so c3 from hos_cumulant3 reproduces its output
 * bit for bit under HOS_TILE_SCHEME=swap, and within the precision's target
 * under the default six-fold plan.
 * Workspace: hos_workspace_size(HOS_OP_BISPECTRUM_FROM_C3, 0, 1, 0, ...).   */
hos_status hos_bispectrum_from_cumulant(const double* d_c3, const hos_params* params, void* d_B, void* ws,
                                        size_t ws_bytes, hos_stream_t stream);

/* ---- The paper's direct method (Algorithm DBS) ------------------------------
 * Steps: 1-2. parts of M samples starting every M - overlap samples (overlap
 * 0: the paper's partition into K = floor(n / M) parts; otherwise K =
 * floor((n - M) / (M - overlap)) + 1; samples past the last whole part are
 * not used), each minus its own mean (FP64) when remove_mean;
 * 3. F_p(k) = sum_u X_p(u) e^{-j 2 pi u k / M}; 4. raw (1/M) F_p(k1) F_p(k2)
 * F_p*(k1+k2) (reading: the third factor conjugated), indices mod M, on the
 * whole M x M grid; 5. M3 x M3 box average over offsets lo .. lo + M3 - 1,
 * lo = -floor(M3/2) (the paper's -M3/2 .. M3/2 - 1 for even M3), indices mod
 * M, computed by window sums (Algorithms WS / WS_PRAM); 6. average over the
 * parts (done before step 5: both are linear).  No (2 pi) normalisation.
 *   M    : part length and transform size: a power of two up to 8192, or any
 *          value 2..2048; M + M3 - 1 <= 13504
 *   M3   : side of the smoothing box, 1 <= M3 <= M (1: no smoothing)
 *   overlap : samples shared by consecutive parts, 0 <= overlap < M
 *   d_B  : M * M complex64, row-major [k1][k2]; the principal domain
 *          0 <= k2 <= k1, k1 + k2 < M/2 is the part the paper keeps
 * The transform is FP32; the running window sums are double-float.
 * Workspace: hos_bispectrum_direct_workspace_size.                          */
hos_status hos_bispectrum_direct_workspace_size(int64_t n, int32_t M, int32_t M3, int32_t overlap, size_t* bytes);
hos_status hos_bispectrum_direct(const void* d_x, int32_t dtype, int64_t n, int32_t M, int32_t M3, int32_t overlap,
                                 int32_t remove_mean, void* d_B, void* ws, size_t ws_bytes, hos_stream_t stream);

/* Bispectrum without a caller-supplied workspace, for callers that cannot
 * allocate device memory (no allocator at hand, or a context where calling
 * cudaMalloc is not allowed, such as a host callback or a plug-in whose host
 * owns all allocations).  The paper has no counterpart: this is a deployment
 * convenience.
 *
 * Same arguments and result as hos_bispectrum, minus `ws`/`ws_bytes`.  The
 * scratch is a fixed array of HOS_NOALLOC_SCRATCH_BYTES inside the library:
 * every GPU that loads the library holds that much device memory until the
 * process exits.  A problem whose hos_workspace_size exceeds it returns
 * HOS_ERR_WORKSPACE and enqueues nothing (for example split-bf16 with the
 * default tiles fits n = 2^20 at L = 32).  Nothing is allocated or freed.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.  All calls on a device share the one
 * array, which keeps the previous call's contents (each call clears the
 * status word it needs at zero): calls that overlap in time on the GPU
 * (different streams, or different host threads) race with each other and
 * must be serialised by the caller.  A device-side timeout is recorded in
 * the array's own status word; read it with hos_bispectrum_noalloc_status
 * once the stream has completed (the next call clears it).  After a device
 * reset the address is looked up again on the next call.                   */
#define HOS_NOALLOC_SCRATCH_BYTES (32u << 20)
hos_status hos_bispectrum_noalloc(const void* d_x, int32_t dtype, int64_t n, const hos_params* params, void* d_B,
                                  hos_stream_t stream);

/* Read (synchronously) the device status word of the current device's
 * no-allocation scratch array, as hos_get_device_status does for a caller's
 * workspace: *status = HOS_OK, HOS_ERR_TIMEOUT or HOS_ERR_DEVICE_FAULT for
 * the last hos_bispectrum_noalloc call on this device.  Call it after that
 * call's stream has completed.  Allocates nothing.                          */
hos_status hos_bispectrum_noalloc_status(int32_t* status);

/* Host-only consistency check of a contraction plan (no GPU is touched): the
 * series layout, every CTA's walk over the cost-weighted work split, the slot
 * each partial tile goes to, the reduction's reading of those slots, and the
 * bounds and 16-byte alignment of every bulk copy the producer would issue,
 * run on the CPU with the code the kernels use.
 *   op        : HOS_OP_BISPECTRUM (one series, parts by segment_len),
 *               HOS_OP_BISPECTRUM_BATCHED (h_offsets: S+1 HOST int64), or
 *               HOS_OP_TRISPECTRUM (tensor-core fourth-order plan)
 *   ctas      : 0 = the plan's own CTA count on the current device; else this many
 *   msg       : optional text buffer for the first violation (or a summary)
 * Returns HOS_OK, HOS_ERR_DEVICE_FAULT for an inconsistent plan, or the
 * argument error the entry point would return.                            */
hos_status hos_check_plan(int32_t op, int64_t n_total, int32_t n_series, const int64_t* h_offsets,
                          const hos_params* params, int32_t ctas, char* msg, size_t msg_len);

/* Read (synchronously) the device status word of a workspace that a finished
 * call used.  *status = HOS_OK, HOS_ERR_TIMEOUT or HOS_ERR_DEVICE_FAULT.     */
hos_status hos_get_device_status(const void* ws, int32_t* status);

/* Clear the device status word (enqueued on stream).                        */
hos_status hos_reset_device_status(void* ws, hos_stream_t stream);

/* Failure-detection self test: one CTA waits on a barrier that nothing
 * signals, with a wait limit of timeout_us microseconds, then records
 * HOS_ERR_TIMEOUT in the workspace status word and exits cleanly (no trap,
 * no fault).  Lets a caller check that device-side timeouts are reported.   */
hos_status hos_selftest_timeout(void* ws, size_t ws_bytes, int32_t timeout_us, hos_stream_t stream);

/* Tracing.  When enabled, each call records CUDA events around its stages on
 * its stream; hos_get_stage_times synchronises on the last call's events and
 * returns per-stage milliseconds in stage order (prep, contraction, reduce,
 * transform, ...), with names from hos_stage_name.  Not for use while a
 * stream is being captured into a graph.                                   */
hos_status hos_set_profiling(int32_t enable);
hos_status hos_get_stage_times(float* ms, int32_t max_stages, int32_t* n_stages);
const char* hos_stage_name(int32_t i);

/* Total kernels this library has launched in the process (all devices).    */
int64_t hos_launch_count(void);

/* Name of the contraction kernel variant the last call used.               */
const char* hos_last_contraction(void);

/* The last call's contraction plan as text: the widest lag tile, the tile
 * count and widths, the flush length, chunk length, CTAs and products per
 * term (what an autotuner chose, or the automatic choice).                 */
const char* hos_last_plan(void);

const char* hos_status_string(int32_t status);
const char* hos_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HOS_H */
