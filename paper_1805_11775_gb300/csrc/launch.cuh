// launch.cuh -- parameter blocks of the kernels and the host-side launch
// wrappers the ABI layer calls.  Each wrapper enqueues on `stream`, counts the
// launch, and returns the launch error.
#pragma once

#include "hos_internal.cuh"

namespace hos {

struct C3TcParams {
    C3Geom geom;
    SeriesView ser;
    const float* y32;
    const void* hi;
    const void* lo;
    float* partials;
    int* status;
    uint64_t limit_ns;
    int products;       // 3: hi*hi + hi*lo + lo*hi (split precision); 1: hi*hi (plain TF32)
    int64_t plane_len;  // samples in each plane (bounds of the HOS_DEBUG_BOUNDS build)
    int64_t n_slots;    // partial slots in the workspace (same)
    // waits of each role (mbar_wait's hint_ns): producer, builders, epilogue, MMA issuer
    uint32_t hint[4];
};

struct C3SimtParams {
    C3Geom geom;
    SeriesView ser;
    const float* y32;
    float* partials;
};

// mode 0: spectrum input grid[g][(w2 mod Nf)][(w1 mod Nf)] = scale * W * c3 (fp32)
// mode 1: raw cumulant c3out[g][w2+L][w1+L] (fp64, symmetric so also [w1][w2])
// Where the parts of one (series, computed tile) live (reduce.cu).
struct TileRec {
    int64_t slot;   // first main slot: one per flush window, contiguous
    int64_t ub;     // cost position where (series, tile) starts
    int32_t nwin;   // main slots
    int32_t xlo;    // CTAs [xlo, xhi) whose first unit lies inside (series, tile), after its first
    int32_t xhi;
    int32_t k;      // cost of one chunk of the tile (its width / 32)
};

// The record of (series s, computed tile t), from the CTAs' first cost
// positions bnd[0..G] (shared by the reduction and the host plan check).
HOS_HD TileRec tile_record(const C3Geom& geo, const SeriesView& sv, const int64_t* bnd, int s, int t) {
    const int64_t len = sv.off[s + 1] - sv.off[s];
    const int64_t nch = ceil_div(len, geo.kc), nwin = ceil_div(nch, geo.flush);
    const int64_t k = geo.tile_w32[t];
    const int64_t ub = sv.unit[s] + nch * geo.tile_kpre[t];
    const int64_t last = ub + (nch - 1) * k;  // cost start of the tile's last chunk
    int lo = 0, hi = geo.G;  // first CTA starting after ub
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (bnd[mid] > ub) hi = mid; else lo = mid + 1;
    }
    int e = lo, eh = geo.G;  // first CTA from lo on whose first unit is past this tile (G if none)
    while (e < eh) {
        const int mid = (e + eh) >> 1;
        if (bnd[mid] > last) eh = mid; else e = mid + 1;
    }
    TileRec r;
    r.slot = sv.win[s] + (int64_t)t * nwin;
    r.ub = ub;
    r.nwin = (int)nwin;
    r.xlo = lo;
    r.xhi = nch > 0 ? e : lo;
    r.k = (int32_t)k;
    return r;
}

// Whether CTA g (xlo <= g < xhi) wrote a part of this (series, tile) to its
// own slot: its first chunk there, ceil((bnd[g] - ub) / k), starts mid flush
// window and inside the CTA's range.
HOS_HD bool cta_slot_used(const TileRec& r, const int64_t* bnd, int g, int flush) {
    if (g < r.xlo || g >= r.xhi) return false;
    const int64_t c = ceil_div(bnd[g] - r.ub, r.k);
    return c % flush != 0 && r.ub + c * r.k < bnd[g + 1];
}

// The image (b, a) of (w1, w2) with 0 <= b <= a: each sector of the lag
// plane, told apart by the signs of w1, w2 and w2 - w1, maps to one of the
// six images.  For (w1, w2) in (-L, L)^2 it is the pair's image in the
// fundamental set.
HOS_HD void c3_sector_image(int w1, int w2, int& b, int& a) {
    if (w1 >= 0 && w2 >= 0) {
        b = w1 < w2 ? w1 : w2;
        a = w1 < w2 ? w2 : w1;
    } else if (w2 >= 0) {  // w1 < 0
        b = -w1;
        a = w2 - w1;
    } else if (w1 >= 0) {  // w2 < 0
        b = -w2;
        a = w1 - w2;
    } else if (w2 >= w1) {  // both < 0
        b = w2 - w1;
        a = -w1;
    } else {
        b = w1 - w2;
        a = -w2;
    }
}

struct Reduce3Params {
    C3Geom geom;
    SeriesView ser;
    const float* partials;
    int window;
    int nfft;
    int mode;
    int per_series_groups;
    double scale;
    float* grid;
    double* c3out;
    int64_t norm_len;  // > 0: divide by this length instead of each series' own (a time slice)
    // six-fold plans: the reduced c3 of each (group, tile), written in place over the
    // first window slot of the group's first part and unfolded onto the grid from there
    float* tiles_out;
    // bounds of the HOS_DEBUG_BOUNDS build's checks: partial slots, grid floats, status word
    int64_t n_slots;
    int64_t grid_floats;
    int* status;
};

struct LineGeom {
    int N;
    int log2N;  // -1 when N is not a power of two
    int64_t nlines;
    int64_t inner;
    int64_t outer_stride;
    int64_t elem_stride;
    int lpb;       // lines per CTA
    int half_out;  // real-input lines: write only k = 0..N/2 (the rest is their conjugate mirror)
    int herm;      // 2-D grid of a real array: the lines are columns c = 0..N/2 of each group, and
                   // each also fills column N - c as B(N - k, N - c) = conj B(k, c)
};

struct C4ReduceArgs {
    int window;
    int nfft;
    int mode;  // 0: windowed transform grid (fp32), 1: raw c4 (fp64), 2: raw m4 (fp64, time slices)
    double scale;
    float* grid;
    double* c4out;
};

// m4 contraction geometry shared by the host plan and the kernels
constexpr int C4_PAIRS_PER_CTA = 128;
constexpr int C4_CHUNK_GROUP = 4;  // 1024-sample chunks per FP32 partial

void count_launch();
// Identifier of the current CUDA context (changes when a device is reset), or 0
// when no context is current or the driver cannot say (abi.cu).
uint64_t current_context_id();

// ktot: cost of one chunk over all tiles (the contraction's C3Geom::ktot)
cudaError_t launch_plan_series(int mode, int64_t n, int64_t seg, const int64_t* d_user_off, int S, int L, int ntiles,
                               int ktot, int flush, int kc, int pad_tail, int64_t* off, int64_t* pad, int64_t* unit,
                               int64_t* win, cudaStream_t st);
// remove_mean < 0: write each series' plain FP64 sum instead of its mean
cudaError_t launch_mean(const void* x, int dtype, const int64_t* off, int S, int nslices, double* part,
                        int remove_mean, double* mean, cudaStream_t st);
// ext_lo / ext_hi: halo samples before / after a time slice (see planes_kernel)
// split 3 (f16 planes) scales each series by scale[s]
cudaError_t launch_planes(const void* x, int dtype, const int64_t* off, const int64_t* pad, const double* mean, int L,
                          int split, float* y32, void* hi, void* lo, int S, int blocks_x, cudaStream_t st,
                          int64_t ext_lo = 0, int64_t ext_hi = 0, const float* scale = nullptr);
// scale[s] = 2^(top - e), 2^e the least power of two >= max |x - mean| over
// series s and the ext_lo / ext_hi halo samples around it (mx: S scratch words)
cudaError_t launch_series_scale(const void* x, int dtype, const int64_t* off, const double* mean, int S,
                                int nslices, int64_t ext_lo, int64_t ext_hi, int top, unsigned* mx, float* scale,
                                cudaStream_t st);
cudaError_t launch_window_c3(const double* c3, int L, int window, int Nf, double scale, float* wtab, float* grid,
                             cudaStream_t st);
cudaError_t launch_gather_parts(const void* x, int dtype, int64_t K, int64_t m, int64_t step, void* out,
                                cudaStream_t st);
cudaError_t launch_series_sum(const void* x, int dtype, int64_t n, int nslices, int64_t* off, double* part,
                              double* sum, cudaStream_t st);
// direct method (direct.cu)
cudaError_t launch_part_prep(const void* x, int dtype, int64_t K, int64_t M, int64_t step, int remove_mean,
                             double* mean, float* y, cudaStream_t st);
cudaError_t launch_direct_smooth(const float2* F, int K, int M, int M3, float2* R, float2* Cw, float2* B,
                                 cudaStream_t st);
cudaError_t launch_slice_mean(const double* sum, int64_t n_total, int remove_mean, double* mean, cudaStream_t st);
// fmt: FMT_BF16, FMT_F16 or FMT_TF32 (operand format); order 3 (c3) or 4 (m4)
cudaError_t launch_c3_tc(int fmt, int order, const C3TcParams& p, int G, cudaStream_t st);
cudaError_t launch_c3_simt(const C3SimtParams& p, int G, cudaStream_t st);
// max_len: longest series (or part); it only sets how threads split the work.
cudaError_t launch_reduce3(const Reduce3Params& p, int groups, int64_t max_len, int64_t* bnd, TileRec* rec,
                           float2* inv_len, float* wtab, cudaStream_t st);
cudaError_t launch_zero_f32(float* p, int64_t n, cudaStream_t st);
cudaError_t launch_twiddles(int N, float2* tw, cudaStream_t st);
cudaError_t launch_lines(bool real_in, const void* in, float2* out, LineGeom g, const float2* tw, int sign,
                         float scale, cudaStream_t st);
cudaError_t launch_c4(const float* y32, const int64_t* off, const int64_t* pad, const int64_t* win, int S, int L,
                      int CG, int64_t total_groups, double* c2, float* partials, const C4ReduceArgs& r,
                      cudaStream_t st);
cudaError_t launch_adjoint(const float* yS, int64_t n, int L, const float2* Gc, int N, int window, double scale,
                           float* Gs, float* T1, float* t2p, float* g, cudaStream_t st);
cudaError_t launch_adjoint_finish(const float* g, int64_t n, const double* gmean, int remove_mean, int dtype, void* dx,
                                  cudaStream_t st);
constexpr int ADJ_ROWS_PER_CTA = 64;
bool adjoint_tc_supported(int L);
size_t adjoint_tc_gs_bytes(int L, int order = 3);
size_t adjoint_tc_t2_floats(int L, int64_t n, int order = 3);
size_t adjoint_tc_t1_floats(int L, int64_t n, int order = 3);
// fmt FMT_BF16 or FMT_F16; sc (FMT_F16): device {series scale, Gs scale}
cudaError_t launch_adjoint_tc(const float* y32, const uint16_t* hi, const uint16_t* lo, int64_t n, int L,
                              const float* Gs, uint8_t* gsb, float* t1p, float* t2p, float* g, int* status,
                              uint64_t limit_ns, int G, cudaStream_t st, int fmt = FMT_BF16,
                              const float* sc = nullptr);
cudaError_t launch_gs(const float2* Gc, int N, int L, int window, double scale, float* Gs, cudaStream_t st);
// trispectrum adjoint (adjoint.cu, adjoint_tc.cu)
cudaError_t launch_gs4(const float2* Gc, int N, int L, int window, double scale, float* Gs4, cudaStream_t st);
cudaError_t launch_gc2(const float* Gs4, const double* c2, int L, double* gc2, cudaStream_t st);
cudaError_t launch_adjoint4_tc(const float* y32, const uint16_t* hi, const uint16_t* lo, int64_t n, int L,
                               const float* Gs4, uint8_t* gsb, float* t1p, float* t2p, const double* gc2, float* g,
                               int* status, uint64_t limit_ns, int G, cudaStream_t st, int fmt = FMT_BF16,
                               const float* sc = nullptr);
// scale[0] = 2^(top - e), 2^e the least power of two >= max |v[0..count)| (mx: one scratch word)
cudaError_t launch_flat_scale(const float* v, int64_t count, int top, unsigned* mx, float* scale, cudaStream_t st);
cudaError_t launch_m4_tile_reduce(const C3Geom& geo, const SeriesView& sv, int64_t max_len, const float* partials,
                                  int64_t* bnd, TileRec* rec, float2* inv_len, double* m4buf, cudaStream_t st,
                                  int64_t norm_len = 0);
// P slices of each part's samples (c2_slices); c2p: S * (4L - 1) * P float2 when P > 1
int c2_slices(int S, int64_t max_len);
cudaError_t launch_c2(const float* y32, const int64_t* off, const int64_t* pad, int S, int L, int P, double* c2,
                      float2* c2p, cudaStream_t st, int tslice = 0, int64_t norm_len = 0);
cudaError_t launch_c4_from_moments(const double* m4, const double* c2, int L, const C4ReduceArgs& r, cudaStream_t st);
cudaError_t launch_c4_assemble(const double* m4buf, const double* c2, const int64_t* off, int S, int L, int ntiles,
                               int tile_n, const C4ReduceArgs& r, int per_series, cudaStream_t st);
cudaError_t launch_timeout_selftest(int* status, uint64_t limit_ns, cudaStream_t st);

}  // namespace hos
