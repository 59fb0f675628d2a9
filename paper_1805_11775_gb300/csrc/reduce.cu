// reduce.cu -- deterministic FP64-class (double-float) reduction of the
// contraction's FP32 partial tiles into c3, the 1/n time average, the average
// over parts (Algorithm DBS step 6), the lag window, and the wrap of lags onto
// the N-point transform grid (lag w -> index w mod N).
#include "launch.cuh"

namespace hos {

// bnd[g] = first work unit of CTA g, g = 0..G (the contraction's stream-K split)
__global__ void bounds_kernel(const int64_t* __restrict__ unit, int S, int G, int64_t* __restrict__ bnd) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g <= G) bnd[g] = range_begin(g, unit[S], G);
}

constexpr int REDUCE_THREADS = 256;

// For every (series s, computed tile t) a record of where its parts are:
// the main slots (one per flush window, contiguous, in chunk order) and the
// CTAs whose first unit lies inside (s, t) after its first chunk, [xlo, xhi)
// -- those CTAs' first parts, when they begin mid flush-window, live in
// per-CTA slots.  (s, t) covers the cost range [ub, ub + nch k); CTA g's
// first unit is the first chunk starting at or after bnd[g]: chunk
// ceil((bnd[g] - ub) / k), inside the tile when bnd[g] <= ub + (nch - 1) k.
// Also 1/n of each series' time average (divided by scale^scale_pow when the
// planes were scaled: the contraction's products carry the series' scale to
// that power).  bnd (G + 1 values) is staged in shared memory once per block;
// both CTA searches are binary searches there.
__global__ void part_ranges_kernel(const C3Geom geo, const SeriesView sv, const int64_t* __restrict__ bnd_g,
                                   TileRec* __restrict__ rec, float2* __restrict__ inv_len, int64_t norm_len,
                                   int scale_pow) {
    extern __shared__ int64_t bnd[];
    for (int g = threadIdx.x; g <= geo.G; g += blockDim.x) bnd[g] = bnd_g[g];
    __syncthreads();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)sv.S * geo.ntiles) return;
    const int s = (int)(q / geo.ntiles), t = (int)(q % geo.ntiles);
    const TileRec r = tile_record(geo, sv, bnd, s, t);
    const int64_t len = sv.off[s + 1] - sv.off[s];
    rec[q] = r;
    // 1/n of the time average: the series' own length, or (a time slice of a
    // longer series) that series' length
    const int64_t nl = norm_len > 0 ? norm_len : len;
    if (t == 0) {  // as a double-float
        double sp = 1.0;
        if (sv.scale)
            for (int k = 0; k < scale_pow; ++k) sp *= (double)sv.scale[s];  // a power of two: exact
        const double inv = len > 0 ? 1.0 / ((double)nl * sp) : 0.0;
        const float h = (float)inv;
        inv_len[s] = make_float2(h, (float)(inv - (double)h));
    }
}

// Lag-window table: wtab[t] = d(t - 2L) for t in [0, 4L) (the lags and
// their differences), as FP32; RECT: 1 for |w| <= L-1, else 0.
__global__ void window_table_kernel(int L, int kind, float* __restrict__ wtab) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * L) return;
    const int w = t - 2 * L;
    wtab[t] = (kind == HOS_WIN_RECT) ? ((w >= -(L - 1) && w <= L - 1) ? 1.0f : 0.0f) : (float)parzen(w, L);
}

// ---- double-float arithmetic ------------------------------------------------
// GB300 issues FP64 at about 1/64 of its FP32 rate, so the cross-partial sums
// run as unevaluated sums of two floats (h + l, TwoSum and FMA-based
// products: about 44-48 significant bits, FP64-class for a sum whose terms
// carry FP32 rounding) on the FP32 pipes; FP64 appears only where an FP64
// array is written.
struct DF {
    float h, l;
};
HOS_DEV DF df_zero() { return DF{0.0f, 0.0f}; }
// (a.h + a.l) + (b.h + b.l), renormalised
HOS_DEV DF df_add(DF a, DF b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    float e = (a.h - (s - bb)) + (b.h - bb);
    e += a.l + b.l;
    const float h = s + e;
    return DF{h, e - (h - s)};
}
// (a.h + a.l) * (b.h + b.l)
HOS_DEV DF df_mul(DF a, DF b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    const float h = p + e;
    return DF{h, e - (h - p)};
}
HOS_DEV double df_to_double(DF a) { return (double)a.h + (double)a.l; }

// This thread's share of the parts of (series s, computed tile t) at the
// four consecutive elements of vector vi (elements 4 vi .. 4 vi + 3), as
// double-float: the main parts in groups of 16 windows, each group a TwoSum
// chain in window order, groups gi, gi + gsplit, ... added in that order;
// then the parts that start at a CTA boundary inside a window, CTA g on row
// (g - xlo) % gsplit, in CTA order.  Not divided by the length.  Loads go
// BATCH windows at a time.
template <int BATCH>
HOS_DEV void tile_share4(const float* __restrict__ partials, const TileRec& r, int tsz, int vi, int gi, int gsplit,
                         int F, const int64_t* __restrict__ bnd, int64_t total_win, DF (&acc)[4]) {
    const int64_t st4 = tsz >> 2;  // float4 per slot
    const float4* p4 = reinterpret_cast<const float4*>(partials + r.slot * (int64_t)tsz) + vi;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = df_zero();
    if (r.nwin == 1 && gi == 0) {  // one window (short series): the group sum is the value itself
        const float4 x = p4[0];
        acc[0] = DF{x.x, 0.0f};
        acc[1] = DF{x.y, 0.0f};
        acc[2] = DF{x.z, 0.0f};
        acc[3] = DF{x.w, 0.0f};
    }
    for (int f0 = 16 * gi; f0 < r.nwin && r.nwin > 1; f0 += 16 * gsplit) {
        const int cnt = (r.nwin - f0 < 16) ? r.nwin - f0 : 16;
        float hi[4] = {0.0f, 0.0f, 0.0f, 0.0f}, lo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int f = 0; f < cnt; f += BATCH) {
            float4 v[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; ++u)
                v[u] = (f + u < cnt) ? p4[(int64_t)(f0 + f + u) * st4] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int u = 0; u < BATCH; ++u) {
                const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {  // a zero term leaves (hi, lo) unchanged
                    const float sm = hi[c] + x[c];
                    const float bv = sm - hi[c];
                    lo[c] += (hi[c] - (sm - bv)) + (x[c] - bv);
                    hi[c] = sm;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = df_add(acc[c], DF{hi[c], lo[c]});
    }
    // parts that start at a CTA boundary inside a window: CTA g to row
    // (g - xlo) % gsplit, each row's in CTA order, four loads in flight
    constexpr int XB = 4;
    for (int g0 = r.xlo + gi; g0 < r.xhi; g0 += XB * gsplit) {
        float4 x[XB];
#pragma unroll
        for (int u = 0; u < XB; ++u) {
            const int g = g0 + u * gsplit;
            const bool use = cta_slot_used(r, bnd, g, F);
            x[u] = use ? reinterpret_cast<const float4*>(partials + (total_win + g) * (int64_t)tsz)[vi]
                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < XB; ++u) {
            acc[0] = df_add(acc[0], DF{x[u].x, 0.0f});
            acc[1] = df_add(acc[1], DF{x[u].y, 0.0f});
            acc[2] = df_add(acc[2], DF{x[u].z, 0.0f});
            acc[3] = df_add(acc[3], DF{x[u].w, 0.0f});
        }
    }
}

// Adds the gsplit thread rows' shares in row order (deterministic); the
// result is valid in row 0.  Called by every thread of the block.
HOS_DEV void combine_rows4(DF (&v)[4], int ei, int gi, int es, int gsplit, float2* red) {
    if (gsplit == 1) return;
#pragma unroll
    for (int c = 0; c < 4; ++c) red[(gi * es + ei) * 4 + c] = make_float2(v[c].h, v[c].l);
    __syncthreads();
    if (gi == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            DF a = df_zero();
            for (int r = 0; r < gsplit; ++r) {
                const float2 q = red[(r * es + ei) * 4 + c];
                a = df_add(a, DF{q.x, q.y});
            }
            v[c] = a;
        }
    }
    __syncthreads();  // red is reused for the next series
}

// Window, scale and wrap of the c3 values of four consecutive elements
// (elem0 = 4 vi, same lag w2, lags w1 .. w1 + 3) onto the transform grid, or
// the raw values into the lag array; and their mirrors (w2, w1) when the tile
// holding those lags is not computed (c3(w1,w2) = c3(w2,w1)).  Rows past the
// last lag (w1 >= L) are padding.
HOS_DEV void emit_c3x4(const Reduce3Params& P, const float* __restrict__ wtab, int grp, int t, int elem0,
                       const DF (&v)[4]) {
    const C3Geom& geo = P.geom;
    const int L = geo.L;
    const int m0 = elem0 & (TILE_M - 1), j = elem0 >> 7;
    const int w10 = -L + TILE_M * geo.tile_a[t] + m0, w2 = -L + 32 * geo.tile_c32[t] + j;
    if (w10 >= L || w2 >= L) return;
    const int twoL = 2 * L, Nf = P.nfft;
    // (w2, w1) is computed when column w1 + L lies in row block (w2 + L) / 128's
    // range; the same for the four (row_c0 is a multiple of 32)
    const bool write_mirror = w10 + L < (int)geo.row_c0[(w2 + L) / TILE_M];
    if (P.mode == 1) {
        double* o = P.c3out + (int64_t)grp * twoL * twoL;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int w1 = w10 + c;
            if (w1 >= L) break;
            const double d = df_to_double(v[c]);
            o[(int64_t)(w2 + L) * twoL + (w1 + L)] = d;
            if (write_mirror) o[(int64_t)(w1 + L) * twoL + (w2 + L)] = d;
        }
        return;
    }
    // window and scale in FP32 (the transform grid is FP32): W = d(w1) d(w2) [d(w1 - w2)]
    float o[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int w1 = w10 + c;
        float wv = wtab[w1 + twoL] * wtab[w2 + twoL];
        if (P.window == HOS_WIN_PARZEN_SYM) wv *= wtab[w1 - w2 + twoL];
        if (P.window == HOS_WIN_RECT && (rect_excluded(w1, L) || rect_excluded(w2, L))) wv = 0.0f;
        o[c] = (v[c].h + v[c].l) * ((float)P.scale * wv);
    }
    float* gr = P.grid + (int64_t)grp * Nf * Nf;
    const int k2 = w2 < 0 ? w2 + Nf : w2;
    const int k10 = w10 < 0 ? w10 + Nf : w10;
    const int64_t at0 = (int64_t)grp * Nf * Nf + (int64_t)k2 * Nf + k10;  // the grid array is 256-byte aligned
    if (w10 + 3 < L && (w10 >= 0 || w10 + 3 < 0) && (at0 & 3) == 0) {  // four live lags, no wrap, 16-byte store
        *reinterpret_cast<float4*>(gr + (int64_t)k2 * Nf + k10) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int w1 = w10 + c;
            if (w1 >= L) break;
            const int k1 = w1 < 0 ? w1 + Nf : w1;
            gr[(int64_t)k2 * Nf + k1] = o[c];
        }
    }
    if (write_mirror) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int w1 = w10 + c;
            if (w1 >= L) break;
            const int k1 = w1 < 0 ? w1 + Nf : w1;
            gr[(int64_t)k1 * Nf + k2] = o[c];
        }
    }
}

// Block = REDUCE_THREADS threads as gsplit rows x es = REDUCE_THREADS / gsplit
// columns.  Column ei owns NV vectors of four consecutive elements (elem =
// j * 128 + m) of computed tile blockIdx.y, output group blockIdx.z: vector
// (blockIdx.x * NV + k) * es + ei.  Rows split the flush windows of long
// series (gsplit > 1 with NV = 1); many short series take NV = 2 instead.
// Per series: sum of its parts / its length; parts (segments) average over
// the group.
// SINGLE_APART: per-series groups whose (series, tile) has one window and no
// mid-window part are left to reduce3_single_kernel (small code, no i-cache
// pressure from the general path); this kernel returns for them.
template <int NV, int BATCH, bool SINGLE_APART = false>
__global__ void __launch_bounds__(REDUCE_THREADS, BATCH >= 16 ? 2 : 3) reduce3_kernel(const Reduce3Params P, const int64_t* __restrict__ bnd,
                                                                 const TileRec* __restrict__ rec,
                                                                 const float2* __restrict__ inv_len,
                                                                 const float* __restrict__ wtab, int gsplit) {
    __shared__ float2 red[REDUCE_THREADS * 4];
    const C3Geom& geo = P.geom;
    const SeriesView& sv = P.ser;
    const int t = blockIdx.y, grp = blockIdx.z;
    // slots hold 128 x tile_n floats; this tile's 128 x width of them are live
    const int tsz = TILE_M * geo.tile_n, nvec = TILE_M * 32 * geo.tile_w32[t] >> 2;
    const int es = REDUCE_THREADS / gsplit, ei = threadIdx.x % es, gi = threadIdx.x / es;
    const int s0 = P.per_series_groups ? grp : 0, s1 = P.per_series_groups ? grp + 1 : sv.S;
    const int64_t total_win = sv.win[sv.S];
    int vi[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) vi[k] = (blockIdx.x * NV + k) * es + ei;
    if (NV > 1 && P.per_series_groups) {
        // one window and no part starting inside (most short series): c3 = x / len,
        // the general path's arithmetic, with all NV vector loads in flight at once
        const TileRec r = rec[(int64_t)grp * geo.ntiles + t];
        if (SINGLE_APART && r.nwin == 1 && r.xlo >= r.xhi) return;
        if (r.nwin == 1 && r.xlo >= r.xhi) {
            const float2 il = inv_len[grp];
            const float4* p4 = reinterpret_cast<const float4*>(P.partials + r.slot * (int64_t)tsz);
            float4 x[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) x[k] = p4[vi[k] < nvec ? vi[k] : 0];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                if (vi[k] >= nvec) continue;
                const float xv[4] = {x[k].x, x[k].y, x[k].z, x[k].w};
                DF v[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c] = df_mul(DF{xv[c], 0.0f}, DF{il.x, il.y});
                emit_c3x4(P, wtab, grp, t, 4 * vi[k], v);
            }
            return;
        }
    }
    DF c3[NV][4];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) c3[k][c] = df_zero();
    int cnt = 0;
    for (int s = s0; s < s1; ++s) {
        const TileRec r = rec[(int64_t)s * geo.ntiles + t];
        if (r.nwin == 0) continue;  // empty series (uniform over the block)
        const float2 il = inv_len[s];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            DF a[4];
            tile_share4<BATCH>(P.partials, r, tsz, vi[k] < nvec ? vi[k] : 0, gi, gsplit, geo.flush, bnd, total_win,
                               a);
            combine_rows4(a, ei, gi, es, gsplit, red);
#pragma unroll
            for (int c = 0; c < 4; ++c) c3[k][c] = df_add(c3[k][c], df_mul(a[c], DF{il.x, il.y}));
        }
        ++cnt;
    }
    if (gi != 0) return;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (vi[k] >= nvec) continue;
        if (!P.per_series_groups && cnt > 1) {  // average over parts (rare: FP64 is fine here)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double q = df_to_double(c3[k][c]) / (double)cnt;
                const float h = (float)q;
                c3[k][c] = DF{h, (float)(q - (double)h)};
            }
        }
        emit_c3x4(P, wtab, grp, t, 4 * vi[k], c3[k]);
    }
}

// Fourth order, tensor-core partials: m4buf[s][t][elem] = sum of the parts of
// (part s, pair tile t) / length, FP64 (elem = (w3 + L) * 128 + pair in tile).
// Same thread layout as reduce3_kernel with NV = 1.
__global__ void __launch_bounds__(REDUCE_THREADS) m4_tile_reduce_kernel(const C3Geom geo, const SeriesView sv,
                                                                        const float* __restrict__ partials,
                                                                        const int64_t* __restrict__ bnd,
                                                                        const TileRec* __restrict__ rec,
                                                                        const float2* __restrict__ inv_len,
                                                                        double* __restrict__ m4buf, int gsplit) {
    __shared__ float2 red[REDUCE_THREADS * 4];
    const int t = blockIdx.y, s = blockIdx.z;
    const int tsz = TILE_M * geo.tile_n, nvec = tsz >> 2;
    const int es = REDUCE_THREADS / gsplit, ei = threadIdx.x % es, gi = threadIdx.x / es;
    const int vi = blockIdx.x * es + ei;
    const TileRec r = rec[(int64_t)s * geo.ntiles + t];
    DF a[4] = {df_zero(), df_zero(), df_zero(), df_zero()};
    if (r.nwin > 0) {  // uniform over the block
        tile_share4<8>(partials, r, tsz, vi < nvec ? vi : 0, gi, gsplit, geo.flush, bnd, sv.win[sv.S], a);
        combine_rows4(a, ei, gi, es, gsplit, red);
    }
    if (gi != 0 || vi >= nvec) return;
    const float2 il = inv_len[s];
    double o[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = df_to_double(df_mul(a[c], DF{il.x, il.y}));
    double2* dst = reinterpret_cast<double2*>(m4buf + ((int64_t)s * geo.ntiles + t) * tsz + 4 * (int64_t)vi);
    dst[0] = make_double2(o[0], o[1]);
    dst[1] = make_double2(o[2], o[3]);
}

// The one-window, no-mid-window-part (series, tile) groups of a per-series
// reduction: c3 = x / len with NV float4 loads in flight per thread, then
// the window and the grid store; other groups return (reduce3_kernel takes
// them).  Same arithmetic as the general path.
template <int NV>
__global__ void __launch_bounds__(REDUCE_THREADS) reduce3_single_kernel(const Reduce3Params P,
                                                                        const TileRec* __restrict__ rec,
                                                                        const float2* __restrict__ inv_len,
                                                                        const float* __restrict__ wtab) {
    const C3Geom& geo = P.geom;
    const int t = blockIdx.y, grp = blockIdx.z;
    const int tsz = TILE_M * geo.tile_n, nvec = TILE_M * 32 * geo.tile_w32[t] >> 2;
    const TileRec r = rec[(int64_t)grp * geo.ntiles + t];
    if (!(r.nwin == 1 && r.xlo >= r.xhi)) return;  // uniform over the block
    const float2 il = inv_len[grp];
    const float4* p4 = reinterpret_cast<const float4*>(P.partials + r.slot * (int64_t)tsz);
    int vi[NV];
    float4 x[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        vi[k] = (blockIdx.x * NV + k) * REDUCE_THREADS + threadIdx.x;
        x[k] = p4[vi[k] < nvec ? vi[k] : 0];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (vi[k] >= nvec) continue;
        const float xv[4] = {x[k].x, x[k].y, x[k].z, x[k].w};
        DF v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = df_mul(DF{xv[c], 0.0f}, DF{il.x, il.y});
        emit_c3x4(P, wtab, grp, t, 4 * vi[k], v);
    }
}

// Rows of threads that split a (series, tile)'s flush windows: one per group
// of 16 windows, at most 8; 1 when the longest series has one group.
static int window_split(const C3Geom& geo, int64_t max_len) {
    const int64_t nch = ceil_div(max_len > 0 ? max_len : 1, geo.kc);
    const int64_t groups = ceil_div(ceil_div(nch, geo.flush), 16);
    int g = 1;
    while (g < 8 && 2 * g <= groups) g *= 2;
    return g;
}

static cudaError_t launch_part_index(const C3Geom& geo, const SeriesView& sv, int64_t* bnd, TileRec* rec,
                                     float2* inv_len, int64_t norm_len, int scale_pow, cudaStream_t st) {
    bounds_kernel<<<(unsigned)ceil_div(geo.G + 1, 256), 256, 0, st>>>(sv.unit, sv.S, geo.G, bnd);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    part_ranges_kernel<<<(unsigned)ceil_div((int64_t)sv.S * geo.ntiles, 256), 256, sizeof(int64_t) * (geo.G + 1), st>>>(
        geo, sv, bnd, rec, inv_len, norm_len, scale_pow);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_m4_tile_reduce(const C3Geom& geo, const SeriesView& sv, int64_t max_len, const float* partials,
                                  int64_t* bnd, TileRec* rec, float2* inv_len, double* m4buf, cudaStream_t st,
                                  int64_t norm_len) {
    cudaError_t e = launch_part_index(geo, sv, bnd, rec, inv_len, norm_len, 4, st);
    if (e != cudaSuccess) return e;
    const int64_t nvec = (int64_t)TILE_M * geo.tile_n / 4;
    const int gsplit = window_split(geo, max_len);
    dim3 grid((unsigned)ceil_div(nvec, REDUCE_THREADS / gsplit), (unsigned)geo.ntiles, (unsigned)sv.S);
    m4_tile_reduce_kernel<<<grid, REDUCE_THREADS, 0, st>>>(geo, sv, partials, bnd, rec, inv_len, m4buf, gsplit);
    count_launch();
    return cudaGetLastError();
}

// Zero the transform grid (entries with no lag when Nf > 2L).
__global__ void zero_f32_kernel(float* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0.0f;
}

// One CTA waits on an mbarrier that nothing signals; the bounded wait gives
// up after limit_ns and records HOS_ERR_TIMEOUT.  No trap, no fault.
__global__ void timeout_selftest_kernel(int* status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, &abort_flag, status, limit_ns);
    __syncthreads();
}

cudaError_t launch_reduce3(const Reduce3Params& p, int groups, int64_t max_len, int64_t* bnd, TileRec* rec,
                           float2* inv_len, float* wtab, cudaStream_t st) {
    cudaError_t e = launch_part_index(p.geom, p.ser, bnd, rec, inv_len, p.norm_len, 3, st);
    if (e != cudaSuccess) return e;
    window_table_kernel<<<(unsigned)ceil_div(4 * p.geom.L, 256), 256, 0, st>>>(p.geom.L, p.window, wtab);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nvec = (int64_t)TILE_M * p.geom.tile_n / 4;
    const int gsplit = window_split(p.geom, max_len);
    if (gsplit == 1 && ceil_div(nvec, REDUCE_THREADS) * p.geom.ntiles * groups >= 4096) {
        // many (short) output groups: four vectors per thread
        dim3 grid((unsigned)ceil_div(nvec, 4 * REDUCE_THREADS), (unsigned)p.geom.ntiles, (unsigned)groups);
        if (p.per_series_groups) {  // one-window groups in their own small kernel
            reduce3_single_kernel<4><<<grid, REDUCE_THREADS, 0, st>>>(p, rec, inv_len, wtab);
            count_launch();
            reduce3_kernel<4, 4, true><<<grid, REDUCE_THREADS, 0, st>>>(p, bnd, rec, inv_len, wtab, 1);
        } else {
            reduce3_kernel<4, 4><<<grid, REDUCE_THREADS, 0, st>>>(p, bnd, rec, inv_len, wtab, 1);
        }
    } else {
        dim3 grid((unsigned)ceil_div(nvec, REDUCE_THREADS / gsplit), (unsigned)p.geom.ntiles, (unsigned)groups);
        // a thread row with several groups of 16 windows keeps all 16 loads of a group in flight;
        // with one group, 8 at a time leave room for a third resident block
        const int64_t nwin_max = ceil_div(ceil_div(max_len > 0 ? max_len : 1, p.geom.kc), p.geom.flush);
        if (nwin_max > 16 * (int64_t)gsplit)
            reduce3_kernel<1, 16><<<grid, REDUCE_THREADS, 0, st>>>(p, bnd, rec, inv_len, wtab, gsplit);
        else
            reduce3_kernel<1, 8><<<grid, REDUCE_THREADS, 0, st>>>(p, bnd, rec, inv_len, wtab, gsplit);
    }
    count_launch();
    return cudaGetLastError();
}

// ---- fused batched tail ---------------------------------------------------------
// For many short series (the batched bispectrum) the reduction, the window and
// both passes of the 2-D transform run in one persistent kernel per series, so
// that the windowed grid and the half-spectrum rows never make an HBM round
// trip: the grid rows live in shared memory, the row transforms go to a
// per-CTA scratch of N x (N/2 + 1) complex values that stays in L2, and only
// the spectrum is written to HBM.  It serves plans whose every row block is one
// tile starting at lag -L (2L <= tile width, N = 2L a power of two, 32..256):
// then the tiles cover the whole lag square and no value is mirrored.
//
// Per series:
//   A. rows of the lag square in chunks of RC lags w1: each element is the
//      series' partials summed in the reduction's order and arithmetic
//      (tile_share4, double-float, 1/n), times the window and (2 pi)^-2 in
//      FP32 as emit_c3x4 does, stored at grid column k2 = w2 mod N; two real
//      rows go through one complex N-point FFT (radix 2 in shared memory) and
//      are separated into their half spectra R[k1][k2], k2 = 0..N/2, written to
//      the scratch transposed (R[k2][k1]);
//   B. columns k2 = 0..N/2 in blocks of 32: the N-point FFT over k1 gives
//      B(k1, k2); the conjugate mirror fills B(N - k1, N - k2) for 0 < k2 < N/2.
constexpr int TAIL_THREADS = 512;
constexpr int TAIL_LINES = 32;  // complex lines per shared-memory FFT batch

HOS_DEV float2 tcmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
HOS_DEV int tsk(int i) { return i + (i >> 4); }  // skewed slot: one pad every 16 (banks)

// In-place radix-2 FFTs of nl lines of N points held bit-reversed in buf
// (line stride SL), forward sign; twiddles tws[k] = e^{-i 2 pi k / N}.
HOS_DEV void tail_fft_lines(float2* buf, int nl, int N, int lg, int SL, const float2* tws) {
    for (int sh = 0; sh < lg; ++sh) {
        const int h = 1 << sh;
        for (int bf = threadIdx.x; bf < nl * (N / 2); bf += blockDim.x) {
            const int l = bf >> (lg - 1), k = bf & ((N >> 1) - 1);
            const int j = k & (h - 1), blk = k >> sh;
            const int i0 = (blk << (sh + 1)) + j, i1 = i0 + h;
            const float2 w = tws[j << (lg - 1 - sh)];
            float2* row = buf + l * SL;
            const float2 a = row[tsk(i0)], b = tcmul(row[tsk(i1)], w);
            row[tsk(i0)] = make_float2(a.x + b.x, a.y + b.y);
            row[tsk(i1)] = make_float2(a.x - b.x, a.y - b.y);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(TAIL_THREADS) batched_tail_kernel(const Reduce3Params P,
                                                                     const int64_t* __restrict__ bnd,
                                                                     const TileRec* __restrict__ rec,
                                                                     const float2* __restrict__ inv_len,
                                                                     const float* __restrict__ wtab,
                                                                     const float2* __restrict__ tw,
                                                                     float2* __restrict__ scratch,
                                                                     float2* __restrict__ out) {
    extern __shared__ float2 tsm[];
    const C3Geom& geo = P.geom;
    const SeriesView& sv = P.ser;
    const int L = geo.L, N = P.nfft, H = N / 2 + 1;
    int lg = 0;
    while ((1 << lg) < N) ++lg;
    const int SL = N + N / 16 + 1;
    float2* buf = tsm;                     // TAIL_LINES lines of SL
    float2* tws = tsm + TAIL_LINES * SL;   // N / 2 twiddles
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x) tws[k] = tw[k];
    float2* R = scratch + (int64_t)blockIdx.x * H * N;  // R[k2][k1]
    const int tsz = TILE_M * geo.tile_n;
    const int64_t total_win = sv.win[sv.S];
    const int twoL = 2 * L;
    const int RC = 2 * TAIL_LINES < twoL ? 2 * TAIL_LINES : twoL;  // lag rows per chunk (two per complex line)
    __syncthreads();
    for (int s = blockIdx.x; s < sv.S; s += gridDim.x) {
        const float2 il = inv_len[s];
        float2* Bs = out + (int64_t)s * N * N;
        // ---- A: rows of the windowed grid, row transforms
        for (int r0 = 0; r0 < twoL; r0 += RC) {
            // element (row i0 + 4q .. +3, column j) from vector vi of tile a; rows of the chunk
            // land at line (i - r0) / 2, real part for even i, imaginary for odd, slot bitrev(k2)
            const int nvec = RC / 4 * twoL;
            for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
                const int j = v / (RC / 4), q = v % (RC / 4);
                const int i0 = r0 + 4 * q, a = i0 / TILE_M, m0 = i0 % TILE_M;
                const TileRec r = rec[(int64_t)s * geo.ntiles + a];
                DF acc[4];
                if (r.nwin > 0) {
                    tile_share4<8>(P.partials, r, tsz, (j * TILE_M + m0) >> 2, 0, 1, geo.flush, bnd, total_win, acc);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[c] = df_zero();
                }
                const int w2 = j - L;
                const int k2 = w2 < 0 ? w2 + N : w2;
                const int slot = tsk((int)(__brev((unsigned)k2) >> (32 - lg)));
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int w1 = i0 + c - L;
                    const DF v3 = df_mul(acc[c], DF{il.x, il.y});
                    float wv = wtab[w1 + twoL] * wtab[w2 + twoL];
                    if (P.window == HOS_WIN_PARZEN_SYM) wv *= wtab[w1 - w2 + twoL];
                    if (P.window == HOS_WIN_RECT && (rect_excluded(w1, L) || rect_excluded(w2, L))) wv = 0.0f;
                    const float o = (v3.h + v3.l) * ((float)P.scale * wv);
                    const int row = i0 + c - r0;
                    float* line = reinterpret_cast<float*>(buf + (row >> 1) * SL + slot);
                    line[row & 1] = o;
                }
            }
            __syncthreads();
            tail_fft_lines(buf, RC / 2, N, lg, SL, tws);
            // separate the two real rows of each line: A = (Z[k] + conj Z[N-k]) / 2,
            // B = (Z[k] - conj Z[N-k]) / 2i, k = 0..N/2; rows i, i + 1 are grid rows k1 = (w1 mod N)
            for (int e = threadIdx.x; e < (RC / 2) * H; e += blockDim.x) {
                const int l = e % (RC / 2), k = e / (RC / 2);
                const float2 z = buf[l * SL + tsk(k)], zc = buf[l * SL + tsk((N - k) & (N - 1))];
                const float2 ra = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
                const float2 rb = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
                const int w1a = r0 + 2 * l - L, w1b = w1a + 1;
                const int k1a = w1a < 0 ? w1a + N : w1a, k1b = w1b < 0 ? w1b + N : w1b;
                R[(int64_t)k * N + k1a] = ra;
                R[(int64_t)k * N + k1b] = rb;
            }
            __syncthreads();
        }
        // ---- B: column transforms, blocks of TAIL_LINES columns k2
        for (int c0 = 0; c0 < H; c0 += TAIL_LINES) {
            const int nc = (H - c0) < TAIL_LINES ? (H - c0) : TAIL_LINES;
            for (int e = threadIdx.x; e < nc * N; e += blockDim.x) {
                const int l = e / N, k1 = e % N;
                buf[l * SL + tsk((int)(__brev((unsigned)k1) >> (32 - lg)))] = R[(int64_t)(c0 + l) * N + k1];
            }
            __syncthreads();
            tail_fft_lines(buf, nc, N, lg, SL, tws);
            // B(k1, k2) row by row (nc consecutive columns), and the mirror
            // B(N - k1, N - k2) = conj B(k1, k2) for 0 < k2 < N/2
            for (int e = threadIdx.x; e < N * nc; e += blockDim.x) {
                const int k1 = e / nc, l = e % nc, k2 = c0 + l;
                const float2 v = buf[l * SL + tsk(k1)];
                Bs[(int64_t)k1 * N + k2] = v;
                if (k2 > 0 && k2 < N / 2) Bs[(int64_t)((N - k1) & (N - 1)) * N + (N - k2)] = make_float2(v.x, -v.y);
            }
            __syncthreads();
        }
    }
}

bool batched_tail_supported(const C3Geom& geo, int nfft) {
    const int twoL = 2 * geo.L;
    if (nfft != twoL || twoL < 32 || twoL > 256 || (twoL & (twoL - 1)) != 0) return false;
    if (geo.tile_n < twoL || geo.ntiles != geo.tiles_m) return false;
    for (int t = 0; t < geo.ntiles; ++t)
        if (geo.tile_a[t] != t || geo.tile_c32[t] != 0 || 32 * geo.tile_w32[t] < twoL) return false;
    return true;
}

size_t batched_tail_scratch_bytes(int nfft, int ctas) {
    return (size_t)ctas * (size_t)(nfft / 2 + 1) * (size_t)nfft * sizeof(float2);
}

cudaError_t launch_batched_tail(const Reduce3Params& p, int ctas, int64_t* bnd, TileRec* rec, float2* inv_len,
                                float* wtab, const float2* tw, float2* scratch, float2* out, cudaStream_t st) {
    cudaError_t e = launch_part_index(p.geom, p.ser, bnd, rec, inv_len, p.norm_len, 3, st);
    if (e != cudaSuccess) return e;
    window_table_kernel<<<(unsigned)ceil_div(4 * p.geom.L, 256), 256, 0, st>>>(p.geom.L, p.window, wtab);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int N = p.nfft;
    const size_t smem = (size_t)(TAIL_LINES * (N + N / 16 + 1) + N / 2) * sizeof(float2);
    e = cudaFuncSetAttribute(batched_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    batched_tail_kernel<<<ctas, TAIL_THREADS, smem, st>>>(p, bnd, rec, inv_len, wtab, tw, scratch, out);
    count_launch();
    return cudaGetLastError();
}

// Window, scale and wrap of a given c3 (hos_cumulant3's layout: element
// (w2 + L) * 2L + (w1 + L)) onto the transform grid, in the arithmetic of
// emit_c3x4, so that a c3 from hos_cumulant3 gives hos_bispectrum's grid.
__global__ void window_c3_kernel(const double* __restrict__ c3, int L, int window, const float* __restrict__ wtab,
                                 int Nf, double scale, float* __restrict__ grid) {
    const int twoL = 2 * L;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= twoL * twoL) return;
    const int w1 = e % twoL - L, w2 = e / twoL - L;
    float wv = wtab[w1 + twoL] * wtab[w2 + twoL];
    if (window == HOS_WIN_PARZEN_SYM) wv *= wtab[w1 - w2 + twoL];
    if (window == HOS_WIN_RECT && (rect_excluded(w1, L) || rect_excluded(w2, L))) wv = 0.0f;
    const int k1 = w1 < 0 ? w1 + Nf : w1, k2 = w2 < 0 ? w2 + Nf : w2;
    grid[(int64_t)k2 * Nf + k1] = (float)c3[e] * ((float)scale * wv);
}

cudaError_t launch_window_c3(const double* c3, int L, int window, int Nf, double scale, float* wtab, float* grid,
                             cudaStream_t st) {
    window_table_kernel<<<(unsigned)ceil_div(4 * L, 256), 256, 0, st>>>(L, window, wtab);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    window_c3_kernel<<<(unsigned)ceil_div(4 * L * L, 256), 256, 0, st>>>(c3, L, window, wtab, Nf, scale, grid);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_zero_f32(float* p, int64_t n, cudaStream_t st) {
    int64_t b = ceil_div(n, 256);
    zero_f32_kernel<<<(unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096), 256, 0, st>>>(p, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_timeout_selftest(int* status, uint64_t limit_ns, cudaStream_t st) {
    timeout_selftest_kernel<<<1, 32, 0, st>>>(status, limit_ns);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hos
