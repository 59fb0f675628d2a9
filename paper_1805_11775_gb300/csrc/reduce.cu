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
// Six-fold plans: the four reduced values go back, as FP32, over the same
// elements of the result slot (res_slot: the first window slot of the group's
// first part; -1 for an empty series, which the unfold writes as zero).  The
// thread that writes an element is the only one that reads it.
HOS_DEV void keep_c3x4(const Reduce3Params& P, int64_t res_slot, int elem0, const DF (&v)[4]) {
    if (res_slot < 0) return;
#ifdef HOS_DEBUG_BOUNDS
    if (res_slot >= P.n_slots) {
        record_status(P.status, HOS_ERR_DEVICE_FAULT);
        return;
    }
#endif
    float4* d = reinterpret_cast<float4*>(P.tiles_out + res_slot * (int64_t)(TILE_M * P.geom.tile_n) + elem0);
    *d = make_float4(v[0].h + v[0].l, v[1].h + v[1].l, v[2].h + v[2].l, v[3].h + v[3].l);
}

HOS_DEV void emit_c3x4(const Reduce3Params& P, const float* __restrict__ wtab, int grp, int t, int elem0,
                       const DF (&v)[4], int64_t res_slot) {
    const C3Geom& geo = P.geom;
    const int L = geo.L;
    if (geo.sym != C3_SWAP) {
        keep_c3x4(P, res_slot, elem0, v);
        return;
    }
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
                emit_c3x4(P, wtab, grp, t, 4 * vi[k], v, r.slot);
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
#ifdef HOS_DEBUG_BOUNDS
        if (r.slot < 0 || r.slot + r.nwin > P.n_slots - geo.G || r.xlo < 0 || r.xhi > geo.G) {
            if (threadIdx.x == 0) record_status(P.status, HOS_ERR_DEVICE_FAULT);
            return;
        }
#endif
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
    // six-fold plans keep the result over the first window slot of the group's first part
    const TileRec r0 = rec[(int64_t)s0 * geo.ntiles + t];
    const int64_t res_slot = r0.nwin > 0 ? r0.slot : -1;
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
        emit_c3x4(P, wtab, grp, t, 4 * vi[k], c3[k], res_slot);
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
#ifdef HOS_DEBUG_BOUNDS
    if (r.slot < 0 || r.slot >= P.n_slots) {
        if (threadIdx.x == 0) record_status(P.status, HOS_ERR_DEVICE_FAULT);
        return;
    }
#endif
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
        emit_c3x4(P, wtab, grp, t, 4 * vi[k], v, r.slot);
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

// Six-fold plans: every entry of each group's transform grid from the
// reduced fundamental set.  The lag pair's image in the set (the sector of
// (w1, w2) fixes which of the six it is), its tile and element, windowed and
// scaled; entries past the lags (Nf > 2L) and the zero-weight lag -L get 0,
// as do an empty series' and, under the band, the zero-weight orbits.
// Writes are coalesced; the reads gather from the group's reduced tiles.
// One block per grid row (lag w2) of one group; threads along the row.
__global__ void __launch_bounds__(256) unfold_c3_kernel(const Reduce3Params P, const TileRec* __restrict__ rec,
                                                        const float* __restrict__ wtab) {
    const C3Geom& geo = P.geom;
    const int L = geo.L, twoL = 2 * L, Nf = P.nfft;
    const int k2 = blockIdx.x, grp = blockIdx.y;
    __shared__ int64_t slot_s[MAX_TILES];  // result slot of each tile (-1: empty series)
    for (int t = threadIdx.x; t < geo.ntiles; t += blockDim.x) {
        const TileRec rr = rec[(int64_t)(P.per_series_groups ? grp : 0) * geo.ntiles + t];
        slot_s[t] = rr.nwin > 0 ? rr.slot : -1;
    }
    __syncthreads();
    float* row = P.grid + ((int64_t)grp * Nf + k2) * Nf;
    // lag of an index: k < L -> k, k > Nf - L -> k - Nf; w = -L (zero weight) and
    // the indices between (Nf > 2L) hold no lag
    const bool in2 = k2 < L || k2 > Nf - L;
    const int w2 = k2 < L ? k2 : k2 - Nf;
    const float sw2 = in2 ? (float)P.scale * wtab[w2 + twoL] : 0.0f;
    const size_t tsz = (size_t)TILE_M * geo.tile_n;
    for (int k1 = threadIdx.x; k1 < Nf; k1 += blockDim.x) {
        float out = 0.0f;
        if (in2 && (k1 < L || k1 > Nf - L)) {
            const int w1 = k1 < L ? k1 : k1 - Nf;
            int b, a;  // the image (b, a) with 0 <= b <= a
            c3_sector_image(w1, w2, b, a);
            if (c3_fundamental(L, geo.sym, b, a)) {
                const int r = b + L, blk = r >> 7, c = a + L;
                const int t = geo.row_t0[blk] + (c - geo.row_c0[blk]) / geo.tile_n;
                const int64_t sl = slot_s[t];
                if (sl >= 0) {
                    const float v = P.tiles_out[(size_t)sl * tsz + (size_t)(c - 32 * geo.tile_c32[t]) * TILE_M +
                                                (r & (TILE_M - 1))];
                    float wv = wtab[w1 + twoL] * sw2;
                    if (P.window == HOS_WIN_PARZEN_SYM) wv *= wtab[w1 - w2 + twoL];
                    out = v * wv;
                }
            }
        }
        row[k1] = out;
    }
}

// The same unfold with one block per group, its reduced tiles staged in
// shared memory first (coalesced 16-byte loads; rows at a pitch of 129 words,
// so that a grid row's gathers from there fall on different banks in every
// sector), for plans whose tiles fit: the many short series of a batch.
constexpr int UNFOLD_PITCH = TILE_M + 1;
__global__ void __launch_bounds__(1024) unfold_c3_smem_kernel(const Reduce3Params P, const TileRec* __restrict__ rec,
                                                              const float* __restrict__ wtab) {
    extern __shared__ float tl[];  // [tile][column][row], row pitch UNFOLD_PITCH
    const C3Geom& geo = P.geom;
    const int L = geo.L, twoL = 2 * L, Nf = P.nfft, N = geo.tile_n;
    const int grp = blockIdx.x;
    const size_t tsz = (size_t)TILE_M * N;
    bool empty = false;
    for (int t = 0; t < geo.ntiles; ++t) {
        const TileRec rr = rec[(int64_t)(P.per_series_groups ? grp : 0) * geo.ntiles + t];
        if (rr.nwin <= 0) {
            empty = true;  // an empty series: every tile's record says so
            break;
        }
        const float4* src = reinterpret_cast<const float4*>(P.tiles_out + (size_t)rr.slot * tsz);
        float* dst = tl + (size_t)t * N * UNFOLD_PITCH;
        for (int q = threadIdx.x; q < (int)(tsz / 4); q += blockDim.x) {
            const float4 v = src[q];
            const int col = (4 * q) / TILE_M, row = (4 * q) % TILE_M;
            float* d = dst + col * UNFOLD_PITCH + row;
            d[0] = v.x;
            d[1] = v.y;
            d[2] = v.z;
            d[3] = v.w;
        }
    }
    float* wt = tl + (size_t)geo.ntiles * N * UNFOLD_PITCH;  // the window table, 4L values
    for (int i = threadIdx.x; i < 4 * L; i += blockDim.x) wt[i] = wtab[i];
    __syncthreads();
    float* out_g = P.grid + (int64_t)grp * Nf * Nf;
    const float sc = (float)P.scale;
    // a warp per grid row (lag w2), lanes along it
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k2 = threadIdx.x >> 5; k2 < Nf; k2 += nw) {
        const bool in2 = !empty && (k2 < L || k2 > Nf - L);
        const int w2 = k2 < L ? k2 : k2 - Nf;
        const float sw2 = in2 ? sc * wt[w2 + twoL] : 0.0f;
        float* orow = out_g + (size_t)k2 * Nf;
        for (int k1 = lane; k1 < Nf; k1 += 32) {
            float out = 0.0f;
            if (in2 && (k1 < L || k1 > Nf - L)) {
                const int w1 = k1 < L ? k1 : k1 - Nf;
                int b, a;  // the image (b, a) with 0 <= b <= a
                c3_sector_image(w1, w2, b, a);
                if (c3_fundamental(L, geo.sym, b, a)) {
                    const int r = b + L, blk = r >> 7, c = a + L;
                    const int t = geo.row_t0[blk] + (c - geo.row_c0[blk]) / N;
                    const float v =
                        tl[((size_t)t * N + (c - 32 * geo.tile_c32[t])) * UNFOLD_PITCH + (r & (TILE_M - 1))];
                    float wv = wt[w1 + twoL] * sw2;
                    if (P.window == HOS_WIN_PARZEN_SYM) wv *= wt[w1 - w2 + twoL];
                    out = v * wv;
                }
            }
            orow[k1] = out;
        }
    }
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
    e = cudaGetLastError();
    if (e != cudaSuccess || p.geom.sym == C3_SWAP || p.mode != 0) return e;
    const size_t smem = ((size_t)p.geom.ntiles * p.geom.tile_n * UNFOLD_PITCH + 4 * (size_t)p.geom.L) * sizeof(float);
    // the staged form takes one block (one SM) per group: for many groups only
    if (smem <= 200 * 1024 && groups >= 256) {
        e = cudaFuncSetAttribute(unfold_c3_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        unfold_c3_smem_kernel<<<(unsigned)groups, 1024, smem, st>>>(p, rec, wtab);
    } else {
        unfold_c3_kernel<<<dim3((unsigned)p.nfft, (unsigned)groups), 256, 0, st>>>(p, rec, wtab);
    }
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
