// reduce.cu -- deterministic FP64 reduction of the contraction's FP32 partial
// tiles into c3, the 1/n time average, the average over parts (Algorithm DBS
// step 6), the lag window, and the wrap of lags onto the N-point transform
// grid (lag w -> index w mod N).
#include "launch.cuh"

namespace hos {

// bnd[g] = first work unit of CTA g, g = 0..G (the contraction's stream-K split)
__global__ void bounds_kernel(const int64_t* __restrict__ unit, int S, int G, int64_t* __restrict__ bnd) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g <= G) bnd[g] = range_begin(g, unit[S], G);
}

// Sum of one group of up to 16 consecutive main slots of (series, tile), as
// an unevaluated sum of two floats (TwoSum, about 48 significant bits).
HOS_DEV double group_sum(const float* __restrict__ p, int64_t tsz, int64_t cnt) {
    float v[16];
    if (cnt == 16) {
#pragma unroll
        for (int f = 0; f < 16; ++f) v[f] = p[f * tsz];  // independent loads in flight together
    } else {
#pragma unroll
        for (int f = 0; f < 16; ++f) v[f] = (f < cnt) ? p[f * tsz] : 0.0f;
    }
    float hi = 0.0f, lo = 0.0f;
#pragma unroll
    for (int f = 0; f < 16; ++f) {
        const float sum = hi + v[f];
        const float bv = sum - hi;
        lo += (hi - (sum - bv)) + (v[f] - bv);
        hi = sum;
    }
    return (double)hi + (double)lo;
}

constexpr int REDUCE_THREADS = 256;

// For every (series s, computed tile t): the CTAs whose unit range starts
// strictly inside the (s, t) unit range, [xr.x, xr.y).  Those CTAs' first
// parts that begin mid flush-window live in per-CTA slots.
__global__ void part_ranges_kernel(const C3Geom geo, const SeriesView sv, const int64_t* __restrict__ bnd,
                                   int2* __restrict__ xr) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)sv.S * geo.ntiles) return;
    const int s = (int)(q / geo.ntiles), t = (int)(q % geo.ntiles);
    const int64_t nch = ceil_div(sv.off[s + 1] - sv.off[s], geo.kc);
    const int64_t ub = sv.unit[s] + (int64_t)t * nch, ue = ub + nch;
    int lo = 0, hi = geo.G;  // first CTA starting after ub
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (bnd[mid] > ub) hi = mid; else lo = mid + 1;
    }
    int e = lo;
    while (e < geo.G && bnd[e] < ue) ++e;
    xr[q] = make_int2(lo, e);
}

// Sum over the parts of (series s, computed tile t) at element `el`, divided
// by the series length: the main parts (one per flush window, contiguous
// slots in chunk order) in groups of 16 as two-float sums, the groups added
// in FP64 in order, then the parts that start at a CTA boundary inside a
// window, in CTA order.
HOS_DEV double tile_part_sum(const C3Geom& geo, const SeriesView& sv, const float* __restrict__ partials, int s, int t,
                             int64_t el, const int64_t* __restrict__ bnd, const int2* __restrict__ xr) {
    const int F = geo.flush;
    const int64_t tsz = (int64_t)TILE_M * geo.tile_n;
    const int64_t total_win = sv.win[sv.S];
    const int64_t len = sv.off[s + 1] - sv.off[s];
    const int64_t nch = ceil_div(len, geo.kc), nwin = ceil_div(nch, F);
    const int64_t ub = sv.unit[s] + (int64_t)t * nch;
    const float* p = partials + (sv.win[s] + (int64_t)t * nwin) * tsz + el;
    double acc = 0.0;
    for (int64_t f0 = 0; f0 < nwin; f0 += 16) acc += group_sum(p + f0 * tsz, tsz, (nwin - f0 < 16) ? nwin - f0 : 16);
    const int2 r = xr[(int64_t)s * geo.ntiles + t];
    for (int g = r.x; g < r.y; ++g)
        if ((int)(bnd[g] - ub) % F != 0 && bnd[g] < bnd[g + 1]) acc += (double)partials[(total_win + g) * tsz + el];
    return acc / (double)len;
}

// One block = 256 consecutive elements (elem = j * 128 + m) of computed tile
// blockIdx.y, output group blockIdx.z.  For each series of the group, thread
// 0 lists the parts of (series, tile) that start at a CTA boundary inside a
// flush window; then every thread sums its element: the main parts (one per
// flush window, contiguous slots in chunk order) in groups of 16 as two-float
// sums added in FP64 in order, then the listed parts in CTA order, and
// divides by the series length.  Parts average over the group's series.
// The value goes to lag (w1, w2) and, when the tile holding (w2, w1) is not
// computed, to that mirrored lag as well (c3(w1,w2) = c3(w2,w1)).
__global__ void __launch_bounds__(REDUCE_THREADS, 3) reduce3_kernel(const Reduce3Params P,
                                                                    const int64_t* __restrict__ bnd,
                                                                    const int2* __restrict__ xr) {
    const C3Geom& geo = P.geom;
    const SeriesView& sv = P.ser;
    const int L = geo.L, N = geo.tile_n;
    const int t = blockIdx.y, grp = blockIdx.z;
    const int64_t tsz = (int64_t)TILE_M * N;
    const int64_t elem = (int64_t)blockIdx.x * REDUCE_THREADS + threadIdx.x;
    const int m = (int)(elem % TILE_M), j = (int)(elem / TILE_M);
    const int w1 = -L + TILE_M * geo.tile_a[t] + m, w2 = -L + N * geo.tile_b[t] + j;
    const bool live = elem < tsz && w1 < L && w2 < L;
    const int64_t el = elem < tsz ? elem : 0;
    const int s0 = P.per_series_groups ? grp : 0, s1 = P.per_series_groups ? grp + 1 : sv.S;
    double c3 = 0.0;
    int k = 0;
    for (int s = s0; s < s1; ++s) {
        if (sv.off[s + 1] <= sv.off[s]) continue;
        c3 += tile_part_sum(geo, sv, P.partials, s, t, el, bnd, xr);
        ++k;
    }
    if (!P.per_series_groups && k > 0) c3 /= (double)k;
    if (!live) return;
    const int twoL = 2 * L;
    const int ma = (w2 + L) / TILE_M, mb = (w1 + L) / N;
    const bool write_mirror = geo.tile_idx[ma][mb] < 0;
    if (P.mode == 1) {
        double* o = P.c3out + (int64_t)grp * twoL * twoL;
        o[(int64_t)(w2 + L) * twoL + (w1 + L)] = c3;
        if (write_mirror) o[(int64_t)(w1 + L) * twoL + (w2 + L)] = c3;
        return;
    }
    const double wv = (P.window == HOS_WIN_RECT && (rect_excluded(w1, L) || rect_excluded(w2, L)))
                          ? 0.0
                          : lag_window2(w1, w2, L, P.window);
    const int Nf = P.nfft;
    const int k1 = (w1 % Nf + Nf) % Nf, k2 = (w2 % Nf + Nf) % Nf;
    float* gr = P.grid + (int64_t)grp * Nf * Nf;
    const float v = (float)(P.scale * wv * c3);
    gr[(int64_t)k2 * Nf + k1] = v;
    if (write_mirror) gr[(int64_t)k1 * Nf + k2] = v;
}

// Fourth order, tensor-core partials: m4buf[s][t][elem] = sum of the parts of
// (part s, pair tile t) / length, FP64 (elem = (w3 + L) * 128 + pair in tile).
__global__ void __launch_bounds__(REDUCE_THREADS, 3) m4_tile_reduce_kernel(const C3Geom geo, const SeriesView sv,
                                                                           const float* __restrict__ partials,
                                                                           const int64_t* __restrict__ bnd,
                                                                           const int2* __restrict__ xr,
                                                                           double* __restrict__ m4buf) {
    const int t = blockIdx.y, s = blockIdx.z;
    const int64_t tsz = (int64_t)TILE_M * geo.tile_n;
    const int64_t elem = (int64_t)blockIdx.x * REDUCE_THREADS + threadIdx.x;
    const int64_t el = elem < tsz ? elem : 0;
    double v = 0.0;
    if (sv.off[s + 1] > sv.off[s]) v = tile_part_sum(geo, sv, partials, s, t, el, bnd, xr);
    if (elem < tsz) m4buf[((int64_t)s * geo.ntiles + t) * tsz + elem] = v;
}

static cudaError_t launch_part_index(const C3Geom& geo, const SeriesView& sv, int64_t* bnd, int2* xr,
                                     cudaStream_t st) {
    bounds_kernel<<<(unsigned)ceil_div(geo.G + 1, 256), 256, 0, st>>>(sv.unit, sv.S, geo.G, bnd);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    part_ranges_kernel<<<(unsigned)ceil_div((int64_t)sv.S * geo.ntiles, 256), 256, 0, st>>>(geo, sv, bnd, xr);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_m4_tile_reduce(const C3Geom& geo, const SeriesView& sv, const float* partials, int64_t* bnd,
                                  int2* xr, double* m4buf, cudaStream_t st) {
    cudaError_t e = launch_part_index(geo, sv, bnd, xr, st);
    if (e != cudaSuccess) return e;
    const int64_t tsz = (int64_t)TILE_M * geo.tile_n;
    dim3 grid((unsigned)ceil_div(tsz, REDUCE_THREADS), (unsigned)geo.ntiles, (unsigned)sv.S);
    m4_tile_reduce_kernel<<<grid, REDUCE_THREADS, 0, st>>>(geo, sv, partials, bnd, xr, m4buf);
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

cudaError_t launch_reduce3(const Reduce3Params& p, int groups, int64_t* bnd, int2* xr, cudaStream_t st) {
    cudaError_t e = launch_part_index(p.geom, p.ser, bnd, xr, st);
    if (e != cudaSuccess) return e;
    const int64_t tsz = (int64_t)TILE_M * p.geom.tile_n;
    dim3 grid((unsigned)ceil_div(tsz, REDUCE_THREADS), (unsigned)p.geom.ntiles, (unsigned)groups);
    reduce3_kernel<<<grid, REDUCE_THREADS, 0, st>>>(p, bnd, xr);
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
