// reduce.cu -- deterministic FP64 reduction of the contraction's FP32 partial
// tiles into c3, the 1/n time average, the average over parts (Algorithm DBS
// step 6), the lag window, and the wrap of lags onto the N-point transform
// grid (lag w -> index w mod N).
#include "launch.cuh"

namespace hos {

// c3 of series s at the element `elem` of computed tile t: the parts of this
// (series, tile) are summed in a fixed order -- first the parts that start at
// a flush-window boundary (their slots are contiguous, in chunk order), in
// groups of 16 accumulated as an unevaluated sum of two floats (TwoSum,
// about 48 significant bits) and each group added in FP64; then, in CTA
// order, the parts that start at a CTA boundary inside a window -- and
// divided by the series length.
HOS_DEV double series_c3(const C3Geom& geo, const SeriesView& sv, const float* __restrict__ part, int s, int t,
                         int64_t elem) {
    const int64_t len = sv.off[s + 1] - sv.off[s];
    if (len <= 0) return 0.0;
    const int64_t nch = ceil_div(len, KC);
    const int64_t F = geo.flush, nwin = ceil_div(nch, F);
    const int64_t U = sv.unit[sv.S], total_win = sv.win[sv.S];
    const int64_t G = geo.G;
    const int64_t tsz = (int64_t)TILE_M * geo.tile_n;
    const float* p = part + (sv.win[s] + (int64_t)t * nwin) * tsz + elem;
    double acc = 0.0;
    for (int64_t f0 = 0; f0 < nwin; f0 += 16) {
        const int64_t f1 = (f0 + 16 < nwin) ? f0 + 16 : nwin;
        float hi = 0.0f, lo = 0.0f;
        for (int64_t f = f0; f < f1; ++f) {
            const float v = p[f * tsz];
            const float sum = hi + v;
            const float bv = sum - hi;
            lo += (hi - (sum - bv)) + (v - bv);
            hi = sum;
        }
        acc += (double)hi + (double)lo;
    }
    const int64_t ub = sv.unit[s] + (int64_t)t * nch, ue = ub + nch;
    for (int64_t g = ((ub + 1) * G + U - 1) / U; g < G; ++g) {
        const int64_t b0 = range_begin(g, U, G);
        if (b0 >= ue) break;
        if ((b0 - ub) % F != 0 && b0 < range_begin(g + 1, U, G)) acc += (double)part[(total_win + g) * tsz + elem];
    }
    return acc / (double)len;
}

HOS_DEV void locate(const C3Geom& geo, int w1, int w2, int& t, int64_t& elem) {
    const int L = geo.L, N = geo.tile_n;
    int a = (w1 + L) / TILE_M, b = (w2 + L) / N;
    t = geo.tile_idx[a][b];
    if (t < 0) {
        const int x = w1;
        w1 = w2;
        w2 = x;
        a = (w1 + L) / TILE_M;
        b = (w2 + L) / N;
        t = geo.tile_idx[a][b];
    }
    elem = (int64_t)(w2 + L - b * N) * TILE_M + (w1 + L - a * TILE_M);
}


__global__ void reduce3_kernel(const Reduce3Params P) {
    const C3Geom& geo = P.geom;
    const int L = geo.L, twoL = 2 * L;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)twoL * twoL) return;
    const int w1 = (int)(e % twoL) - L, w2 = (int)(e / twoL) - L;
    const int grp = blockIdx.y;
    int t;
    int64_t elem;
    locate(geo, w1, w2, t, elem);
    double c3;
    if (P.per_series_groups) {
        c3 = series_c3(geo, P.ser, P.partials, grp, t, elem);
    } else {
        c3 = 0.0;
        int k = 0;
        for (int s = 0; s < P.ser.S; ++s) {
            if (P.ser.off[s + 1] > P.ser.off[s]) {
                c3 += series_c3(geo, P.ser, P.partials, s, t, elem);
                ++k;
            }
        }
        if (k > 0) c3 /= (double)k;
    }
    if (P.mode == 1) {
        P.c3out[(int64_t)grp * twoL * twoL + (int64_t)(w2 + L) * twoL + (w1 + L)] = c3;
        return;
    }
    double wv = (P.window == HOS_WIN_RECT && (rect_excluded(w1, L) || rect_excluded(w2, L)))
                    ? 0.0
                    : lag_window2(w1, w2, L, P.window);
    const int Nf = P.nfft;
    const int k1 = (w1 % Nf + Nf) % Nf, k2 = (w2 % Nf + Nf) % Nf;
    P.grid[(int64_t)grp * Nf * Nf + (int64_t)k2 * Nf + k1] = (float)(P.scale * wv * c3);
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

cudaError_t launch_reduce3(const Reduce3Params& p, int groups, cudaStream_t st) {
    const int64_t n = 4LL * p.geom.L * p.geom.L;
    dim3 grid((unsigned)ceil_div(n, 256), (unsigned)groups);
    reduce3_kernel<<<grid, 256, 0, st>>>(p);
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
