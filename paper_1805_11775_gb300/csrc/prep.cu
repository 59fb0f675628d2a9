// prep.cu -- series layout planning and mean removal (Algorithm DBS steps 1-2).
//
// plan_series_kernel : per-series offsets, zero-padded block starts, work-unit
//                      and flush-window prefix sums (one block, scan).
// mean_partial_kernel / mean_final_kernel : FP64 per-series mean, two-level
//                      tree, fixed order (deterministic).
// planes_kernel      : y = x - mean into the padded sample planes: FP32 y, and
//                      its hi/lo split (bf16 pair, or tf32-rounded FP32 pair).
#include "launch.cuh"

namespace hos {

// Block-wide exclusive scan of int64 over blockDim.x <= 1024 values.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int d = 1; d < blockDim.x; d <<= 1) {
        int64_t a = (t >= d) ? sh[t - d] : 0;
        __syncthreads();
        sh[t] += a;
        __syncthreads();
    }
    int64_t incl = sh[t];
    *total = sh[blockDim.x - 1];
    __syncthreads();
    return incl - v;
}

// mode 0: single series of n samples cut into parts of seg (seg <= 0: one part)
// mode 1: S series given by device offsets d_user_off[S+1]
__global__ void plan_series_kernel(int mode, int64_t n, int64_t seg, const int64_t* __restrict__ d_user_off, int S,
                                   int L, int ntiles, int ktot, int flush, int kc, int pad_tail, int64_t* off,
                                   int64_t* pad, int64_t* unit, int64_t* win) {
    __shared__ int64_t sh[1024];
    __shared__ int64_t carry[3];
    if (threadIdx.x == 0) carry[0] = carry[1] = carry[2] = 0;
    __syncthreads();
    for (int base = 0; base < S; base += blockDim.x) {
        const int s = base + threadIdx.x;
        int64_t o0 = 0, o1 = 0;
        if (s < S) {
            if (mode == 0) {
                o0 = (seg > 0) ? (int64_t)s * seg : 0;
                o1 = (seg > 0) ? ((int64_t)(s + 1) * seg < n ? (int64_t)(s + 1) * seg : n) : n;
            } else {
                o0 = d_user_off[s];
                o1 = d_user_off[s + 1];
            }
        }
        const int64_t len = (s < S && o1 > o0) ? (o1 - o0) : 0;
        const SeriesPlan sp = series_plan(len, L, ntiles, ktot, flush, kc, pad_tail);
        const int64_t plen = (s < S) ? sp.plen : 0;
        const int64_t nu = sp.cost;  // cost of the series' units
        const int64_t nw = sp.wins;
        int64_t tot;
        const int64_t ep = block_exclusive_scan(plen, sh, &tot);
        const int64_t c0 = carry[0];
        __syncthreads();
        if (s < S) pad[s] = c0 + ep;
        if (threadIdx.x == 0) carry[0] = c0 + tot;
        __syncthreads();
        const int64_t eu = block_exclusive_scan(nu, sh, &tot);
        const int64_t c1 = carry[1];
        __syncthreads();
        if (s < S) unit[s] = c1 + eu;
        if (threadIdx.x == 0) carry[1] = c1 + tot;
        __syncthreads();
        const int64_t ew = block_exclusive_scan(nw, sh, &tot);
        const int64_t c2 = carry[2];
        __syncthreads();
        if (s < S) {
            win[s] = c2 + ew;
            off[s] = o0;
        }
        if (threadIdx.x == 0) carry[2] = c2 + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pad[S] = carry[0];
        unit[S] = carry[1];
        win[S] = carry[2];
        off[S] = (mode == 0) ? n : d_user_off[S];
    }
}

// Partial sums of each series: blockIdx.y = series, blockIdx.x = slice.
template <typename T>
__global__ void mean_partial_kernel(const T* __restrict__ x, const int64_t* __restrict__ off, int nslices,
                                    double* __restrict__ part) {
    __shared__ double sh[256];
    const int s = blockIdx.y;
    const int64_t o0 = off[s], len = off[s + 1] - o0;
    const int64_t per = ceil_div(len, nslices);
    const int64_t b0 = (int64_t)blockIdx.x * per;
    const int64_t b1 = b0 + per < len ? b0 + per : len;
    // four independent accumulators keep four loads in flight per thread
    const int64_t bd = blockDim.x;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t i = b0 + threadIdx.x;
    for (; i + 3 * bd < b1; i += 4 * bd) {
        a0 += (double)x[o0 + i];
        a1 += (double)x[o0 + i + bd];
        a2 += (double)x[o0 + i + 2 * bd];
        a3 += (double)x[o0 + i + 3 * bd];
    }
    for (; i < b1; i += bd) a0 += (double)x[o0 + i];
    sh[threadIdx.x] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)s * nslices + blockIdx.x] = sh[0];
}

// One warp per series: lanes take slices k = lane, lane + 32, ..., then a
// fixed shuffle tree (deterministic).
__global__ void mean_final_kernel(const double* __restrict__ part, const int64_t* __restrict__ off, int S,
                                  int nslices, int remove_mean, double* __restrict__ mean) {
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= S) return;  // uniform per warp
    double acc = 0.0;
    for (int k = lane; k < nslices; k += 32) acc += part[(int64_t)s * nslices + k];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if (lane == 0) {
        const int64_t len = off[s + 1] - off[s];
        if (remove_mean < 0) mean[s] = acc;  // the plain sum (hos_series_sum)
        else mean[s] = (remove_mean && len > 0) ? acc / (double)len : 0.0;
    }
}

// Mean of a time slice of a longer series: the whole series' FP64 sum over
// its length (or 0 without mean removal).
__global__ void slice_mean_kernel(const double* __restrict__ sum, int64_t n_total, int remove_mean,
                                  double* __restrict__ mean) {
    if (threadIdx.x == 0) mean[0] = (remove_mean && n_total > 0) ? sum[0] / (double)n_total : 0.0;
}

// y = x - mean into the padded planes.  blockIdx.y = series; the block's
// x-slices stride over that series' padded block [pad[s], pad[s+1]).
// split: 0 = none (f32 plane only), 1 = bf16 hi/lo, 2 = tf32 hi/lo (as f32),
// 3 = f16 hi/lo of the series scaled by scale[s] (a power of two: exact).
// A time slice of a longer series also carries ext_lo samples before and
// ext_hi after it (its neighbours' halo, x[o0 - ext_lo ..]); they go into the
// zero padding on either side (ext_lo, ext_hi <= L).
template <typename T>
__global__ void planes_kernel(const T* __restrict__ x, const int64_t* __restrict__ off,
                              const int64_t* __restrict__ pad, const double* __restrict__ mean, int L, int split,
                              int64_t ext_lo, int64_t ext_hi, float* __restrict__ y32, void* __restrict__ hi,
                              void* __restrict__ lo, const float* __restrict__ scale) {
    const int s = blockIdx.y;
    const int64_t p0 = pad[s], p1 = pad[s + 1];
    const int64_t o0 = off[s], len = off[s + 1] - o0;
    const double mu = mean[s];
    if (split == 1 || split == 3) {
        const float sc = (split == 3) ? scale[s] : 1.0f;
        // four samples per thread: one 16-byte y store and 8-byte hi and lo
        // stores (p0 and p1 are multiples of 64)
        for (int64_t p = p0 + 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); p < p1;
             p += 4 * (int64_t)gridDim.x * blockDim.x) {
            float v[4];
            uint32_t hv[2], lv[2];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t i = p + c - p0 - L;
                v[c] = (i >= -ext_lo && i < len + ext_hi) ? (float)((double)x[o0 + i] - mu) : 0.0f;
            }
#pragma unroll
            for (int c = 0; c < 4; c += 2) {
                if (split == 1) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[c]), h1 = __float2bfloat16_rn(v[c + 1]);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[c] - __bfloat162float(h0));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[c + 1] - __bfloat162float(h1));
                    hv[c / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    lv[c / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                } else {
                    const float a = v[c] * sc, b = v[c + 1] * sc;
                    hv[c / 2] = pack_f16x2(a, b);
                    const float2 f = unpack2<FMT_F16>(hv[c / 2]);
                    lv[c / 2] = pack_f16x2(a - f.x, b - f.y);
                }
            }
            *reinterpret_cast<float4*>(y32 + p) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<uint2*>(reinterpret_cast<uint16_t*>(hi) + p) = make_uint2(hv[0], hv[1]);
            *reinterpret_cast<uint2*>(reinterpret_cast<uint16_t*>(lo) + p) = make_uint2(lv[0], lv[1]);
        }
        return;
    }
    for (int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < p1;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = p - p0 - L;
        float v = 0.0f;
        if (i >= -ext_lo && i < len + ext_hi) v = (float)((double)x[o0 + i] - mu);
        y32[p] = v;
        if (split == 1) {
            __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(hi);
            __nv_bfloat16* l = reinterpret_cast<__nv_bfloat16*>(lo);
            const __nv_bfloat16 hb = __float2bfloat16_rn(v);
            h[p] = hb;
            l[p] = __float2bfloat16_rn(v - __bfloat162float(hb));
        } else if (split == 2) {
            const uint32_t hb = to_tf32(v);
            reinterpret_cast<uint32_t*>(hi)[p] = hb;
            reinterpret_cast<uint32_t*>(lo)[p] = to_tf32(v - __uint_as_float(hb));
        }
    }
}

// Power-of-two scale of each series' FP16 planes.  Pass 1: the largest
// |x - mean| over the series (and a time slice's halos), per slice of
// samples, as the bit pattern of a non-negative float (whose integer order is
// the float order: atomicMax finds the maximum exactly, in any order).  Pass 2:
// scale = 2^(top - e) with 2^e the least power of two at or above the maximum,
// so that every |scale y| <= 2^top; 1 for a series of zeros.
template <typename T>
__global__ void absmax_kernel(const T* __restrict__ x, const int64_t* __restrict__ off,
                              const double* __restrict__ mean, int64_t ext_lo, int64_t ext_hi, int nslices,
                              unsigned* __restrict__ mx) {
    __shared__ float sh[256];
    const int s = blockIdx.y;
    const int64_t o0 = off[s] - ext_lo, len = off[s + 1] - off[s] + ext_lo + ext_hi;
    const int64_t per = ceil_div(len, nslices);
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = b0 + per < len ? b0 + per : len;
    const double mu = mean[s];
    float m = 0.0f;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) m = fmaxf(m, fabsf((float)((double)x[o0 + i] - mu)));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + d]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(mx + s, __float_as_uint(sh[0]));
}

__global__ void scale_kernel(const unsigned* __restrict__ mx, int S, int top, float* __restrict__ scale) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const float m = __uint_as_float(mx[s]);
    int e = 0;
    if (m > 0.0f) {
        frexpf(m, &e);                      // m = f 2^e, 0.5 <= f < 1: m < 2^e
        if (ldexpf(1.0f, e - 1) == m) --e;  // m a power of two: 2^e = m
    }
    scale[s] = (m > 0.0f) ? ldexpf(1.0f, top - e) : 1.0f;
}

cudaError_t launch_series_scale(const void* x, int dtype, const int64_t* off, const double* mean, int S,
                                int nslices, int64_t ext_lo, int64_t ext_hi, int top, unsigned* mx, float* scale,
                                cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned) * (size_t)S, st);
    if (e != cudaSuccess) return e;
    dim3 g((unsigned)nslices, (unsigned)S);
    if (dtype == HOS_F64)
        absmax_kernel<double><<<g, 256, 0, st>>>((const double*)x, off, mean, ext_lo, ext_hi, nslices, mx);
    else
        absmax_kernel<float><<<g, 256, 0, st>>>((const float*)x, off, mean, ext_lo, ext_hi, nslices, mx);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scale_kernel<<<(unsigned)ceil_div(S, 256), 256, 0, st>>>(mx, S, top, scale);
    count_launch();
    return cudaGetLastError();
}

// The same power-of-two scale for one flat array (the adjoint's Gs).
__global__ void flat_absmax_kernel(const float* __restrict__ v, int64_t count, unsigned* __restrict__ mx) {
    __shared__ float sh[256];
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(v[i]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + d]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(mx, __float_as_uint(sh[0]));
}

cudaError_t launch_flat_scale(const float* v, int64_t count, int top, unsigned* mx, float* scale, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    int64_t b = ceil_div(count, 256);
    flat_absmax_kernel<<<(unsigned)(b < 1024 ? (b > 0 ? b : 1) : 1024), 256, 0, st>>>(v, count, mx);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scale_kernel<<<1, 32, 0, st>>>(mx, 1, top, scale);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_plan_series(int mode, int64_t n, int64_t seg, const int64_t* d_user_off, int S, int L, int ntiles,
                               int ktot, int flush, int kc, int pad_tail, int64_t* off, int64_t* pad, int64_t* unit,
                               int64_t* win, cudaStream_t st) {
    int threads = 32;  // one block; its scans take log2(threads) steps
    while (threads < S && threads < 1024) threads <<= 1;
    plan_series_kernel<<<1, threads, 0, st>>>(mode, n, seg, d_user_off, S, L, ntiles, ktot, flush, kc, pad_tail, off,
                                              pad, unit, win);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mean(const void* x, int dtype, const int64_t* off, int S, int nslices, double* part,
                        int remove_mean, double* mean, cudaStream_t st) {
    dim3 g1((unsigned)nslices, (unsigned)S);
    if (dtype == HOS_F64) mean_partial_kernel<double><<<g1, 256, 0, st>>>((const double*)x, off, nslices, part);
    else mean_partial_kernel<float><<<g1, 256, 0, st>>>((const float*)x, off, nslices, part);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mean_final_kernel<<<(unsigned)ceil_div(S, 8), 256, 0, st>>>(part, off, S, nslices, remove_mean, mean);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_planes(const void* x, int dtype, const int64_t* off, const int64_t* pad, const double* mean, int L,
                          int split, float* y32, void* hi, void* lo, int S, int blocks_x, cudaStream_t st,
                          int64_t ext_lo, int64_t ext_hi, const float* scale) {
    dim3 g((unsigned)blocks_x, (unsigned)S);
    if (dtype == HOS_F64)
        planes_kernel<double><<<g, 256, 0, st>>>((const double*)x, off, pad, mean, L, split, ext_lo, ext_hi, y32, hi,
                                                 lo, scale);
    else
        planes_kernel<float><<<g, 256, 0, st>>>((const float*)x, off, pad, mean, L, split, ext_lo, ext_hi, y32, hi,
                                                lo, scale);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_slice_mean(const double* sum, int64_t n_total, int remove_mean, double* mean, cudaStream_t st) {
    slice_mean_kernel<<<1, 32, 0, st>>>(sum, n_total, remove_mean, mean);
    count_launch();
    return cudaGetLastError();
}

// off = {0, n}: the one-series view hos_series_sum reduces over
__global__ void series_range_kernel(int64_t n, int64_t* off) {
    if (threadIdx.x == 0) {
        off[0] = 0;
        off[1] = n;
    }
}

cudaError_t launch_series_sum(const void* x, int dtype, int64_t n, int nslices, int64_t* off, double* part,
                              double* sum, cudaStream_t st) {
    series_range_kernel<<<1, 32, 0, st>>>(n, off);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_mean(x, dtype, off, 1, nslices, part, -1, sum, st);
}

// Overlapping parts written out one after another: out[k m + i] = x[k step + i],
// k < K, i < m (element type T: the caller's float or double).
template <typename T>
__global__ void gather_parts_kernel(const T* __restrict__ x, int64_t K, int64_t m, int64_t step, T* __restrict__ out) {
    const int64_t tot = K * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / m, i = e - k * m;
        out[e] = x[k * step + i];
    }
}

cudaError_t launch_gather_parts(const void* x, int dtype, int64_t K, int64_t m, int64_t step, void* out,
                                cudaStream_t st) {
    int64_t blocks = ceil_div(K * m, 256);
    if (blocks > 16 * 152) blocks = 16 * 152;
    if (dtype == HOS_F64)
        gather_parts_kernel<double><<<(unsigned)blocks, 256, 0, st>>>((const double*)x, K, m, step, (double*)out);
    else
        gather_parts_kernel<float><<<(unsigned)blocks, 256, 0, st>>>((const float*)x, K, m, step, (float*)out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hos
