// adjoint.cu -- gradient of a real loss l through the bispectrum (one part).
//
// With G = dl/dRe B + i dl/dIm B on the N x N grid, the chain rule through
// B = (2 pi)^-2 DFT(W c3) and c3(w) = (1/n) sum_i y(i) y(i+w1) y(i+w2) gives
//   G'(w)  = W(w) (2 pi)^-2 (1/n) Re sum_k G(k) exp(+i 2 pi k.w / N)
//   Gs     = (G' + G'^T) / 2                      (c3 is symmetric in w1, w2)
//   g(j)   = sum_w Gs(w) [ y(j+w1) y(j+w2) + 2 y(j-w1) y(j-w1+w2) ]
//   dx     = g - mean(g)                          (adjoint of the mean removal)
// Both terms of g come from one contraction over the Hankel matrix of y:
//   U[u, w1] = sum_w2 y(u + w2) Gs(w1, w2)
//   T1(u)    = sum_w1 U[u, w1] y(u + w1)            (row sums)
//   T2(j)    = sum_w1 U[j - w1, w1] y(j - w1)       (anti-diagonal sums)
//   g        = T1 + 2 T2.
// The contraction is FP32 FFMA on the CUDA cores; every reduction runs in a
// fixed order (deterministic).
#include "launch.cuh"

namespace hos {

// Gs[(w1+L)*2L + (w2+L)] from the adjoint transform Gc (complex, [w1 mod N][w2 mod N]).
__global__ void gs_kernel(const float2* __restrict__ Gc, int N, int L, int window, double scale,
                          float* __restrict__ Gs) {
    const int twoL = 2 * L;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= twoL * twoL) return;
    const int w1 = e / twoL - L, w2 = e % twoL - L;
    auto gp = [&](int a, int b) -> double {
        if (window == HOS_WIN_RECT && (rect_excluded(a, L) || rect_excluded(b, L))) return 0.0;
        const double wv = lag_window2(a, b, L, window);
        const int ka = (a % N + N) % N, kb = (b % N + N) % N;
        return wv * (double)Gc[(int64_t)ka * N + kb].x;
    };
    Gs[e] = (float)(0.5 * scale * (gp(w1, w2) + gp(w2, w1)));
}

constexpr int ADJ_U = 64;   // rows u per CTA
constexpr int ADJ_W = 64;   // w1 columns per pass, w2 per K step

// One CTA per 64 rows u.  Writes T1[u] for its rows and its T2 contributions
// t2p[cta][e], e = (u - u0) + (w1 + L) in [0, 64 + 2L - 1).
__global__ void __launch_bounds__(256) adjoint_u_kernel(const float* __restrict__ y, int64_t n, int L,
                                                        const float* __restrict__ Gs, float* __restrict__ T1,
                                                        float* __restrict__ t2p) {
    __shared__ float gsT[ADJ_W][ADJ_W + 1];   // gsT[w2 - w2c][w1 - w1c]
    __shared__ float yb[2 * ADJ_W];           // y(u0 + w2c + t)
    __shared__ float ya[2 * ADJ_W];           // y(u0 + w1c + t)
    __shared__ float yu[ADJ_U];               // y(u0 + t)
    __shared__ float Sd[ADJ_U][ADJ_W + 1];    // U[u, w1] * y(u)
    __shared__ float t1s[16][ADJ_U];
    extern __shared__ float t2cta[];           // 64 + 2L
    const int twoL = 2 * L;
    const int tu = threadIdx.x & 15, tw = threadIdx.x >> 4;
    const int64_t u0 = (int64_t)blockIdx.x * ADJ_U;
    const int e2 = ADJ_U + twoL;
    for (int t = threadIdx.x; t < e2; t += blockDim.x) t2cta[t] = 0.0f;
    for (int t = threadIdx.x; t < ADJ_U; t += blockDim.x) yu[t] = y[u0 + t];
    float t1[4] = {0.f, 0.f, 0.f, 0.f};
    for (int w1c = -L; w1c < L; w1c += ADJ_W) {
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int w2c = -L; w2c < L; w2c += ADJ_W) {
            __syncthreads();
            for (int t = threadIdx.x; t < ADJ_W * ADJ_W; t += blockDim.x) {
                const int r = t / ADJ_W, c = t % ADJ_W;  // r: w1 offset, c: w2 offset
                const int w1 = w1c + r, w2 = w2c + c;
                gsT[c][r] = (w1 < L && w2 < L) ? Gs[(int64_t)(w1 + L) * twoL + (w2 + L)] : 0.f;
            }
            for (int t = threadIdx.x; t < 2 * ADJ_W; t += blockDim.x) yb[t] = y[u0 + w2c + t];
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < ADJ_W; ++k) {
                float yv[4], gv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) yv[a] = yb[tu + 16 * a + k];
#pragma unroll
                for (int b = 0; b < 4; ++b) gv[b] = gsT[k][tw + 16 * b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(yv[a], gv[b], acc[a][b]);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * ADJ_W; t += blockDim.x) ya[t] = y[u0 + w1c + t];
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int r = tu + 16 * a;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int c = tw + 16 * b;
                t1[a] = fmaf(acc[a][b], ya[r + c], t1[a]);  // U[u, w1] y(u + w1)
                Sd[r][c] = acc[a][b] * yu[r];                // U[u, w1] y(u)
            }
        }
        __syncthreads();
        // anti-diagonal d = r + c in [0, 127): fixed order over r
        if (threadIdx.x < 2 * ADJ_W - 1) {
            const int d = threadIdx.x;
            float sdiag = 0.f;
            const int r0 = d < ADJ_W ? 0 : d - ADJ_W + 1, r1 = d < ADJ_W ? d : ADJ_W - 1;
            for (int r = r0; r <= r1; ++r) {
                const int c = d - r;
                if (w1c + c < L) sdiag += Sd[r][c];
            }
            if (d + (w1c + L) < e2) t2cta[d + (w1c + L)] += sdiag;  // only valid columns contribute
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) t1s[tw][tu + 16 * a] = t1[a];
    __syncthreads();
    if (threadIdx.x < ADJ_U) {
        float s = 0.f;
        for (int k = 0; k < 16; ++k) s += t1s[k][threadIdx.x];
        if (u0 + threadIdx.x < n) T1[u0 + threadIdx.x] = s;
    }
    float* dst = t2p + (int64_t)blockIdx.x * e2;
    for (int t = threadIdx.x; t < e2; t += blockDim.x) dst[t] = t2cta[t];
}

// g(j) = T1(j) + 2 sum_cta t2p[cta][j - u0(cta) + L], CTAs in increasing order.
__global__ void adjoint_gather_kernel(const float* __restrict__ T1, const float* __restrict__ t2p, int64_t n, int L,
                                      int64_t nctas, float* __restrict__ g) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int e2 = ADJ_U + 2 * L;
    int64_t c0 = j + L - (e2 - 1);
    c0 = c0 < 0 ? 0 : ceil_div(c0, ADJ_U);
    int64_t c1 = (j + L) / ADJ_U;
    if (c1 > nctas - 1) c1 = nctas - 1;
    double t2 = 0.0;
    for (int64_t c = c0; c <= c1; ++c) {
        const int64_t e = j - c * ADJ_U + L;
        if (e >= 0 && e < e2) t2 += (double)t2p[c * e2 + e];
    }
    g[j] = (float)((double)T1[j] + 2.0 * t2);
}

template <typename T>
__global__ void adjoint_finish_kernel(const float* __restrict__ g, int64_t n, const double* __restrict__ gmean,
                                      int remove_mean, T* __restrict__ dx) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double m = remove_mean ? gmean[0] : 0.0;
    dx[j] = (T)((double)g[j] - m);
}

cudaError_t launch_adjoint(const float* yS, int64_t n, int L, const float2* Gc, int N, int window, double scale,
                           float* Gs, float* T1, float* t2p, float* g, cudaStream_t st) {
    const int twoL = 2 * L;
    gs_kernel<<<(unsigned)ceil_div((int64_t)twoL * twoL, 256), 256, 0, st>>>(Gc, N, L, window, scale, Gs);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nctas = ceil_div(n, ADJ_U);
    const size_t dyn = sizeof(float) * (size_t)(ADJ_U + twoL);
    adjoint_u_kernel<<<(unsigned)nctas, 256, dyn, st>>>(yS, n, L, Gs, T1, t2p);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_gather_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(T1, t2p, n, L, nctas, g);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gs(const float2* Gc, int N, int L, int window, double scale, float* Gs, cudaStream_t st) {
    const int twoL = 2 * L;
    gs_kernel<<<(unsigned)ceil_div((int64_t)twoL * twoL, 256), 256, 0, st>>>(Gc, N, L, window, scale, Gs);
    count_launch();
    return cudaGetLastError();
}

// ---- fourth order ----------------------------------------------------------------
// Gs4[((w1+L)*2L + (w2+L))*2L + (w3+L)] = scale W(w) (1/6) sum over the six
// orders of (w1, w2, w3) of Re Gc[a mod N][b mod N][c mod N]: the lag-domain
// gradient of c4 (adjoint transform, window, 1/n folded into scale),
// symmetrised because c4 is symmetric in its three lags.
__global__ void gs4_kernel(const float2* __restrict__ Gc, int N, int L, int window, float scale,
                           float* __restrict__ Gs4) {
    // per-lag window factor d(w) (RECT: 0 at w = -L), in FP32 like the forward's grid
    __shared__ float wsh[2 * 64];
    const int twoL = 2 * L;
    for (int i = threadIdx.x; i < twoL; i += blockDim.x)
        wsh[i] = (window == HOS_WIN_RECT) ? (i == 0 ? 0.0f : 1.0f) : (float)parzen(i - L, L);
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)twoL * twoL * twoL) return;
    const int w3 = (int)(e % twoL) - L;
    const int w2 = (int)((e / twoL) % twoL) - L;
    const int w1 = (int)(e / ((int64_t)twoL * twoL)) - L;
    auto re = [&](int a, int b, int c) -> float {
        const int ka = a < 0 ? a + N : a, kb = b < 0 ? b + N : b, kc = c < 0 ? c + N : c;  // N >= 2L
        return Gc[((int64_t)ka * N + kb) * N + kc].x;
    };
    // the six terms in an order fixed by the sorted lags, so that every
    // permutation of (w1, w2, w3) gets the same FP32 value (exact symmetry)
    int a = w1, b = w2, c = w3, tmp;
    if (a > b) { tmp = a; a = b; b = tmp; }
    if (b > c) { tmp = b; b = c; c = tmp; }
    if (a > b) { tmp = a; a = b; b = tmp; }
    const float sym = ((re(a, b, c) + re(a, c, b)) + (re(b, a, c) + re(b, c, a))) + (re(c, a, b) + re(c, b, a));
    const float wv = wsh[w1 + L] * wsh[w2 + L] * wsh[w3 + L];
    Gs4[e] = sym * (scale * wv * (1.0f / 6.0f));
}

// dl/dc2(t) (times 1/n, which Gs4 carries) through the three c2 c2 products of
// c4(w) = m4(w) - c2(w1) c2(w3-w2) - c2(w2) c2(w3-w1) - c2(w3) c2(w2-w1):
// each product c2(a) c2(b) sends -Gs4(w) c2(b) to c2(a) and -Gs4(w) c2(a) to
// c2(b).  Gs4 is exactly symmetric in its three lags (gs4_kernel), so the
// three terms where a lag equals t are equal, H(t) = sum_{u,v} Gs4(t, u, v)
// c2(v - u), and so are the three where a lag difference equals t,
// K(t) = sum_{w2} sum_{w1} Gs4(w2, w2 + t, w1) c2(w1):
//   dl/dc2(t) = -3 (H(t) + K(t)),
// both read with the last lag fastest (coalesced).  One block per t in
// [-(2L-1), 2L-1]; FP32 per thread, FP64 tree across the block.
constexpr int GC2_THREADS = 256;
__global__ void __launch_bounds__(GC2_THREADS) gc2_kernel(const float* __restrict__ Gs4, const double* __restrict__ c2,
                                                          int L, double* __restrict__ gc2) {
    __shared__ double red[GC2_THREADS];
    __shared__ float cs[4 * 64];
    const int twoL = 2 * L, T = 2 * L - 1;
    for (int i = threadIdx.x; i < 2 * T + 1; i += GC2_THREADS) cs[i] = (float)c2[i];
    __syncthreads();
    const int t = (int)blockIdx.x - T;
    const float* c = cs + T;  // c[d], |d| <= T
    auto G = [&](int a, int b, int d) -> float {
        return Gs4[((int64_t)(a + L) * twoL + (b + L)) * twoL + (d + L)];
    };
    float acc = 0.0f;  // at most 2 (2L)^2 / 256 terms per thread
    for (int q = threadIdx.x; q < twoL * twoL; q += GC2_THREADS) {
        const int u = q / twoL - L, v = q % twoL - L;  // v fastest
        if (t >= -L && t < L) acc = fmaf(G(t, u, v), c[v - u], acc);          // H: a lag equals t
        if (u + t >= -L && u + t < L) acc = fmaf(G(u, u + t, v), c[v], acc);  // K: w2 = u, w1 = v
    }
    red[threadIdx.x] = (double)acc;
    __syncthreads();
    for (int d = GC2_THREADS / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) gc2[t + T] = -3.0 * red[0];
}

cudaError_t launch_gs4(const float2* Gc, int N, int L, int window, double scale, float* Gs4, cudaStream_t st) {
    const int64_t tot = (int64_t)8 * L * L * L;
    gs4_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Gc, N, L, window, (float)scale, Gs4);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gc2(const float* Gs4, const double* c2, int L, double* gc2, cudaStream_t st) {
    gc2_kernel<<<(unsigned)(4 * L - 1), GC2_THREADS, 0, st>>>(Gs4, c2, L, gc2);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_adjoint_finish(const float* g, int64_t n, const double* gmean, int remove_mean, int dtype, void* dx,
                                  cudaStream_t st) {
    const unsigned b = (unsigned)ceil_div(n, 256);
    if (dtype == HOS_F64) adjoint_finish_kernel<double><<<b, 256, 0, st>>>(g, n, gmean, remove_mean, (double*)dx);
    else adjoint_finish_kernel<float><<<b, 256, 0, st>>>(g, n, gmean, remove_mean, (float*)dx);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hos
