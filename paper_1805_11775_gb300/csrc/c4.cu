// c4.cu -- fourth-order cumulant over the lag cube (trispectrum path).
//
//   c4(w1,w2,w3) = m4(w1,w2,w3) - c2(w1) c2(w3-w2) - c2(w2) c2(w3-w1) - c2(w3) c2(w2-w1)
//   m4(w1,w2,w3) = (1/n) sum_i y(i) y(i+w1) y(i+w2) y(i+w3),   c2(t) = (1/n) sum_i y(i) y(i+t)
// (Problem Statement: moments and cumulants "and so on"; the zero-mean
// moment-to-cumulant identity is the reading of the fourth order.)
//
// m4 is symmetric in (w1, w2, w3), so only pairs w1 <= w2 are contracted:
//   M[p, w3] = sum_i T[p, i] * y(i + w3),   T[p, i] = y(i) y(i + w1_p) y(i + w2_p),
// an FP32 FFMA contraction (SIMT) over blocks of 128 pairs, in chunk groups of
// CG * 1024 samples, each group's FP32 partial summed in FP64 (this SIMT
// cross-check path).  c2 is accumulated in double-float (c2_kernel).
#include "launch.cuh"

namespace hos {

// lag pair index of (w1, w2), w1 <= w2, both in [-L, L): row-major over the triangle
HOS_HD int pair_index(int w1, int w2, int L) {
    const int a = w1 + L, b = w2 + L, twoL = 2 * L;
    return a * twoL - (a * (a - 1)) / 2 + (b - a);
}

// c2_s(t) for t in [-(2L-1), 2L-1] of every part s.  blockIdx.x = lag, .y =
// part, .z = slice of the part's samples (P slices).  GB300 issues FP64 at
// about 1/64 of its FP32 rate, so the sum runs in double-float on the FP32
// pipes: each product y(i) y(i+t) of two floats is split exactly into p + e
// (FMA), and p, e are added to a TwoSum chain per thread; the block combines
// the chains in a fixed tree.  P = 1 writes FP64 c2 directly; otherwise each
// slice writes its double-float sum and c2_finish_kernel adds the P slices
// in order.
// Time slice of a longer series (tslice = 1): the sum runs over the slice's
// own samples i in [0, len) and reads y(i + |t|) past the end from the halo
// the planes hold; lag -t gets the same value as t (the whole series'
// c2(t) = c2(-t), which is all the joined sum needs).  norm_len > 0 replaces
// the part's length as the divisor (the whole series' length).
constexpr int C2_THREADS = 512;
HOS_DEV float2 df2_add(float2 a, float2 b) {  // (a.h + a.l) + (b.h + b.l), renormalised
    const float sm = a.x + b.x;
    const float bb = sm - a.x;
    float e = (a.x - (sm - bb)) + (b.x - bb);
    e += a.y + b.y;
    const float h = sm + e;
    return make_float2(h, e - (h - sm));
}

__global__ void __launch_bounds__(C2_THREADS) c2_kernel(const float* __restrict__ y32, const int64_t* __restrict__ off,
                                                        const int64_t* __restrict__ pad, int L, int P, int tslice,
                                                        int64_t norm_len, double* __restrict__ c2,
                                                        float2* __restrict__ c2p) {
    __shared__ float2 sh[C2_THREADS];
    const int T = 2 * L - 1;
    const int bt = (int)blockIdx.x - T;
    const int t = (tslice && bt < 0) ? -bt : bt;
    const int s = blockIdx.y, z = blockIdx.z;
    const int64_t len = off[s + 1] - off[s];
    const double nl = (double)(norm_len > 0 ? norm_len : len);
    const float* y = y32 + pad[s] + L;  // y[i], zero-padded on both sides by >= L
    float hi = 0.0f, lo = 0.0f;
    const int64_t a0 = t < 0 ? -t : 0, a1 = (t > 0 && !tslice) ? len - t : len;
    const int64_t span = a1 > a0 ? a1 - a0 : 0, per = (span + P - 1) / P;
    const int64_t i0 = a0 + per * z, i1 = (i0 + per < a1) ? i0 + per : a1;
#pragma unroll 4
    for (int64_t i = i0 + threadIdx.x; i < i1; i += C2_THREADS) {
        const float a = y[i], b = y[i + t];
        const float p = a * b;
        const float e = fmaf(a, b, -p);  // a b = p + e exactly
        const float sm = hi + p;
        const float bv = sm - hi;
        lo += ((hi - (sm - bv)) + (p - bv)) + e;
        hi = sm;
    }
    sh[threadIdx.x] = make_float2(hi, lo);
    __syncthreads();
    for (int d = C2_THREADS / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) sh[threadIdx.x] = df2_add(sh[threadIdx.x], sh[threadIdx.x + d]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const int64_t e = (int64_t)s * (2 * T + 1) + blockIdx.x;
    if (P == 1) c2[e] = len > 0 ? ((double)sh[0].x + (double)sh[0].y) / nl : 0.0;
    else c2p[e * P + z] = sh[0];
}

__global__ void c2_finish_kernel(const float2* __restrict__ c2p, const int64_t* __restrict__ off, int S, int L, int P,
                                 int64_t norm_len, double* __restrict__ c2) {
    const int T = 2 * L - 1;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)S * (2 * T + 1)) return;
    const int s = (int)(e / (2 * T + 1));
    const int64_t len = off[s + 1] - off[s];
    float2 a = c2p[e * P];
    for (int z = 1; z < P; ++z) a = df2_add(a, c2p[e * P + z]);
    c2[e] = len > 0 ? ((double)a.x + (double)a.y) / (double)(norm_len > 0 ? norm_len : len) : 0.0;
}

constexpr int M4_PAIRS = 128;  // pairs per CTA
constexpr int M4_KI = 32;      // samples per inner step

// blockIdx.x = pair block, blockIdx.y = global chunk group (series found by
// search in the group prefix win[]).  Thread (tq, tp): pairs tp + 16a (a < 8),
// w3 = -L + tq + 16b (b < NB, NB = 2L/16).
template <int NB>
__global__ void __launch_bounds__(256) m4_simt_kernel(const float* __restrict__ y32, const int64_t* __restrict__ off,
                                                      const int64_t* __restrict__ pad, const int64_t* __restrict__ win,
                                                      int S, int L, int CG, int npairs, float* __restrict__ part) {
    constexpr int W3 = 16 * NB;  // w3 columns, 2L rounded up to a multiple of 16
    __shared__ float T[M4_KI][M4_PAIRS];
    __shared__ float yw[M4_KI + W3];  // yw[k] = y(i0 + k - L)
    __shared__ int pw1[M4_PAIRS], pw2[M4_PAIRS];
    const int tq = threadIdx.x & 15, tp = threadIdx.x >> 4;
    const int twoL = 2 * L;
    const int64_t g = blockIdx.y;
    int lo = 0, hi = S;  // series with win[s] <= g < win[s+1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (win[mid] <= g) lo = mid; else hi = mid;
    }
    const int s = lo;
    const int64_t len = off[s + 1] - off[s];
    const int64_t cg = g - win[s];
    const int64_t i_begin = cg * CG * KC;
    const int64_t i_end = (i_begin + (int64_t)CG * KC < len) ? i_begin + (int64_t)CG * KC : len;
    const float* y = y32 + pad[s] + L;  // y[i] valid for i in [-L, len + pad_tail)
    // this block's pairs
    for (int q = threadIdx.x; q < M4_PAIRS; q += blockDim.x) {
        const int p = blockIdx.x * M4_PAIRS + q;
        int w1 = L, w2 = L;  // out of range marks an unused slot
        if (p < npairs) {
            int a = 0;
            while (a < twoL - 1 && pair_index(a + 1 - L, a + 1 - L, L) <= p) ++a;
            w1 = a - L;
            w2 = w1 + (p - pair_index(w1, w1, L));
        }
        pw1[q] = w1;
        pw2[q] = w2;
    }
    float acc[8][NB];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[a][b] = 0.0f;
    for (int64_t i0 = i_begin; i0 < i_end; i0 += M4_KI) {
        __syncthreads();
        for (int k = threadIdx.x; k < M4_KI + W3; k += blockDim.x) yw[k] = y[i0 + k - L];
        __syncthreads();
        // T[k][q] = y(i0+k) y(i0+k+w1) y(i0+k+w2); samples past the series are zero
        for (int e = threadIdx.x; e < M4_KI * M4_PAIRS; e += blockDim.x) {
            const int k = e / M4_PAIRS, q = e % M4_PAIRS;
            const int w1 = pw1[q], w2 = pw2[q];
            float v = 0.0f;
            if (w1 < L && w2 < L) v = yw[k + L] * yw[k + L + w1] * yw[k + L + w2];
            T[k][q] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < M4_KI; ++k) {
            float tv[8], yv[NB];
#pragma unroll
            for (int a = 0; a < 8; ++a) tv[a] = T[k][tp + 16 * a];
#pragma unroll
            for (int b = 0; b < NB; ++b) yv[b] = yw[k + tq + 16 * b];  // y(i0 + k + w3), w3 = -L + tq + 16b
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b) acc[a][b] = fmaf(tv[a], yv[b], acc[a][b]);
        }
    }
    // partial[g][pair][w3 + L], rows of W3
    const int64_t ppad = (int64_t)gridDim.x * M4_PAIRS;
    float* dst = part + g * ppad * W3;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int64_t p = (int64_t)blockIdx.x * M4_PAIRS + tp + 16 * a;
#pragma unroll
        for (int b = 0; b < NB; ++b) dst[p * W3 + tq + 16 * b] = acc[a][b];
    }
}

// mode 0: grid3[(w1 mod N)][(w2 mod N)][(w3 mod N)] = scale * W * c4 (fp32)
// mode 1: c4out[w1+L][w2+L][w3+L] = c4 (fp64)
struct Reduce4Params {
    const float* partials;
    int w3;
    const double* c2;
    const int64_t* off;
    const int64_t* win;
    int S;
    int L;
    int npblocks;
    int window;
    int nfft;
    int mode;
    double scale;
    float* grid;
    double* c4out;
};

__global__ void reduce4_kernel(const Reduce4Params P) {
    const int L = P.L, twoL = 2 * L, T = 2 * L - 1, W3 = P.w3;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)twoL * twoL * twoL) return;
    const int w3 = (int)(e % twoL) - L;
    const int w2 = (int)((e / twoL) % twoL) - L;
    const int w1 = (int)(e / ((int64_t)twoL * twoL)) - L;
    const int p = (w1 <= w2) ? pair_index(w1, w2, L) : pair_index(w2, w1, L);
    const int64_t ppad = (int64_t)P.npblocks * M4_PAIRS;
    double c4 = 0.0;
    int k = 0;
    for (int s = 0; s < P.S; ++s) {
        const int64_t len = P.off[s + 1] - P.off[s];
        if (len <= 0) continue;
        double m4 = 0.0;
        const int64_t g0 = P.win[s], g1 = P.win[s + 1];
        for (int64_t gb = g0; gb < g1; gb += 16) {  // groups of 16 as a two-float sum, added in FP64
            const int64_t ge = (gb + 16 < g1) ? gb + 16 : g1;
            float hi = 0.0f, lo = 0.0f;
            for (int64_t g = gb; g < ge; ++g) {
                const float v = P.partials[(g * ppad + p) * W3 + (w3 + L)];
                const float sum = hi + v;
                const float bv = sum - hi;
                lo += (hi - (sum - bv)) + (v - bv);
                hi = sum;
            }
            m4 += (double)hi + (double)lo;
        }
        m4 /= (double)len;
        const double* c2 = P.c2 + (int64_t)s * (2 * T + 1) + T;  // c2[t], t in [-T, T]
        c4 += m4 - c2[w1] * c2[w3 - w2] - c2[w2] * c2[w3 - w1] - c2[w3] * c2[w2 - w1];
        ++k;
    }
    if (k > 0) c4 /= (double)k;
    if (P.mode == 1) {
        P.c4out[((int64_t)(w1 + L) * twoL + (w2 + L)) * twoL + (w3 + L)] = c4;
        return;
    }
    const double wv = (P.window == HOS_WIN_RECT && (w1 == -L || w2 == -L || w3 == -L))
                          ? 0.0
                          : lag_window3(w1, w2, w3, L, P.window);
    const int N = P.nfft;
    const int k1 = (w1 % N + N) % N, k2 = (w2 % N + N) % N, k3 = (w3 % N + N) % N;
    P.grid[((int64_t)k1 * N + k2) * N + k3] = (float)(P.scale * wv * c4);
}

// Fourth order from the tensor-core path: c4 of each part from its m4 (m4buf)
// and c2, averaged over parts, then windowed onto the grid (mode 0) or
// written raw (mode 1).
// per_series: blockIdx.y = series s, whose c4 goes to its own grid (no average).
__global__ void c4_assemble_kernel(const double* __restrict__ m4buf, const double* __restrict__ c2,
                                   const int64_t* __restrict__ off, int S, int L, int ntiles, int tile_n,
                                   C4ReduceArgs r, int per_series) {
    const int twoL = 2 * L, T = 2 * L - 1;
    // per-lag window factor d(w) (RECT: 0 at w = -L), FP32 like the grid
    __shared__ float wsh[2 * 64];
    for (int i = threadIdx.x; i < twoL; i += blockDim.x)
        wsh[i] = (r.window == HOS_WIN_RECT) ? (i == 0 ? 0.0f : 1.0f) : (float)parzen(i - L, L);
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)twoL * twoL * twoL) return;
    const int w3 = (int)(e % twoL) - L;
    const int w2 = (int)((e / twoL) % twoL) - L;
    const int w1 = (int)(e / ((int64_t)twoL * twoL)) - L;
    const int p = (w1 <= w2) ? pair_index(w1, w2, L) : pair_index(w2, w1, L);
    const int t = p / TILE_M, m = p % TILE_M;
    const int64_t tsz = (int64_t)TILE_M * tile_n;
    const int64_t elem = (int64_t)(w3 + L) * TILE_M + m;
    double c4 = 0.0;
    int k = 0;
    const int s0 = per_series ? (int)blockIdx.y : 0, s1 = per_series ? s0 + 1 : S;
    for (int s = s0; s < s1; ++s) {
        if (off[s + 1] <= off[s]) continue;
        const double m4 = m4buf[((int64_t)s * ntiles + t) * tsz + elem];
        const double* c = c2 + (int64_t)s * (2 * T + 1) + T;
        c4 += (r.mode == 2) ? m4 : m4 - c[w1] * c[w3 - w2] - c[w2] * c[w3 - w1] - c[w3] * c[w2 - w1];
        ++k;
    }
    if (k > 0) c4 /= (double)k;
    if (r.mode >= 1) {  // 1: raw c4, 2: raw m4 (time slices), both FP64 over the cube
        r.c4out[(int64_t)(per_series ? blockIdx.y : 0) * twoL * twoL * twoL +
                ((int64_t)(w1 + L) * twoL + (w2 + L)) * twoL + (w3 + L)] = c4;
        return;
    }
    const float wv = wsh[w1 + L] * wsh[w2 + L] * wsh[w3 + L];
    const int N = r.nfft;  // >= 2L, so w + N >= 0
    const int k1 = w1 < 0 ? w1 + N : w1, k2 = w2 < 0 ? w2 + N : w2, k3 = w3 < 0 ? w3 + N : w3;
    r.grid[(int64_t)(per_series ? blockIdx.y : 0) * N * N * N + ((int64_t)k1 * N + k2) * N + k3] =
        (float)c4 * ((float)r.scale * wv);
}

int c2_slices(int S, int64_t max_len) {
    if (S > 16) return 1;  // S x (4L - 1) blocks already fill the GPU
    int64_t p = max_len / 8192;
    return (int)(p < 1 ? 1 : (p > 16 ? 16 : p));
}

cudaError_t launch_c2(const float* y32, const int64_t* off, const int64_t* pad, int S, int L, int P, double* c2,
                      float2* c2p, cudaStream_t st, int tslice, int64_t norm_len) {
    const int T = 2 * L - 1;
    c2_kernel<<<dim3((unsigned)(2 * T + 1), (unsigned)S, (unsigned)P), C2_THREADS, 0, st>>>(y32, off, pad, L, P, tslice,
                                                                                             norm_len, c2, c2p);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || P == 1) return err;
    const int64_t tot = (int64_t)S * (2 * T + 1);
    c2_finish_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(c2p, off, S, L, P, norm_len, c2);
    count_launch();
    return cudaGetLastError();
}

// The trispectrum's lag-domain input from a joined fourth moment and c2 (the
// sums of a series' time slices): c4 = m4 - c2(w1) c2(w3-w2) - c2(w2) c2(w3-w1)
// - c2(w3) c2(w2-w1) in FP64, then window and scale onto the N^3 grid as
// c4_assemble_kernel's mode 0 does.  m4: (2L)^3 [w1+L][w2+L][w3+L]; c2: 4L-1
// values, index t + 2L - 1.
__global__ void c4_from_moments_kernel(const double* __restrict__ m4, const double* __restrict__ c2, int L,
                                       C4ReduceArgs r) {
    const int twoL = 2 * L, T = 2 * L - 1;
    __shared__ float wsh[2 * 64];
    for (int i = threadIdx.x; i < twoL; i += blockDim.x)
        wsh[i] = (r.window == HOS_WIN_RECT) ? (i == 0 ? 0.0f : 1.0f) : (float)parzen(i - L, L);
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)twoL * twoL * twoL) return;
    const int w3 = (int)(e % twoL) - L;
    const int w2 = (int)((e / twoL) % twoL) - L;
    const int w1 = (int)(e / ((int64_t)twoL * twoL)) - L;
    const double* c = c2 + T;
    const double c4 = m4[e] - c[w1] * c[w3 - w2] - c[w2] * c[w3 - w1] - c[w3] * c[w2 - w1];
    const float wv = wsh[w1 + L] * wsh[w2 + L] * wsh[w3 + L];
    const int N = r.nfft;  // >= 2L
    const int k1 = w1 < 0 ? w1 + N : w1, k2 = w2 < 0 ? w2 + N : w2, k3 = w3 < 0 ? w3 + N : w3;
    r.grid[((int64_t)k1 * N + k2) * N + k3] = (float)c4 * ((float)r.scale * wv);
}

cudaError_t launch_c4_from_moments(const double* m4, const double* c2, int L, const C4ReduceArgs& r, cudaStream_t st) {
    const int64_t n3 = 8LL * L * L * L;
    c4_from_moments_kernel<<<(unsigned)ceil_div(n3, 256), 256, 0, st>>>(m4, c2, L, r);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_c4_assemble(const double* m4buf, const double* c2, const int64_t* off, int S, int L, int ntiles,
                               int tile_n, const C4ReduceArgs& r, int per_series, cudaStream_t st) {
    const int64_t n3 = 8LL * L * L * L;
    dim3 grid((unsigned)ceil_div(n3, 256), per_series ? (unsigned)S : 1u);
    c4_assemble_kernel<<<grid, 256, 0, st>>>(m4buf, c2, off, S, L, ntiles, tile_n, r, per_series);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_c4(const float* y32, const int64_t* off, const int64_t* pad, const int64_t* win, int S, int L,
                      int CG, int64_t total_groups, double* c2, float* partials, const C4ReduceArgs& r,
                      cudaStream_t st) {
    const int T = 2 * L - 1;
    c2_kernel<<<dim3((unsigned)(2 * T + 1), (unsigned)S), C2_THREADS, 0, st>>>(y32, off, pad, L, 1, 0, 0, c2, nullptr);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int twoL = 2 * L;
    const int npairs = twoL * (twoL + 1) / 2;
    const int npb = (npairs + M4_PAIRS - 1) / M4_PAIRS;
    const int nb = (twoL + 15) / 16;
    if (total_groups > 0) {
        dim3 grid((unsigned)npb, (unsigned)total_groups);
#define HOS_M4_CASE(K) \
    case K: m4_simt_kernel<K><<<grid, 256, 0, st>>>(y32, off, pad, win, S, L, CG, npairs, partials); break;
        switch (nb) {
            HOS_M4_CASE(1) HOS_M4_CASE(2) HOS_M4_CASE(3) HOS_M4_CASE(4)
            HOS_M4_CASE(5) HOS_M4_CASE(6) HOS_M4_CASE(7) HOS_M4_CASE(8)
            default: return cudaErrorInvalidValue;
        }
#undef HOS_M4_CASE
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    Reduce4Params rp{partials, 16 * nb, c2, off, win, S, L, npb, r.window, r.nfft, r.mode, r.scale, r.grid, r.c4out};
    const int64_t n3 = (int64_t)twoL * twoL * twoL;
    reduce4_kernel<<<(unsigned)ceil_div(n3, 256), 256, 0, st>>>(rp);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hos
