// dft.cu -- transform of the windowed cumulant onto the N-point grid, one axis
// at a time (the separable form of the 2-D / 3-D DFT), staged in shared memory.
//
//   out[k] = sum_e in[e] exp(sign * i 2 pi e k / N)     (sign -1: forward, the
//   sign of Algorithm DBS step 3; +1: the adjoint)
//
// A "line" is one 1-D transform along an axis of a row-major array:
//   line l starts at (l / inner) * outer_stride + (l % inner), element e at
//   + e * elem_stride.
// N a power of two: radix-2 Cooley-Tukey in shared memory (bit-reversed load,
// log2 N butterfly stages).  Otherwise: direct O(N^2) sum per line.
// Twiddles tw[k] = exp(-i 2 pi k / N), k < N, from FP64 sincospi, rounded to
// FP32 once per call.
#include "launch.cuh"

namespace hos {

__global__ void twiddle_kernel(int N, float2* tw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)N, &s, &c);
    tw[k] = make_float2((float)c, (float)-s);
}


HOS_DEV int64_t line_base(const LineGeom& g, int64_t l) { return (l / g.inner) * g.outer_stride + (l % g.inner); }

HOS_DEV float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// Shared-memory slot of element i of a line: one float2 of padding every 16
// keeps bit-reversed and strided butterfly accesses off a single bank; the
// line stride is odd (in float2) so that the same element of neighbouring
// lines falls in different banks.
HOS_DEV int sk(int i) { return i + (i >> 4); }
HOS_HD int skewed_len(int N) { return N + (N >> 4) + 1; }

template <bool REAL_IN>
HOS_DEV float2 load_in(const void* in, int64_t idx) {
    if constexpr (REAL_IN) return make_float2(reinterpret_cast<const float*>(in)[idx], 0.0f);
    else return reinterpret_cast<const float2*>(in)[idx];
}

// in and out may alias (every CTA reads all its lines before writing them).
template <bool REAL_IN>
__global__ void fft_lines_kernel(const void* in, float2* out, const LineGeom g, const float2* __restrict__ tw,
                                 int sign, float scale) {
    extern __shared__ float2 sbuf[];
    const int N = g.N, lpb = g.lpb, SL = skewed_len(N);
    int64_t* lbase = reinterpret_cast<int64_t*>(sbuf + (size_t)lpb * SL);  // line starts, computed once
    const int64_t l0 = (int64_t)blockIdx.x * lpb;
    const int nl = (int)((g.nlines - l0) < lpb ? (g.nlines - l0) : lpb);
    const int total = nl * N;
    const bool contiguous = (g.elem_stride == 1);
    for (int l = threadIdx.x; l < nl; l += blockDim.x) lbase[l] = line_base(g, l0 + l);
    __syncthreads();
    // loads in batches of 8 per thread so that several are in flight
    for (int base = 0; base < total; base += 8 * blockDim.x) {
        float2 v[8];
        int dst[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = base + u * blockDim.x + threadIdx.x;
            dst[u] = -1;
            if (idx < total) {
                int l, e;
                if (contiguous) { l = idx >> g.log2N; e = idx & (N - 1); }
                else { e = idx / nl; l = idx - e * nl; }
                v[u] = load_in<REAL_IN>(in, lbase[l] + (int64_t)e * g.elem_stride);
                dst[u] = l * SL + sk((int)(__brev((unsigned)e) >> (32 - g.log2N)));
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (dst[u] >= 0) sbuf[dst[u]] = v[u];
    }
    __syncthreads();
    const int lg = g.log2N;
    for (int sh = 0; sh < lg; ++sh) {  // butterfly span h = 2^sh, twiddle stride N / 2h
        const int h = 1 << sh;
        for (int bf = threadIdx.x; bf < nl * (N / 2); bf += blockDim.x) {
            const int l = bf >> (lg - 1), k = bf & ((N >> 1) - 1);
            const int j = k & (h - 1), blk = k >> sh;
            const int i0 = (blk << (sh + 1)) + j, i1 = i0 + h;
            float2 w = tw[j << (lg - 1 - sh)];
            if (sign > 0) w.y = -w.y;
            float2* row = sbuf + l * SL;
            const float2 a = row[sk(i0)], b = cmul(row[sk(i1)], w);
            row[sk(i0)] = make_float2(a.x + b.x, a.y + b.y);
            row[sk(i1)] = make_float2(a.x - b.x, a.y - b.y);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int l, e;
        if (contiguous) { l = idx >> g.log2N; e = idx & (N - 1); }
        else { e = idx / nl; l = idx - e * nl; }
        const float2 v = sbuf[l * SL + sk(e)];
        out[lbase[l] + (int64_t)e * g.elem_stride] = make_float2(v.x * scale, v.y * scale);
    }
}

// Radix-8 passes in registers.  A pass covers r <= 3 consecutive radix-2
// stages s0 .. s0+r-1 (span h = 2^s0): the index set {i0 + m h : m < 2^r},
// i0 = blk 2^(s0+r) + j (j < h), is closed under those stages, so one thread
// holds it in registers and does all r stages there (r 2^(r-1) butterflies).
// Each thread holds 8 values: 2^(3-r) such groups, g = q T + t (T = N/8
// threads per line).  The first pass reads the bit-reversed input straight
// from global memory, the last writes natural-order output straight back;
// passes in between exchange through shared memory.  Thread-to-line
// mapping: lanes run along the line when the line is contiguous, across
// lines when lines are strided (so that a warp's accesses are coalesced
// either way).
HOS_DEV int bitrev_n(int i, int lg) { return (int)(__brev((unsigned)i) >> (32 - lg)); }

template <int R>
HOS_DEV int group_index(int q, int m, int s0, int t, int T) {
    const int gidx = q * T + t, h = 1 << s0;
    return ((gidx >> s0) << (s0 + R)) + (gidx & (h - 1)) + m * h;
}

template <int R>
HOS_DEV void radix_pass(float2 (&v)[8], int s0, int lg, int t, int T, const float2* __restrict__ tws) {
    const int h = 1 << s0;
#pragma unroll
    for (int q = 0; q < (8 >> R); ++q) {
        const int j = (q * T + t) & (h - 1);
#pragma unroll
        for (int k = 0; k < R; ++k) {
#pragma unroll
            for (int m = 0; m < (1 << R); ++m) {
                if (m & (1 << k)) continue;
                const int jj = j + (m & ((1 << k) - 1)) * h;  // index within the span 2^(s0+k) h
                const float2 w = tws[jj << (lg - 1 - (s0 + k))];
                float2& a = v[q * (1 << R) + m];
                float2& b = v[q * (1 << R) + m + (1 << k)];
                const float2 bw = cmul(b, w);
                b = make_float2(a.x - bw.x, a.y - bw.y);
                a = make_float2(a.x + bw.x, a.y + bw.y);
            }
        }
    }
}

// The first pass (stages 0-2, span 1): twiddles W_2^0, W_4^j, W_8^j only, so
// they are constants -- 1, -/+i and (+/-1 -/+ i)/sqrt 2 -- and no table loads
// or general complex products are needed.  sg = -1 forward, +1 adjoint.
HOS_DEV void radix8_first(float2 (&v)[8], float sg) {
    const float r = 0.70710678118654752f;  // 1/sqrt(2)
#pragma unroll
    for (int m = 0; m < 8; m += 2) {  // stage 0
        const float2 a = v[m], b = v[m + 1];
        v[m] = make_float2(a.x + b.x, a.y + b.y);
        v[m + 1] = make_float2(a.x - b.x, a.y - b.y);
    }
#pragma unroll
    for (int q = 0; q < 8; q += 4) {  // stage 1: w = 1 (m = q), W_4^1 = (0, sg) (m = q + 1)
        const float2 a0 = v[q], b0 = v[q + 2];
        v[q] = make_float2(a0.x + b0.x, a0.y + b0.y);
        v[q + 2] = make_float2(a0.x - b0.x, a0.y - b0.y);
        const float2 a1 = v[q + 1], c = v[q + 3];
        const float2 b1 = make_float2(-sg * c.y, sg * c.x);
        v[q + 1] = make_float2(a1.x + b1.x, a1.y + b1.y);
        v[q + 3] = make_float2(a1.x - b1.x, a1.y - b1.y);
    }
    float2 b[4];  // stage 2: w = W_8^m, m = 0..3
    b[0] = v[4];
    b[1] = make_float2(r * (v[5].x - sg * v[5].y), r * (sg * v[5].x + v[5].y));
    b[2] = make_float2(-sg * v[6].y, sg * v[6].x);
    b[3] = make_float2(r * (-v[7].x - sg * v[7].y), r * (sg * v[7].x - v[7].y));
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float2 a = v[m];
        v[m] = make_float2(a.x + b[m].x, a.y + b[m].y);
        v[m + 4] = make_float2(a.x - b[m].x, a.y - b[m].y);
    }
}

template <int R>
HOS_DEV void pass_store(const float2 (&v)[8], float2* row, int s0, int t, int T) {
#pragma unroll
    for (int q = 0; q < (8 >> R); ++q)
#pragma unroll
        for (int m = 0; m < (1 << R); ++m) row[sk(group_index<R>(q, m, s0, t, T))] = v[q * (1 << R) + m];
}

template <int R>
HOS_DEV void pass_load(float2 (&v)[8], const float2* row, int s0, int t, int T) {
#pragma unroll
    for (int q = 0; q < (8 >> R); ++q)
#pragma unroll
        for (int m = 0; m < (1 << R); ++m) v[q * (1 << R) + m] = row[sk(group_index<R>(q, m, s0, t, T))];
}

template <bool REAL_IN, bool STRIDED>
__global__ void __launch_bounds__(1024) fft_r8_kernel(const void* in, float2* out, const LineGeom g,
                                                     const float2* __restrict__ tw, int sign, float scale) {
    extern __shared__ float2 sbuf[];
    const int N = g.N, lg = g.log2N, lpb = g.lpb, SL = skewed_len(N), T = N >> 3;
    float2* tws = sbuf + (size_t)lpb * SL;                          // N/2 twiddles, conjugated when sign > 0
    int64_t* lbase = reinterpret_cast<int64_t*>(tws + (N >> 1));  // line starts
    const int64_t l0 = (int64_t)blockIdx.x * lpb;
    const int nl = (int)((g.nlines - l0) < lpb ? (g.nlines - l0) : lpb);
    for (int k = threadIdx.x; k < (N >> 1); k += blockDim.x) {
        float2 w = tw[k];
        if (sign > 0) w.y = -w.y;
        tws[k] = w;
    }
    for (int l = threadIdx.x; l < nl; l += blockDim.x) lbase[l] = line_base(g, l0 + l);
    __syncthreads();
    const int l = STRIDED ? (int)(threadIdx.x % lpb) : (int)(threadIdx.x / T);
    const int t = STRIDED ? (int)(threadIdx.x / lpb) : (int)(threadIdx.x % T);
    const bool live = l < nl;
    const int64_t base = live ? lbase[l] : 0;
    const int64_t es = g.elem_stride;
    // Hermitian columns: line = column c of group gb; column N - c gets the conjugate mirror
    const int64_t lglob = l0 + l;
    const int hc = g.herm ? (int)(lglob % g.inner) : 0;
    const bool mirror = g.herm && hc != 0 && 2 * hc != N;
    const int64_t mbase = g.herm ? (lglob / g.inner) * g.outer_stride + (N - hc) : 0;
    float2* row = sbuf + (size_t)l * SL;
    float2 v[8];
    // first pass (s0 = 0, radix 8): group t holds inputs bitrev(8t + m)
    if (live) {
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = load_in<REAL_IN>(in, base + (int64_t)bitrev_n(8 * t + m, lg) * es);
    }
    radix8_first(v, sign > 0 ? 1.0f : -1.0f);
    int s0 = 3;
    while (s0 < lg) {
        const int r = (lg - s0) < 3 ? (lg - s0) : 3;
        __syncthreads();  // previous pass's reads of the rows are done (none before the first store)
        if (live) pass_store<3>(v, row, s0 - 3, t, T);  // layout of the previous (radix-8) pass
        __syncthreads();
        // the stored layout is the previous pass's; reload in this pass's groups
        if (r == 3) { if (live) pass_load<3>(v, row, s0, t, T); radix_pass<3>(v, s0, lg, t, T, tws); }
        else if (r == 2) { if (live) pass_load<2>(v, row, s0, t, T); radix_pass<2>(v, s0, lg, t, T, tws); }
        else { if (live) pass_load<1>(v, row, s0, t, T); radix_pass<1>(v, s0, lg, t, T, tws); }
        if (s0 + r >= lg) {  // last pass: natural-order output straight to global memory
            if (live) {
                auto put = [&](int idx, float2 o) {
                    const float2 w = make_float2(o.x * scale, o.y * scale);
                    out[base + (int64_t)idx * es] = w;
                    if (mirror) out[mbase + (int64_t)((N - idx) & (N - 1)) * es] = make_float2(w.x, -w.y);
                };
                if (r == 3) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) put(group_index<3>(0, m, s0, t, T), v[m]);
                } else if (r == 2) {
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int m = 0; m < 4; ++m) put(group_index<2>(q, m, s0, t, T), v[q * 4 + m]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int m = 0; m < 2; ++m) put(group_index<1>(q, m, s0, t, T), v[q * 2 + m]);
                }
            }
            return;
        }
        // a middle pass is always radix 8 (only the last can be shorter)
        s0 += 3;
    }
    // lg == 3: the first pass was the whole transform
    if (live) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const float2 w = make_float2(v[m].x * scale, v[m].y * scale);
            out[base + (int64_t)m * es] = w;
            if (mirror) out[mbase + (int64_t)((N - m) & (N - 1)) * es] = make_float2(w.x, -w.y);
        }
    }
}

// Two real contiguous lines a, b per complex transform: z = a + i b, Z =
// FFT(z), then A[k] = (Z[k] + conj Z[N-k]) / 2 and B[k] = (Z[k] - conj
// Z[N-k]) / (2i) (the transforms of real lines are Hermitian), which halves
// the butterfly work of a real-input pass.  Same passes as fft_r8_kernel;
// the last one leaves Z in shared memory in natural order for the split.
// lpb (real lines per CTA) is even, and so is the line count.
__global__ void __launch_bounds__(1024) fft_r8_pair_kernel(const float* __restrict__ in, float2* __restrict__ out,
                                                          const LineGeom g, const float2* __restrict__ tw, int sign,
                                                          float scale) {
    extern __shared__ float2 sbuf[];
    const int N = g.N, lg = g.log2N, lpb = g.lpb, SL = skewed_len(N), T = N >> 3;
    float2* tws = sbuf + (size_t)(lpb >> 1) * SL;
    int64_t* lbase = reinterpret_cast<int64_t*>(tws + (N >> 1));
    const int64_t l0 = (int64_t)blockIdx.x * lpb;
    const int nl = (int)((g.nlines - l0) < lpb ? (g.nlines - l0) : lpb);
    for (int k = threadIdx.x; k < (N >> 1); k += blockDim.x) {
        float2 w = tw[k];
        if (sign > 0) w.y = -w.y;
        tws[k] = w;
    }
    for (int l = threadIdx.x; l < nl; l += blockDim.x) lbase[l] = line_base(g, l0 + l);
    __syncthreads();
    const int pl = (int)(threadIdx.x / T), t = (int)(threadIdx.x % T);
    const bool live = 2 * pl < nl;
    const int64_t ba = live ? lbase[2 * pl] : 0, bb = live ? lbase[2 * pl + 1] : 0;
    float2* row = sbuf + (size_t)pl * SL;
    float2 v[8];
    if (live) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int e = bitrev_n(8 * t + m, lg);
            v[m] = make_float2(in[ba + e], in[bb + e]);
        }
    }
    radix8_first(v, sign > 0 ? 1.0f : -1.0f);
    int s0 = 3, slast = 0, rlast = 3;
    while (s0 < lg) {
        const int r = (lg - s0) < 3 ? (lg - s0) : 3;
        __syncthreads();
        if (live) pass_store<3>(v, row, s0 - 3, t, T);
        __syncthreads();
        if (r == 3) { if (live) pass_load<3>(v, row, s0, t, T); radix_pass<3>(v, s0, lg, t, T, tws); }
        else if (r == 2) { if (live) pass_load<2>(v, row, s0, t, T); radix_pass<2>(v, s0, lg, t, T, tws); }
        else { if (live) pass_load<1>(v, row, s0, t, T); radix_pass<1>(v, s0, lg, t, T, tws); }
        slast = s0;
        rlast = r;
        if (s0 + r >= lg) break;
        s0 += 3;
    }
    __syncthreads();  // the last pass's reads of the rows are done
    if (live) {
        if (rlast == 3) pass_store<3>(v, row, slast, t, T);
        else if (rlast == 2) pass_store<2>(v, row, slast, t, T);
        else pass_store<1>(v, row, slast, t, T);
    }
    __syncthreads();
    if (!live) return;
    const float h = 0.5f * scale;
    const int kend = g.half_out ? (N >> 1) + 1 : N;
    for (int k = t; k < kend; k += T) {
        const float2 zk = row[sk(k)], zn = row[sk((N - k) & (N - 1))];
        out[ba + k] = make_float2((zk.x + zn.x) * h, (zk.y - zn.y) * h);
        out[bb + k] = make_float2((zk.y + zn.y) * h, (zn.x - zk.x) * h);
    }
}

template <bool REAL_IN>
__global__ void dft_lines_kernel(const void* in, float2* out, const LineGeom g, const float2* __restrict__ tw,
                                 int sign, float scale) {
    extern __shared__ float2 sbuf[];
    const int N = g.N, lpb = g.lpb;
    int64_t* lbase = reinterpret_cast<int64_t*>(sbuf + 2 * (size_t)lpb * N);
    const int64_t l0 = (int64_t)blockIdx.x * lpb;
    const int nl = (int)((g.nlines - l0) < lpb ? (g.nlines - l0) : lpb);
    const int total = nl * N;
    for (int l = threadIdx.x; l < nl; l += blockDim.x) lbase[l] = line_base(g, l0 + l);
    __syncthreads();
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l = idx / N, e = idx % N;
        sbuf[idx] = load_in<REAL_IN>(in, lbase[l] + (int64_t)e * g.elem_stride);
    }
    __syncthreads();
    float2* res = sbuf + lpb * N;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l = idx / N, k = idx % N;
        float ax = 0.0f, ay = 0.0f;
        for (int e = 0; e < N; ++e) {
            float2 w = tw[(int)(((int64_t)e * k) % N)];
            if (sign > 0) w.y = -w.y;
            const float2 v = sbuf[l * N + e];
            ax += v.x * w.x - v.y * w.y;
            ay += v.x * w.y + v.y * w.x;
        }
        res[idx] = make_float2(ax * scale, ay * scale);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l = idx / N, e = idx % N;
        out[lbase[l] + (int64_t)e * g.elem_stride] = res[idx];
    }
}

cudaError_t launch_twiddles(int N, float2* tw, cudaStream_t st) {
    twiddle_kernel<<<(unsigned)ceil_div(N, 256), 256, 0, st>>>(N, tw);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lines(bool real_in, const void* in, float2* out, LineGeom g, const float2* tw, int sign,
                         float scale, cudaStream_t st) {
    if (g.nlines <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)ceil_div(g.nlines, g.lpb);
    if (g.log2N >= 3 && real_in && g.elem_stride == 1 && g.nlines % 2 == 0) {
        // real contiguous lines in pairs, one complex transform per pair
        const int T = g.N >> 3;
        int pairs = 256 / T;
        if (pairs > 32) pairs = 32;
        if (pairs < 1) pairs = 1;
        int lpb = 2 * pairs;
        if (lpb > g.nlines) lpb = (int)g.nlines;
        g.lpb = lpb;
        const unsigned nb = (unsigned)ceil_div(g.nlines, lpb);
        const size_t smem = (size_t)(lpb / 2) * skewed_len(g.N) * sizeof(float2) +
                            (size_t)(g.N >> 1) * sizeof(float2) + (size_t)lpb * sizeof(int64_t);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(fft_r8_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fft_r8_pair_kernel<<<nb, (unsigned)((lpb / 2) * T), smem, st>>>(reinterpret_cast<const float*>(in), out, g,
                                                                       tw, sign, scale);
    } else if (g.log2N >= 3) {
        // radix-8 register passes: N/8 threads per line (up to 1024 at N = 8192)
        const int T = g.N >> 3;
        const bool strided = g.elem_stride != 1;
        int lpb = strided ? 512 / T : 256 / T;
        if (lpb > 32) lpb = 32;
        if (lpb < 1) lpb = 1;
        if (lpb > g.nlines) lpb = (int)g.nlines;
        g.lpb = lpb;
        const unsigned nb = (unsigned)ceil_div(g.nlines, lpb);
        const size_t smem = (size_t)lpb * skewed_len(g.N) * sizeof(float2) + (size_t)(g.N >> 1) * sizeof(float2) +
                            (size_t)lpb * sizeof(int64_t);
        if (smem > 48 * 1024) {  // large nfft: opt in above the default 48 KB (per device, so on every such call)
            cudaFuncSetAttribute(fft_r8_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(fft_r8_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(fft_r8_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(fft_r8_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        }
        const unsigned th = (unsigned)(lpb * T);
        if (real_in) {
            if (strided) fft_r8_kernel<true, true><<<nb, th, smem, st>>>(in, out, g, tw, sign, scale);
            else fft_r8_kernel<true, false><<<nb, th, smem, st>>>(in, out, g, tw, sign, scale);
        } else {
            if (strided) fft_r8_kernel<false, true><<<nb, th, smem, st>>>(in, out, g, tw, sign, scale);
            else fft_r8_kernel<false, false><<<nb, th, smem, st>>>(in, out, g, tw, sign, scale);
        }
    } else if (g.log2N >= 0) {
        const size_t smem = (size_t)g.lpb * skewed_len(g.N) * sizeof(float2) + (size_t)g.lpb * sizeof(int64_t);
        if (real_in) fft_lines_kernel<true><<<blocks, 256, smem, st>>>(in, out, g, tw, sign, scale);
        else fft_lines_kernel<false><<<blocks, 256, smem, st>>>(in, out, g, tw, sign, scale);
    } else {
        const size_t smem = 2 * (size_t)g.lpb * g.N * sizeof(float2) + (size_t)g.lpb * sizeof(int64_t);
        if (real_in) dft_lines_kernel<true><<<blocks, 256, smem, st>>>(in, out, g, tw, sign, scale);
        else dft_lines_kernel<false><<<blocks, 256, smem, st>>>(in, out, g, tw, sign, scale);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace hos
