// direct.cu -- the paper's direct method (Algorithm DBS) on the GPU:
//
//   1-2. parts of M samples every M - overlap samples (overlap 0: the paper's
//        partition into K = floor(n / M) parts), each minus its own mean (FP64);
//   3.   F_p(k) = sum_u X_p(u) e^{-j 2 pi u k / M}: the transform kernels of
//        dft.cu over the K part lines;
//   4.   raw C3_p(k1,k2) = (1/M) F_p(k1) F_p(k2) F_p*(k1+k2), indices mod M,
//        averaged over the parts here already (step 6 moved before step 5:
//        both steps are linear, so the order does not change the result, and
//        the smoothing runs once instead of K times);
//   5.   M3 x M3 box smoothing by window sums: down each column a running
//        window sum updated in O(1) per step, s(i+1) = s(i) - a(i) + a(i+M3)
//        (Algorithm WS); along each row window sums as differences of prefix
//        sums (Algorithm WS_PRAM).  Offsets lo .. lo + M3 - 1 with
//        lo = -floor(M3 / 2), indices mod M.
// Running sums and prefix sums are double-float (a pair of floats kept
// renormalised with TwoSum): a window sum is the difference of much larger
// running values.
#include "launch.cuh"

namespace hos {

namespace {

HOS_DEV void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (h + l) += (bh + bl), renormalised
HOS_DEV void df_acc(float& h, float& l, float bh, float bl) {
    float s, e;
    two_sum(h, bh, s, e);
    e += l + bl;
    h = s + e;
    l = e - (h - s);
}

}  // namespace

// mean[p] of part p = x[p step .. p step + M), FP64, fixed-order tree per
// block (one block per part); 0 without mean removal.
template <typename T>
__global__ void __launch_bounds__(256) part_mean_kernel(const T* __restrict__ x, int64_t M, int64_t step,
                                                        int remove_mean, double* __restrict__ mean) {
    __shared__ double sh[256];
    const T* xp = x + (int64_t)blockIdx.x * step;
    double a = 0.0;
    if (remove_mean)
        for (int64_t u = threadIdx.x; u < M; u += 256) a += (double)xp[u];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
        if (threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[blockIdx.x] = remove_mean ? sh[0] / (double)M : 0.0;
}

// y[p][u] = x[p step + u] - mean[p] (FP64 difference, FP32 result)
template <typename T>
__global__ void demean_parts_kernel(const T* __restrict__ x, int64_t total, int64_t M, int64_t step,
                                    const double* __restrict__ mean, float* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / M;
        y[i] = (float)((double)x[p * step + (i - p * M)] - mean[p]);
    }
}

// R[k1][k2] = (1 / (K M)) sum_p F_p(k1) F_p(k2) conj F_p((k1 + k2) mod M)
__global__ void triple_product_kernel(const float2* __restrict__ F, int K, int M, float2* __restrict__ R) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * M) return;
    const int k1 = (int)(e / M), k2 = (int)(e % M);
    const int k3 = (k1 + k2) % M;
    float re = 0.0f, im = 0.0f;
    for (int p = 0; p < K; ++p) {
        const float2* f = F + (int64_t)p * M;
        const float2 a = f[k1], b = f[k2], c = f[k3];
        const float pr = a.x * b.x - a.y * b.y, pi = a.x * b.y + a.y * b.x;  // F(k1) F(k2)
        re += pr * c.x + pi * c.y;                                          // times conj F(k3)
        im += pi * c.x - pr * c.y;
    }
    const float s = 1.0f / ((float)K * (float)M);
    R[e] = make_float2(re * s, im * s);
}

// Column window sums: Cw[k1][k2] = sum_{n = lo}^{lo + M3 - 1} R[(k1 + n) mod M][k2].
// Thread = (column k2, run of `seg` rows): the first sum directly (M3 reads),
// then the O(1) update per step (2 reads).  Consecutive threads take
// consecutive columns, so every row access is coalesced; runs several times
// longer than M3 keep the first sums' extra reads small.
__global__ void col_window_sums_kernel(const float2* __restrict__ R, int M, int M3, int seg,
                                       float2* __restrict__ Cw) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k2 = (int)(tid % M);
    const int r0 = (int)(tid / M) * seg;
    if (r0 >= M) return;
    const int r1 = (r0 + seg < M) ? r0 + seg : M;
    const int lo = -(M3 / 2);
    auto row = [&](int k) { k %= M; if (k < 0) k += M; return k; };
    float rh = 0.0f, rl = 0.0f, ih = 0.0f, il = 0.0f;
#pragma unroll 8
    for (int n = lo; n < lo + M3; ++n) {  // independent loads: several in flight
        const float2 v = R[(int64_t)row(r0 + n) * M + k2];
        df_acc(rh, rl, v.x, 0.0f);
        df_acc(ih, il, v.y, 0.0f);
    }
    Cw[(int64_t)r0 * M + k2] = make_float2(rh + rl, ih + il);
#pragma unroll 4
    for (int k1 = r0 + 1; k1 < r1; ++k1) {
        const float2 out = R[(int64_t)row(k1 - 1 + lo) * M + k2];
        const float2 in = R[(int64_t)row(k1 - 1 + lo + M3) * M + k2];
        df_acc(rh, rl, in.x, 0.0f);  // each term added exactly (TwoSum)
        df_acc(rh, rl, -out.x, 0.0f);
        df_acc(ih, il, in.y, 0.0f);
        df_acc(ih, il, -out.y, 0.0f);
        Cw[(int64_t)k1 * M + k2] = make_float2(rh + rl, ih + il);
    }
}

// Row window sums and the 1/M3^2 average: block = one row k1.  The row plus
// its circular continuation (M + M3 - 1 values, starting at column lo) goes to
// shared memory as double-float; an inclusive prefix sum P follows (each
// thread scans a contiguous run; warp 0 turns the runs' totals into offsets,
// 32 runs per lane in order, then a fixed-order scan across the lanes; each
// thread adds its offset);
// then B[k1][k2] = (P[k2 + M3 - 1] - P[k2 - 1]) / M3^2 (P[-1] = 0).
constexpr int ROW_THREADS = 1024;
__global__ void __launch_bounds__(ROW_THREADS) row_window_sums_kernel(const float2* __restrict__ Cw, int M, int M3,
                                                              float2* __restrict__ B) {
    extern __shared__ float4 pre[];  // (re.h, re.l, im.h, im.l), M + M3 - 1 entries
    __shared__ float4 runs[ROW_THREADS];
    const int k1 = blockIdx.x;
    const int lo = -(M3 / 2);
    const int len = M + M3 - 1;
    const float2* src = Cw + (int64_t)k1 * M;
#pragma unroll 4
    for (int j = threadIdx.x; j < len; j += blockDim.x) {
        int k = j + lo;  // lo > -M, j < M + M3 - 1 <= 2M - 1
        k = k < 0 ? k + M : (k >= M ? k - M : k);
        const float2 v = src[k];
        pre[j] = make_float4(v.x, 0.0f, v.y, 0.0f);
    }
    __syncthreads();
    // each thread: inclusive scan of its run [a, b)
    const int per = (len + blockDim.x - 1) / blockDim.x;
    const int a = threadIdx.x * per, b = (a + per < len) ? a + per : len;
    float rh = 0.0f, rl = 0.0f, ih = 0.0f, il = 0.0f;
    for (int j = a; j < b; ++j) {
        const float4 v = pre[j];
        df_acc(rh, rl, v.x, v.y);
        df_acc(ih, il, v.z, v.w);
        pre[j] = make_float4(rh, rl, ih, il);
    }
    runs[threadIdx.x] = make_float4(rh, rl, ih, il);
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive offsets of the runs: warp 0, PER runs per lane, then a lane scan
        constexpr int PER = ROW_THREADS / 32;
        const int lane = threadIdx.x;
        float oh = 0.0f, ol = 0.0f, qh = 0.0f, ql = 0.0f;  // this lane's PER runs, inclusive
        for (int t = lane * PER; t < lane * PER + PER; ++t) {
            const float4 r = runs[t];
            df_acc(oh, ol, r.x, r.y);
            df_acc(qh, ql, r.z, r.w);
        }
        // inclusive scan of the lane totals over the warp (Hillis-Steele, fixed order)
        for (int d = 1; d < 32; d <<= 1) {
            const float a = __shfl_up_sync(0xffffffffu, oh, d), b = __shfl_up_sync(0xffffffffu, ol, d);
            const float c = __shfl_up_sync(0xffffffffu, qh, d), e = __shfl_up_sync(0xffffffffu, ql, d);
            if (lane >= d) {
                df_acc(oh, ol, a, b);
                df_acc(qh, ql, c, e);
            }
        }
        // exclusive offset of this lane's first run: the previous lane's inclusive total
        float xh = __shfl_up_sync(0xffffffffu, oh, 1), xl = __shfl_up_sync(0xffffffffu, ol, 1);
        float yh = __shfl_up_sync(0xffffffffu, qh, 1), yl = __shfl_up_sync(0xffffffffu, ql, 1);
        if (lane == 0) xh = xl = yh = yl = 0.0f;
        for (int t = lane * PER; t < lane * PER + PER; ++t) {
            const float4 r = runs[t];
            runs[t] = make_float4(xh, xl, yh, yl);
            df_acc(xh, xl, r.x, r.y);
            df_acc(yh, yl, r.z, r.w);
        }
    }
    __syncthreads();
    {
        const float4 o = runs[threadIdx.x];
        for (int j = a; j < b; ++j) {
            float4 v = pre[j];
            df_acc(v.x, v.y, o.x, o.y);
            df_acc(v.z, v.w, o.z, o.w);
            pre[j] = v;
        }
    }
    __syncthreads();
    const float inv = 1.0f / ((float)M3 * (float)M3);
    for (int k2 = threadIdx.x; k2 < M; k2 += blockDim.x) {
        float4 hi = pre[k2 + M3 - 1];
        if (k2 > 0) {
            const float4 lo4 = pre[k2 - 1];
            df_acc(hi.x, hi.y, -lo4.x, -lo4.y);
            df_acc(hi.z, hi.w, -lo4.z, -lo4.w);
        }
        B[(int64_t)k1 * M + k2] = make_float2((hi.x + hi.y) * inv, (hi.z + hi.w) * inv);
    }
}

cudaError_t launch_part_prep(const void* x, int dtype, int64_t K, int64_t M, int64_t step, int remove_mean,
                             double* mean, float* y, cudaStream_t st) {
    if (dtype == HOS_F64)
        part_mean_kernel<double><<<(unsigned)K, 256, 0, st>>>((const double*)x, M, step, remove_mean, mean);
    else
        part_mean_kernel<float><<<(unsigned)K, 256, 0, st>>>((const float*)x, M, step, remove_mean, mean);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t b = ceil_div(K * M, 256);
    if (b > 8192) b = 8192;
    if (dtype == HOS_F64)
        demean_parts_kernel<double><<<(unsigned)b, 256, 0, st>>>((const double*)x, K * M, M, step, mean, y);
    else
        demean_parts_kernel<float><<<(unsigned)b, 256, 0, st>>>((const float*)x, K * M, M, step, mean, y);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_direct_smooth(const float2* F, int K, int M, int M3, float2* R, float2* Cw, float2* B,
                                 cudaStream_t st) {
    const int64_t MM = (int64_t)M * M;
    triple_product_kernel<<<(unsigned)ceil_div(MM, 256), 256, 0, st>>>(F, K, M, R);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int seg = 4 * M3;  // rows per thread: 4 x the box, 64 .. 512
    if (seg < 64) seg = 64;
    if (seg > 512) seg = 512;
    const int64_t cthreads = (int64_t)M * ceil_div(M, seg);
    col_window_sums_kernel<<<(unsigned)ceil_div(cthreads, 256), 256, 0, st>>>(R, M, M3, seg, Cw);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)(M + M3 - 1) * sizeof(float4);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(row_window_sums_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    row_window_sums_kernel<<<(unsigned)M, ROW_THREADS, smem, st>>>(Cw, M, M3, B);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hos
