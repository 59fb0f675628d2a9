// c3_simt.cu -- the same contraction C[w1,w2] = sum_i y(i) y(i+w1) y(i+w2) in
// plain FP32 FFMA on the CUDA cores.  It walks the same stream-K unit ranges
// and writes the same partial tiles as the tensor-core kernel, so the
// reduction is shared; it serves as the FP32 cross-check path.
//
// CTA = 256 threads over a 128 x N tile: thread (tx, ty) owns rows
// ty + 16 r (r < 8) and columns tx + 16 c (c < N/16).  Per chunk the CTA
// stages three 1-D windows of y in shared memory:
//   ya[t] = y(i0 + w1_0 + t), yi[t] = y(i0 + t), yb[t] = y(i0 + w2_0 + t).
#include "launch.cuh"

namespace hos {


template <int NC>  // columns per thread = N / 16
__global__ void __launch_bounds__(256) c3_simt_kernel(const C3SimtParams P) {
    __shared__ float ya[KC + TILE_M];
    __shared__ float yi[KC];
    __shared__ float yb[KC + 16 * NC];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const C3Geom& geo = P.geom;
    const int N = 16 * NC;
    Walk walk;
    walk.init(geo, P.ser, blockIdx.x, gridDim.x);
    Part part;
    while (walk.next(part)) {
        const int a = geo.tile_a[part.t], col0 = 32 * geo.tile_c32[part.t];
        const int64_t base = P.ser.pad[part.s];
        const int64_t slen = P.ser.off[part.s + 1] - P.ser.off[part.s];  // rows i >= len: y(i) = 0
        float acc[8][NC];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[r][c] = 0.0f;
        const int kc = geo.kc;
        for (int64_t ch = part.c0; ch < part.c1; ++ch) {
            const int64_t i0 = ch * kc;
            const float* ga = P.y32 + base + i0 + (int64_t)a * TILE_M;
            const float* gi = P.y32 + base + geo.L + i0;
            const float* gb = P.y32 + base + i0 + col0;  // all N columns (the reduction reads the tile's width)
            __syncthreads();
            for (int t = threadIdx.x; t < kc + TILE_M; t += 256) ya[t] = ga[t];
            for (int t = threadIdx.x; t < kc; t += 256) yi[t] = (i0 + t < slen) ? gi[t] : 0.0f;
            for (int t = threadIdx.x; t < kc + N; t += 256) yb[t] = gb[t];
            __syncthreads();
#pragma unroll 4
            for (int i = 0; i < kc; ++i) {
                const float v = yi[i];
                float av[8], bv[NC];
#pragma unroll
                for (int r = 0; r < 8; ++r) av[r] = v * ya[i + ty + 16 * r];
#pragma unroll
                for (int c = 0; c < NC; ++c) bv[c] = yb[i + tx + 16 * c];
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
            }
        }
        float* dst = P.partials + part.slot * (int64_t)(TILE_M * N);
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < NC; ++c) dst[(int64_t)(tx + 16 * c) * TILE_M + ty + 16 * r] = acc[r][c];
    }
}

cudaError_t launch_c3_simt(const C3SimtParams& p, int G, cudaStream_t st) {
    switch (p.geom.tile_n) {
        case 32: c3_simt_kernel<2><<<G, 256, 0, st>>>(p); break;
        case 64: c3_simt_kernel<4><<<G, 256, 0, st>>>(p); break;
        case 128: c3_simt_kernel<8><<<G, 256, 0, st>>>(p); break;
        case 256: c3_simt_kernel<16><<<G, 256, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace hos
