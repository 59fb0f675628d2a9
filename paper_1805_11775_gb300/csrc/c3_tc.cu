// c3_tc.cu -- third-order cumulant contraction on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators), sm_103a.
//
// The sample cumulant c3(w1,w2) = (1/n) sum_i y(i) y(i+w1) y(i+w2) (Problem
// Statement; biased time average, zero outside the series) is the contraction
//     C[w1, w2] = sum_i Y[w1, i] * X[i, w2],
//     Y[w1, i] = y(i) y(i+w1)          (lag-product rows),
//     X[i, w2] = y(i + w2)             (Hankel matrix of the series).
//
// Operands of one tcgen05.mma (M = 128 rows of w1, N = the tile's width in
// columns of w2, at most 256; K = 16 samples for kind::f16, 8 for kind::tf32):
//   A = Y, built by four "builder" warps in registers and stored straight into
//       tensor memory (tcgen05.st); the MMA reads A from TMEM, so shared memory
//       carries only B.
//   B = X, never expanded.  Eight (bf16) or four (tf32) copies of the 1-D
//       sample window, each shifted by one sample, are interleaved in 16-byte
//       blocks: block (q, r) = samples [R*q + r, R*q + r + 16/elt).  In the
//       no-swizzle K-major canonical layout a core matrix is 8 rows of 16
//       bytes at a 16-byte pitch, so row n of the core matrix at group q is
//       block (q, n): the unit shift between Hankel rows falls out of the
//       layout, with LBO (K direction) and SBO (N direction) equal to the byte
//       distance of the next 8 (resp. 4) samples.
//   D = FP32 accumulator, 128 lanes x (widest tile) columns of TMEM.
//
// Precision: y = hi + lo (bf16 pair, f16 pair of the series scaled by a
// power of two, or tf32 pair); Y is formed in FP32 (times the scale's square,
// or cube for the fourth order) and split the same way; three products
// hi*hi + hi*lo + lo*hi per step (plain TF32: hi*hi alone).
//
// Warp roles (320 threads, one CTA per SM, persistent, stream-K ranges):
//   warps 0-3 builders (TMEM lane quadrants 0-3), warps 4-7 epilogue,
//   warp 8 producer (1-D bulk copies + window interleave), warp 9 MMA issuer.
// Every wait is bounded; on a timeout the CTA records HOS_ERR_TIMEOUT, drains
// its MMAs, frees TMEM and exits.
#include "launch.cuh"

namespace hos {


// ---- shared-memory plan ------------------------------------------------------
constexpr int MAX_STAGE = 6;     // A stages in TMEM (64 columns each): 4, or 6 when the tile is <= 64 wide
constexpr int WIN_SAMPLES = KC + 256 + 16;
constexpr int WIN_BYTES = WIN_SAMPLES * 16;  // interleaved window, one plane
constexpr int YA_FLOATS = KC + TILE_M;
// Four copies of the A window, copy s shifted by s samples, so that a row at
// any lag offset reads four consecutive samples with one aligned 16-byte
// load.  The copy pitch is 8 words mod 32: eight lanes at consecutive
// offsets then touch eight distinct bank quads.
constexpr int YA_STRIDE = YA_FLOATS + 8;
constexpr int YI_FLOATS = KC + 4;

// The producer's bulk copies land in two staging sets (the next chunk's copies
// fly while the current one is interleaved); the consumers read the buffers.
struct __align__(16) C3Smem {
    uint8_t win_hi[2][WIN_BYTES];
    uint8_t win_lo[2][WIN_BYTES];
    float ya[2][4][YA_STRIDE];        // [buffer][shift]; copies 1-3 only for fourth order
    float yi[2][KC];                  // y(i0 + t), 16-byte aligned for broadcast loads
    float st_ya[2][YA_FLOATS];        // staging: the A window
    float st_yi[2][YI_FLOATS];        // staging: y(i0 ..) from an aligned global start
    uint8_t st_hi[2][WIN_SAMPLES * 4];  // staging: the hi plane window, linear
    uint8_t st_lo[2][WIN_SAMPLES * 4];
    uint64_t full_b[2], empty_b[2], full_a[MAX_STAGE], empty_a[MAX_STAGE];
    uint64_t acc_full[2], acc_empty[2], drain, tma_bar[2];
    uint32_t tmem_base;
    int abort;
};

HOS_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
HOS_DEV void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// ORDER 3: rows of A are lags w1 (Y = y(i) y(i+w1)), tile row a covers
//          w1 = -L + 128a + m; columns are lags w2 of tile column b.
// ORDER 4: rows of A are lag pairs p = 128a + m with w1 <= w2
//          (T = y(i) y(i+w1) y(i+w2)); columns are lags w3 = -L + j.
template <int FMT, int ORDER>
__global__ void __launch_bounds__(320, 1) c3_tc_kernel(const C3TcParams P) {
    constexpr bool TF32 = FMT == FMT_TF32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    C3Smem& sm = *reinterpret_cast<C3Smem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const C3Geom& geo = P.geom;
    const int N = geo.tile_n;
    const int L = geo.L;
    constexpr int ELT = TF32 ? 4 : 2;              // bytes per plane element
    constexpr int R = 16 / ELT;                    // samples per 16-byte block
    constexpr int KB = TF32 ? 32 : 64;             // samples per A stage
    constexpr int KSTEP = TF32 ? 8 : 16;           // samples per MMA
    constexpr uint32_t GROUP_BYTES = 16u * R;      // bytes per R-sample group
    constexpr uint32_t LBO = GROUP_BYTES;          // next core matrix along K: +R samples
    constexpr uint32_t SBO = 16u * 8u;             // next 8 rows along N: +8 samples = 128 bytes
    const int csz = geo.kc;  // samples per chunk (the role loops below count chunks in kc)
    // TMEM columns: accumulators first -- two buffers when the tile is at most
    // 128 wide (the epilogue drains one while the MMAs fill the other), one of
    // N columns otherwise -- then the A stages, 64 columns each.  A tile at
    // most 64 wide has 4x less MMA work per stage than a 256-wide one, so it
    // takes 6 stages (two 64-column accumulators) to keep as much work queued.
    const uint32_t nacc = (N <= 128) ? 2u : 1u;
    const uint32_t acc_cols = (N <= 64) ? 64u : 128u;  // column stride between accumulators
    const uint32_t a_base = (N <= 64) ? 128u : 256u;   // first A stage column
    const int nst = (N <= 64) ? 6 : 4;                 // A stages
    const bool split = P.products != 1;                // plain TF32 issues hi*hi only

    if (threadIdx.x == 0) {
        // one elected arrival per arriving warp
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.full_b[i], 1);
            mbar_init(&sm.empty_b[i], 1);
        }
        for (int i = 0; i < MAX_STAGE; ++i) {
            mbar_init(&sm.full_a[i], 4);
            mbar_init(&sm.empty_a[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.acc_full[i], 1);
            mbar_init(&sm.acc_empty[i], 4);
        }
        mbar_init(&sm.drain, 1);
        mbar_init(&sm.tma_bar[0], 1);
        mbar_init(&sm.tma_bar[1], 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    if (warp == 9) {
        tmem_alloc(&sm.tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int* abort = &sm.abort;
    const uint64_t lim = P.limit_ns;

    Walk walk;
    walk.init(geo, P.ser, blockIdx.x, gridDim.x);
    Part part;

    if (warp == 8) {
        // ------------------------------------------------------------ producer
        // Chunk kc's copies go to staging set kc & 1; they are issued one chunk
        // ahead, before the previous chunk's window is interleaved, so that
        // their latency overlaps that work.  A chunk is (part, c).
        uint32_t kc = 0, tph[2] = {0u, 0u};
        bool inflight[2] = {false, false};
        bool ok = true;
        Part cur;
        bool have = walk.next(cur);
        int64_t cc = have ? cur.c0 : 0;
        // issue the copies of chunk (p, c) into staging set q; false on a failed bounds check
        auto issue = [&](const Part& p, int64_t c, int q) -> bool {
            const int64_t base = P.ser.pad[p.s];
            const int64_t i0 = c * csz;
            const int wt = 32 * geo.tile_w32[p.t];
            const int64_t wb = base + i0 + 32 * geo.tile_c32[p.t];  // plane index of the window start
            // A window: y(i0 + w1_0 + t) for ORDER 3; y(i0 - L + t) for ORDER 4
            const int64_t ab = (ORDER == 3) ? base + i0 + (int64_t)geo.tile_a[p.t] * TILE_M : base + i0;
            const int64_t ib_al = (base + L + i0) & ~(int64_t)3;  // y(i0), from an aligned start
            const uint32_t wbytes = (uint32_t)(csz + wt + 16) * ELT;
#ifdef HOS_DEBUG_BOUNDS
            {   // every copy inside this series' padded block, the part's slot inside the
                // workspace: otherwise record a fault and stop before any access
                const int64_t b0 = P.ser.pad[p.s], b1 = P.ser.pad[p.s + 1];
                const bool bad = b1 > P.plane_len || wb < b0 || wb + csz + wt + 16 > b1 || ab < b0 ||
                                 ab + csz + TILE_M > b1 || ib_al < b0 || ib_al + csz + 4 > b1 || p.slot < 0 ||
                                 p.slot >= P.n_slots;
                if (bad) {
                    if (lane == 0) {
                        record_status(P.status, HOS_ERR_DEVICE_FAULT);
                        *abort = 1;
                    }
                    return false;
                }
            }
#endif
            fence_proxy_async_smem();  // this set's earlier reads, before the copies overwrite it
            __syncwarp();
            if (lane == 0) {
                const uint32_t yab = (uint32_t)(csz + TILE_M) * 4, yib = (uint32_t)(csz + 4) * 4;
                mbar_expect_tx(&sm.tma_bar[q], 2 * wbytes + yab + yib);
                bulk_g2s(sm.st_hi[q], (const uint8_t*)P.hi + wb * ELT, wbytes, &sm.tma_bar[q]);
                bulk_g2s(sm.st_lo[q], (const uint8_t*)P.lo + wb * ELT, wbytes, &sm.tma_bar[q]);
                bulk_g2s(sm.st_ya[q], P.y32 + ab, yab, &sm.tma_bar[q]);
                bulk_g2s(sm.st_yi[q], P.y32 + ib_al, yib, &sm.tma_bar[q]);
            }
            inflight[q] = true;
            return true;
        };
        if (have) ok = issue(cur, cc, 0);
        while (ok && have) {
            const int buf = kc & 1;
            // the chunk after this one (possibly in the next part)
            Part nxt = cur;
            int64_t nc = cc + 1;
            bool have_next = true;
            if (nc >= cur.c1) {
                have_next = walk.next(nxt);
                nc = have_next ? nxt.c0 : 0;
            }
            ok = warp_wait(&sm.tma_bar[buf], tph[buf], abort, P.status, lim, P.hint[0]);
            if (!ok) break;
            inflight[buf] = false;
            tph[buf] ^= 1;
            if (have_next) {
                ok = issue(nxt, nc, buf ^ 1);
                if (!ok) break;
            }
            ok = warp_wait(&sm.empty_b[buf], ((kc >> 1) & 1) ^ 1, abort, P.status, lim, P.hint[0]);
            if (!ok) break;
            const int64_t base = P.ser.pad[cur.s];
            // rows i >= len carry y(i) = 0 (a time slice keeps its neighbour's
            // samples after it in the plane, for the lags only)
            const int64_t slen = P.ser.off[cur.s + 1] - P.ser.off[cur.s];
            // the row factor carries the series' scale s to the power ORDER - 1 (times the
            // window's s: the products come out scaled by s^ORDER, divided out in the reduction)
            float sA = 1.0f;
            if (P.ser.scale) {
                const float sc = P.ser.scale[cur.s];
                sA = (ORDER == 3) ? sc * sc : sc * sc * sc;
            }
            const int wt = 32 * geo.tile_w32[cur.t];
            const int64_t i0 = cc * csz;
            {   // realign y(i0 + t) so that builders can use 16-byte broadcast loads
                const int64_t ib = base + L + i0;
                const int ish = (int)(ib - (ib & ~(int64_t)3));
                for (int t = lane; t < csz; t += 32)
                    sm.yi[buf][t] = (i0 + t < slen) ? sm.st_yi[buf][ish + t] * sA : 0.0f;
            }
            {   // the A window; fourth order also its shifted copies ya[buf][s][j] = y0[j + s].
                // The last group reads up to 4 words past the window (inside the staging row);
                // those land only at j + s past the window, which no row reads.
                const float* y0 = sm.st_ya[buf];
                for (int g = lane; g < (csz + TILE_M) / 4; g += 32) {
                    const float4 u = *reinterpret_cast<const float4*>(y0 + 4 * g);
                    *reinterpret_cast<float4*>(sm.ya[buf][0] + 4 * g) = u;
                    if constexpr (ORDER == 4) {
                        const float4 v = (4 * g + 4 < YA_FLOATS) ? *reinterpret_cast<const float4*>(y0 + 4 * g + 4)
                                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                        *reinterpret_cast<float4*>(sm.ya[buf][1] + 4 * g) = make_float4(u.y, u.z, u.w, v.x);
                        *reinterpret_cast<float4*>(sm.ya[buf][2] + 4 * g) = make_float4(u.z, u.w, v.x, v.y);
                        *reinterpret_cast<float4*>(sm.ya[buf][3] + 4 * g) = make_float4(u.w, v.x, v.y, v.z);
                    }
                }
            }
            // interleave: block (q, r) <- samples [R q + r, R q + r + R)
            const int ngroups = (csz + wt) / R + 2;
            const int nblocks = ngroups * R;
            const uint32_t* sh = reinterpret_cast<const uint32_t*>(sm.st_hi[buf]);
            const uint32_t* sl = reinterpret_cast<const uint32_t*>(sm.st_lo[buf]);
            for (int blk = lane; blk < nblocks; blk += 32) {
                const int q = blk / R, r = blk % R;
                const int e0 = R * q + r;  // first sample of the block
                uint4 vh, vl;
                if constexpr (TF32) {
                    vh = make_uint4(sh[e0], sh[e0 + 1], sh[e0 + 2], sh[e0 + 3]);
                    vl = make_uint4(sl[e0], sl[e0 + 1], sl[e0 + 2], sl[e0 + 3]);
                } else {
                    const int w0 = e0 >> 1;
                    const uint32_t sft = (e0 & 1) * 16;
                    uint32_t h[5], l[5];
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        h[k] = sh[w0 + k];
                        l[k] = sl[w0 + k];
                    }
                    vh = make_uint4(__funnelshift_r(h[0], h[1], sft), __funnelshift_r(h[1], h[2], sft),
                                    __funnelshift_r(h[2], h[3], sft), __funnelshift_r(h[3], h[4], sft));
                    vl = make_uint4(__funnelshift_r(l[0], l[1], sft), __funnelshift_r(l[1], l[2], sft),
                                    __funnelshift_r(l[2], l[3], sft), __funnelshift_r(l[3], l[4], sft));
                }
                *reinterpret_cast<uint4*>(sm.win_hi[buf] + (size_t)blk * 16) = vh;
                *reinterpret_cast<uint4*>(sm.win_lo[buf] + (size_t)blk * 16) = vl;
            }
            fence_proxy_async_smem();  // every lane's window writes, for the MMA's reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.full_b[buf]);
            cur = nxt;
            cc = nc;
            have = have_next;
            ++kc;
        }
        // copies still in flight land in this CTA's shared memory: wait for them
        // (bounded, whatever the abort flag says) before the CTA exits
        for (int q = 0; q < 2; ++q)
            if (inflight[q] && lane == 0) {
                volatile int keep_waiting = 0;
                mbar_wait(&sm.tma_bar[q], tph[q], &keep_waiting, P.status, lim);
            }
        __syncwarp();
    } else if (warp < 4) {
        // ------------------------------------------------------------ builders
        const int m = warp * 32 + lane;  // TMEM lane = row of A (lag w1, or lag pair, in the tile)
        uint32_t kc = 0, ks = 0;
        bool ok = true;
        while (ok && walk.next(part)) {
            // ORDER 4: this row's lag pair (w1 <= w2).  Rows past the last pair
            // take the pair (-L, 0); nothing downstream reads those rows.
            int o1 = 0, o2 = 0;
            if constexpr (ORDER == 4) {
                const int twoL = 2 * L, npairs = twoL * (twoL + 1) / 2;
                const int pidx = geo.tile_a[part.t] * TILE_M + m;
                int r = 0, start = 0;  // row r of the triangle holds pairs (r, r..2L-1)
                while (r < twoL - 1 && start + (twoL - r) <= pidx) {
                    start += twoL - r;
                    ++r;
                }
                if (pidx >= npairs) {
                    r = 0;
                    start = 0;
                }
                o1 = L + (r - L);                  // ya index offset of y(i + w1): L + w1
                o2 = L + (r + (pidx - start) - L);  // ya index offset of y(i + w2)
                if (pidx >= npairs) o2 = L;
            }
            for (int64_t c = part.c0; c < part.c1 && ok; ++c, ++kc) {
                const int buf = kc & 1;
                ok = warp_wait(&sm.full_b[buf], (kc >> 1) & 1, abort, P.status, lim, P.hint[1]);
                if (!ok) break;
                const float* ya = sm.ya[buf][0] + (ORDER == 3 ? m : 0);
                // ORDER 4: y(i + w1) and y(i + w2) from the copies that put them on
                // a 16-byte boundary
                const float* c1 = sm.ya[buf][o1 & 3] + (o1 & ~3);
                const float* c2 = sm.ya[buf][o2 & 3] + (o2 & ~3);
                const float* yi = sm.yi[buf];
                for (int kb = 0; kb < csz / KB; ++kb, ++ks) {
                    const int st = (int)(ks % (uint32_t)nst);
                    ok = warp_wait(&sm.empty_a[st], ((ks / (uint32_t)nst) & 1) ^ 1, abort, P.status, lim, P.hint[1]);
                    if (!ok) break;
                    tc_fence_after();  // the MMAs that read this stage have completed
                    uint32_t H[32], Lw[32];
                    const float* pa = ya + kb * KB;
                    const float* pi = yi + kb * KB;
                    const float4* pi4 = reinterpret_cast<const float4*>(pi);
                    if constexpr (ORDER == 4) {
                        // T = y(i) y(i+w1) y(i+w2); ya[t] = y(i0 - L + t)
                        const float4* q1 = reinterpret_cast<const float4*>(c1 + kb * KB);
                        const float4* q2 = reinterpret_cast<const float4*>(c2 + kb * KB);
                        if constexpr (TF32) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 v = pi4[q], a1 = q1[q], a2 = q2[q];
                                const float pv[4] = {v.x * a1.x * a2.x, v.y * a1.y * a2.y, v.z * a1.z * a2.z,
                                                     v.w * a1.w * a2.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const uint32_t h = to_tf32(pv[e]);
                                    H[4 * q + e] = h;
                                    Lw[4 * q + e] = to_tf32(pv[e] - __uint_as_float(h));
                                }
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const float4 v = pi4[q], a1 = q1[q], a2 = q2[q];
                                const float p0 = v.x * a1.x * a2.x, p1 = v.y * a1.y * a2.y;
                                const float p2 = v.z * a1.z * a2.z, p3 = v.w * a1.w * a2.w;
                                const uint32_t h0 = pack2<FMT>(p0, p1), h1 = pack2<FMT>(p2, p3);
                                const float2 f0 = unpack2<FMT>(h0), f1 = unpack2<FMT>(h1);
                                H[2 * q] = h0;
                                H[2 * q + 1] = h1;
                                Lw[2 * q] = pack2<FMT>(p0 - f0.x, p1 - f0.y);
                                Lw[2 * q + 1] = pack2<FMT>(p2 - f1.x, p3 - f1.y);
                            }
                        }
                    } else if constexpr (TF32) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 v = pi4[q];
                            const float pv[4] = {v.x * pa[4 * q], v.y * pa[4 * q + 1], v.z * pa[4 * q + 2],
                                                 v.w * pa[4 * q + 3]};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const uint32_t h = to_tf32(pv[e]);
                                H[4 * q + e] = h;
                                Lw[4 * q + e] = to_tf32(pv[e] - __uint_as_float(h));
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const float4 v = pi4[q];
                            const float p0 = v.x * pa[4 * q], p1 = v.y * pa[4 * q + 1];
                            const float p2 = v.z * pa[4 * q + 2], p3 = v.w * pa[4 * q + 3];
                            const uint32_t h0 = pack2<FMT>(p0, p1), h1 = pack2<FMT>(p2, p3);
                            const float2 f0 = unpack2<FMT>(h0), f1 = unpack2<FMT>(h1);
                            H[2 * q] = h0;
                            H[2 * q + 1] = h1;
                            Lw[2 * q] = pack2<FMT>(p0 - f0.x, p1 - f0.y);
                            Lw[2 * q + 1] = pack2<FMT>(p2 - f1.x, p3 - f1.y);
                        }
                    }
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + a_base + (uint32_t)st * 64u;
                    tmem_st32(ta, H);
                    if (split) tmem_st32(ta + 32u, Lw);
                    tmem_wait_st();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.full_a[st]);
                }
            }
        }
    } else if (warp < 8) {
        // ------------------------------------------------------------ epilogue
        const int q = warp - 4;  // lane quadrant
        const int m = q * 32 + lane;
        uint32_t it = 0;
        bool ok = true;
        while (ok && walk.next(part)) {
            const uint32_t ab_ = it % nacc;
            ok = warp_wait(&sm.acc_full[ab_], (it / nacc) & 1, abort, P.status, lim, P.hint[2]);
            if (!ok) break;
            tc_fence_after();
            float* dst = P.partials + part.slot * (int64_t)(TILE_M * N) + m;
            const int wt = 32 * geo.tile_w32[part.t];
            for (int cc = 0; cc < wt; cc += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + ab_ * acc_cols + (uint32_t)cc, v);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) dst[(int64_t)(cc + j) * TILE_M] = __uint_as_float(v[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.acc_empty[ab_]);
            ++it;
        }
    } else if (warp == 9 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        uint32_t kc = 0, ks = 0, it = 0;
        bool ok = true;
        const uint32_t wh0 = smem_u32(sm.win_hi[0]), wl0 = smem_u32(sm.win_lo[0]);
        while (ok && walk.next(part)) {
            const uint32_t ab_ = it % nacc;
            const uint32_t dacc = tmem + ab_ * acc_cols;  // this part's accumulator
            const uint32_t idesc = make_idesc(FMT, TILE_M, 32 * geo.tile_w32[part.t]);  // N = the tile's width
            ok = mbar_wait(&sm.acc_empty[ab_], ((it / nacc) & 1) ^ 1, abort, P.status, lim, P.hint[3]);
            if (!ok) break;
            tc_fence_after();
            uint32_t acc = 0;
            for (int64_t c = part.c0; c < part.c1 && ok; ++c, ++kc) {
                const int buf = kc & 1;
                ok = mbar_wait(&sm.full_b[buf], (kc >> 1) & 1, abort, P.status, lim, P.hint[3]);
                if (!ok) break;
                tc_fence_after();
                const uint32_t wh = wh0 + (uint32_t)buf * WIN_BYTES, wl = wl0 + (uint32_t)buf * WIN_BYTES;
                // descriptors of the chunk's first K step; later steps add their byte
                // offset / 16 to the start-address field (addresses stay below 256 KB,
                // so the 14-bit field does not carry)
                const uint64_t bh0 = make_sdesc(wh, LBO, SBO), bl0 = make_sdesc(wl, LBO, SBO);
                for (int kb = 0; kb < csz / KB; ++kb, ++ks) {
                    const int st = (int)(ks % (uint32_t)nst);
                    ok = mbar_wait(&sm.full_a[st], (ks / (uint32_t)nst) & 1, abort, P.status, lim, P.hint[3]);
                    if (!ok) break;
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < KB / KSTEP; ++k) {
                        const uint32_t a_hi = tmem + a_base + (uint32_t)st * 64u + (uint32_t)k * 8u;
                        const uint32_t a_lo = a_hi + 32u;
                        const uint32_t koff = (uint32_t)(kb * KB + k * KSTEP);  // samples into the chunk
                        const uint64_t boff16 = (uint64_t)((koff / R) * GROUP_BYTES) >> 4;
                        const uint64_t bh = bh0 + boff16;
                        const uint64_t bl = bl0 + boff16;
                        mma_ts<TF32>(dacc, a_hi, bh, idesc, acc);
                        acc = 1;
                        if (split) {
                            mma_ts<TF32>(dacc, a_hi, bl, idesc, 1);
                            mma_ts<TF32>(dacc, a_lo, bh, idesc, 1);
                        }
                    }
                    mma_commit(&sm.empty_a[st]);
                }
                mma_commit(&sm.empty_b[buf]);
            }
            if (!ok) break;
            mma_commit(&sm.acc_full[ab_]);
            ++it;
        }
        // drain every MMA this thread issued before TMEM is released
        mma_commit(&sm.drain);
        {   // every MMA must have completed before TMEM is freed, also after an
            // abort: wait whatever the abort flag says, bounded (at least 0.2 s)
            volatile int keep_waiting = 0;
            mbar_wait(&sm.drain, 0, &keep_waiting, P.status, lim > 200000000ull ? lim : 200000000ull);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 9) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}



template <int FMT, int ORDER>
static cudaError_t launch_one(const C3TcParams& p, int G, cudaStream_t st) {
    // at least 116 KB so that exactly one CTA (and one 512-column TMEM
    // allocation) lands on each SM
    const size_t smem = sizeof(C3Smem) > 118784 ? sizeof(C3Smem) : 118784;
    // The attribute belongs to the current device (and context): set it on
    // every launch, so that any device the caller switches to has it.
    cudaError_t e =
        cudaFuncSetAttribute(c3_tc_kernel<FMT, ORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    c3_tc_kernel<FMT, ORDER><<<G, 320, smem, st>>>(p);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_c3_tc(int fmt, int order, const C3TcParams& p, int G, cudaStream_t st) {
    if (order == 4) {
        if (fmt == FMT_TF32) return launch_one<FMT_TF32, 4>(p, G, st);
        return fmt == FMT_F16 ? launch_one<FMT_F16, 4>(p, G, st) : launch_one<FMT_BF16, 4>(p, G, st);
    }
    if (fmt == FMT_TF32) return launch_one<FMT_TF32, 3>(p, G, st);
    return fmt == FMT_F16 ? launch_one<FMT_F16, 3>(p, G, st) : launch_one<FMT_BF16, 3>(p, G, st);
}

}  // namespace hos
