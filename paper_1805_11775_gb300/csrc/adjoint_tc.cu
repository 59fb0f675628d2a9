// adjoint_tc.cu -- the adjoint contraction U[u, w1] = sum_w2 y(u + w2) Gs(w1, w2)
// on the tensor cores (tcgen05, split-bf16 or split-FP16 of power-of-two scaled
// operands, FP32 accumulate), with both
// gradient terms taken in the epilogue:
//   T1(u) = sum_w1 U[u, w1] y(u + w1)         (row sums, per thread)
//   T2(j) = sum_w1 U[j - w1, w1] y(j - w1)    (anti-diagonal sums)
//
// MMA operands (M = 128 rows u, N = 128 lags w1 of one block, K = 16 lags w2):
//   A = Hankel X[u, w2] = y(u + w2): the interleaved 1-D window of the forward
//       kernel (8 copies shifted by one sample, 16-byte blocks), read straight
//       by the descriptor (LBO = SBO = 128 bytes) -- never expanded.
//   B = Gs(w1, w2) of one 128-lag block of w1, K-major canonical layout,
//       loaded once per block and kept in shared memory (all K = 2L lags).
//   D = two FP32 TMEM accumulators (128 columns each), so the epilogue drains
//       one item while the MMAs fill the next.
// T2 is summed per warp and 32-column chunk: the products U[u, c] y(u) go to
// shared memory, lane l adds up the chunk's anti-diagonals l and l + 32, and
// the chunk sums accumulate per warp; the four warps' diagonals are then added
// in warp order.  Every sum runs in a fixed order.
//
// Work items (w1 block b, 128-row tile of u), b-major, split into equal
// contiguous ranges over the persistent CTAs.  Every wait is bounded.
//
// Fourth order (the trispectrum adjoint).  With Gs the symmetrised lag-domain
// gradient of c4 and E(u, w1) = sum_{w2,w3} Gs(w1, w2, w3) y(u + w2) y(u + w3),
// the fourth-moment part of the gradient is T1 + 3 T2 with
//   T1(u) = sum_w1 E(u, w1) y(u + w1),   T2(j) = sum_w1 E(j - w1, w1) y(j - w1).
// The same MMA computes D[u, (w1, w2)] = sum_w3 y(u + w3) Gs(w1, w2, w3): the
// B rows are the (w1, w2) combinations, 128 per block, w2 fastest, K = w3.
// The epilogue forms E(u, w1) = sum_w2 D[u, (w1, w2)] y(u + w2) one w1 run at
// a time (a run split between two blocks gives two partial E's, which T1 and
// T2 take linearly) and adds E y(u + w1) to T1 and E y(u) to the warp's T2
// positions u + w1.
#include "launch.cuh"

namespace hos {

namespace {

constexpr int AU = 128;               // rows u per item
constexpr int AW = 128;               // lags w1 per block
constexpr int AMAXK = 256;            // K = 2L <= 256 (L <= 128)
constexpr int AWIN = AU + AMAXK + 16;  // window samples (u0 - L .. u0 + 128 + L + 16)
constexpr int B_BYTES = (AMAXK / 8) * 2048;  // one Gs plane of a block: (K/8) x 16 groups x 128 B
// Item buffers (window, staging, y rows): the producer keeps NBUF - 2 items'
// copies in flight ahead of the one it interleaves, so one item's copy
// latency overlaps the others' work.
constexpr int NBUF = 4;

struct __align__(16) AdjSmem {
    uint8_t gs_hi[B_BYTES];
    uint8_t gs_lo[B_BYTES];
    uint8_t win_hi[NBUF][AWIN * 16];
    uint8_t win_lo[NBUF][AWIN * 16];
    uint16_t lin_hi[NBUF][AWIN + 16];
    uint16_t lin_lo[NBUF][AWIN + 16];
    float yw[NBUF][AU + AW];   // ORDER 3: y(u0 + w1_0 + t), the y(u + w1) of T1; ORDER 4: y(u0 - L + t)
    float yu[NBUF][AU + 4];    // y(u0 + t - sh) from a 16-byte aligned start, sh = L & 3
    float t2w[4][AU / 4 + AW];  // each warp's anti-diagonal sums (private to the warp)
    float pw[4][32 * 33];       // third order: one 32 x 32 chunk of U y(u) per warp, row pitch 33
    uint64_t full[NBUF], empty[NBUF], tma_bar[NBUF], acc_full[2], acc_empty[2], b_full, b_empty, btma_bar, drain;
    uint32_t tmem_base;
    int abort;
};

}  // namespace

struct AdjTcParams {
    const float* y32;       // padded sample planes of the series: y(i) at index L + i
    int t2d;                // floats per warp in t2p: 32 + (w1 values per block) - 1
    const uint16_t* hi;     // bf16 or f16 planes
    const uint16_t* lo;
    const uint8_t* gsb;     // Gs hi/lo planes per block, canonical layout, 2 * B_BYTES per block
    float* t1p;             // [nb][n_round]
    float* t2p;             // [items][4 warps][32 + AW - 1]
    int64_t n;
    int L;
    int kpad;               // 2L rounded up to 16
    int nb;                 // w1 blocks
    int64_t nut;            // u tiles
    int* status;
    uint64_t limit_ns;
};

HOS_DEV void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
HOS_DEV void expect_bytes(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

template <int ORDER, int FMT>
__global__ void __launch_bounds__(192, 1) adjoint_tc_kernel(const AdjTcParams P) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    AdjSmem& sm = *reinterpret_cast<AdjSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = P.L, K = P.kpad;
    const uint32_t idesc = make_idesc(FMT, AU, AW);
    const int64_t items = (int64_t)P.nb * P.nut;
    const int64_t it0 = range_begin(blockIdx.x, items, gridDim.x), it1 = range_begin(blockIdx.x + 1, items, gridDim.x);

    if (threadIdx.x == 0) {
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&sm.full[i], 1);  // one elected arrival per arriving warp
            mbar_init(&sm.empty[i], 1 + 4);  // MMA commit + four epilogue warps
            mbar_init(&sm.tma_bar[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.acc_full[i], 1);
            mbar_init(&sm.acc_empty[i], 4);
        }
        mbar_init(&sm.b_full, 1);
        mbar_init(&sm.b_empty, 1);
        mbar_init(&sm.btma_bar, 1);
        mbar_init(&sm.drain, 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    if (warp == 5) {
        tmem_alloc(&sm.tmem_base, 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int* abort = &sm.abort;
    const uint64_t lim = P.limit_ns;

    if (warp == 4) {
        // ---------------------------------------------------------- producer
        uint32_t bph = 0;
        int cur_b = -1;
        uint32_t nbl = 0;  // blocks loaded
        bool ok = true;
        const int64_t cnt = it1 - it0;
        // items whose copies run ahead; the buffer item k + PD reuses was freed by
        // item k + PD - NBUF = k - 2, so the producer never waits on the item the
        // consumers are working on
        constexpr int PD = NBUF - 2;
        int64_t issued = 0, landed = 0;  // items whose copies were issued / have landed
        bool b_pending = false;          // a Gs block copy issued and not yet waited for
        // copies of item k (into buffer k % NBUF) once the consumers are done with
        // the item that used the buffer before (k - NBUF, already published)
        auto issue = [&](int64_t k) -> bool {
            const int64_t it = it0 + k;
            const int b = (int)(it / P.nut);
            const int64_t u0 = (it % P.nut) * AU;
            const int buf = (int)(k % NBUF);
            if (!warp_wait(&sm.empty[buf], (uint32_t)((k / NBUF) & 1) ^ 1u, abort, P.status, lim, 2000)) return false;
            // window of y(u0 - L + t): plane index u0 (multiple of 128, 16-byte aligned for bf16)
            const uint32_t wsamp = (uint32_t)(AU + K + 16);
            // ORDER 3: yw = y(u0 + w1b + t), w1b the block's first lag (L + u0 + w1b
            // = u0 + 128 b, aligned); ORDER 4: yw = y(u0 - L + t) (plane index u0)
            const int64_t yw0 = (ORDER == 3) ? (L + u0 + (int64_t)b * AW - L) : u0;
            if (lane == 0) {
                expect_bytes(&sm.tma_bar[buf], 2 * wsamp * 2 + (AU + AW) * 4 + (AU + 4) * 4);
                bulk_copy(sm.lin_hi[buf], P.hi + u0, wsamp * 2, &sm.tma_bar[buf]);
                bulk_copy(sm.lin_lo[buf], P.lo + u0, wsamp * 2, &sm.tma_bar[buf]);
                bulk_copy(sm.yw[buf], P.y32 + yw0, (AU + AW) * 4, &sm.tma_bar[buf]);
                bulk_copy(sm.yu[buf], P.y32 + ((L + u0) & ~(int64_t)3), (AU + 4) * 4, &sm.tma_bar[buf]);
            }
            issued = k + 1;
            return true;
        };
        for (int64_t k = 0; k < PD && k < cnt && ok; ++k) ok = issue(k);
        for (int64_t k = 0; k < cnt && ok; ++k) {
            const int b = (int)((it0 + k) / P.nut);
            if (b != cur_b) {  // the Gs block: wait until every MMA on the previous one is done
                ok = warp_wait(&sm.b_empty, (nbl & 1) ^ 1, abort, P.status, lim, 2000);
                if (!ok) break;
                if (lane == 0) {
                    expect_bytes(&sm.btma_bar, 2 * (uint32_t)((K / 8) * 2048));
                    const uint8_t* src = P.gsb + (size_t)b * 2 * B_BYTES;
                    bulk_copy(sm.gs_hi, src, (K / 8) * 2048, &sm.btma_bar);
                    bulk_copy(sm.gs_lo, src + B_BYTES, (K / 8) * 2048, &sm.btma_bar);
                }
                b_pending = true;
                ok = warp_wait(&sm.btma_bar, bph, abort, P.status, lim, 1000);
                if (!ok) break;
                b_pending = false;
                bph ^= 1;
                if (lane == 0) mbar_arrive(&sm.b_full);
                cur_b = b;
                ++nbl;
            }
            const int buf = (int)(k % NBUF);
            ok = warp_wait(&sm.tma_bar[buf], (uint32_t)((k / NBUF) & 1), abort, P.status, lim, 1000);
            if (!ok) break;
            landed = k + 1;
            // interleave: block (q, r) <- samples [8q + r, 8q + r + 8)
            const int nblocks = (int)(((AU + K) / 8 + 2) * 8);
            const uint32_t* sh = reinterpret_cast<const uint32_t*>(sm.lin_hi[buf]);
            const uint32_t* sl = reinterpret_cast<const uint32_t*>(sm.lin_lo[buf]);
            for (int blk = lane; blk < nblocks; blk += 32) {
                const int e0 = blk;  // 8q + r
                const int w0 = e0 >> 1;
                const uint32_t sft = (e0 & 1) * 16;
                uint32_t h[5], l[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    h[q] = sh[w0 + q];
                    l[q] = sl[w0 + q];
                }
                *reinterpret_cast<uint4*>(sm.win_hi[buf] + (size_t)blk * 16) =
                    make_uint4(__funnelshift_r(h[0], h[1], sft), __funnelshift_r(h[1], h[2], sft),
                               __funnelshift_r(h[2], h[3], sft), __funnelshift_r(h[3], h[4], sft));
                *reinterpret_cast<uint4*>(sm.win_lo[buf] + (size_t)blk * 16) =
                    make_uint4(__funnelshift_r(l[0], l[1], sft), __funnelshift_r(l[1], l[2], sft),
                               __funnelshift_r(l[2], l[3], sft), __funnelshift_r(l[3], l[4], sft));
            }
            fence_proxy_async_smem();  // every lane's window writes, for the MMA's reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.full[buf]);
            // after publishing item k: the copies of item k + PD
            if (k + PD < cnt) ok = issue(k + PD);
        }
        // copies issued ahead of a failure still land in this CTA's shared
        // memory: wait for them (bounded, whatever the abort flag says) before
        // the CTA exits
        if (!ok && lane == 0) {
            volatile int keep_waiting = 0;
            for (int64_t k = landed; k < issued; ++k)
                mbar_wait(&sm.tma_bar[k % NBUF], (uint32_t)((k / NBUF) & 1), &keep_waiting, P.status, lim);
            if (b_pending) mbar_wait(&sm.btma_bar, bph, &keep_waiting, P.status, lim);
        }
        __syncwarp();
    } else if (warp == 5 && lane == 0) {
        // ---------------------------------------------------------- MMA issuer
        int cur_b = -1;
        uint32_t nbl = 0;
        bool ok = true;
        const uint32_t wh0 = smem_u32(sm.win_hi[0]), wl0 = smem_u32(sm.win_lo[0]);
        const uint32_t gh = smem_u32(sm.gs_hi), gl = smem_u32(sm.gs_lo);
        for (int64_t it = it0, k = 0; it < it1 && ok; ++it, ++k) {
            const int b = (int)(it / P.nut);
            if (b != cur_b) {
                if (cur_b >= 0) mma_commit(&sm.b_empty);  // MMAs on the previous block are all issued
                ok = mbar_wait(&sm.b_full, nbl & 1, abort, P.status, lim);
                if (!ok) break;
                cur_b = b;
                ++nbl;
            }
            const int buf = (int)(k % NBUF);
            const uint32_t ab = (uint32_t)(k & 1);
            ok = mbar_wait(&sm.acc_empty[ab], ((k >> 1) & 1) ^ 1, abort, P.status, lim);
            if (!ok) break;
            ok = mbar_wait(&sm.full[buf], (uint32_t)((k / NBUF) & 1), abort, P.status, lim);
            if (!ok) break;
            tc_fence_after();
            const uint32_t d = tmem + ab * 128u;
            const uint32_t wh = wh0 + (uint32_t)buf * (AWIN * 16), wl = wl0 + (uint32_t)buf * (AWIN * 16);
            uint32_t acc = 0;
            for (int ks = 0; ks < K / 16; ++ks) {
                // A rows u, K = lags w2 (-L + 16 ks ..): window offset 16 ks samples = 2 groups of 128 B
                const uint64_t ah = make_sdesc(wh + (uint32_t)ks * 256u, 128, 128);
                const uint64_t al = make_sdesc(wl + (uint32_t)ks * 256u, 128, 128);
                // B rows w1 (16 groups of 8 at 128 B), K groups of 8 lags at 2048 B
                const uint64_t bh = make_sdesc(gh + (uint32_t)ks * 4096u, 2048, 128);
                const uint64_t bl = make_sdesc(gl + (uint32_t)ks * 4096u, 2048, 128);
                mma_ss<false>(d, ah, bh, idesc, acc);
                acc = 1;
                mma_ss<false>(d, ah, bl, idesc, 1);
                mma_ss<false>(d, al, bh, idesc, 1);
            }
            mma_commit(&sm.empty[buf]);
            mma_commit(&sm.acc_full[ab]);
        }
        if (ok && cur_b >= 0) mma_commit(&sm.b_empty);
        mma_commit(&sm.drain);
        {   // every MMA must have completed before TMEM is freed, also after an
            // abort: wait whatever the abort flag says, bounded (at least 0.2 s)
            volatile int keep_waiting = 0;
            mbar_wait(&sm.drain, 0, &keep_waiting, P.status, lim > 200000000ull ? lim : 200000000ull);
        }
    } else if (warp < 4) {
        // ---------------------------------------------------------- epilogue
        const int q = warp;                // TMEM lane quadrant
        const int m = q * 32 + lane;       // row u - u0
        const int ysh = L & 3;           // yu was staged from an aligned start
        bool ok = true;
        for (int64_t it = it0, k = 0; it < it1 && ok; ++it, ++k) {
            const int b = (int)(it / P.nut);
            const int64_t ut = it % P.nut, u0 = ut * AU;
            const int buf = (int)(k % NBUF);
            const uint32_t ab = (uint32_t)(k & 1);
            ok = warp_wait(&sm.full[buf], (uint32_t)((k / NBUF) & 1), abort, P.status, lim, 2000);  // this item's windows
            if (!ok) break;
            ok = warp_wait(&sm.acc_full[ab], (k >> 1) & 1, abort, P.status, lim, 5000);
            if (!ok) break;
            tc_fence_after();
            const float yu = sm.yu[buf][ysh + m];
            if constexpr (ORDER == 4) {
                const float* yw = sm.yw[buf] + m;  // yw[t] = y(u - L + t): y(u + w) = yw[w + L]
                float* t2w = sm.t2w[q];
                for (int e = lane; e < P.t2d; e += 32) t2w[e] = 0.f;
                __syncwarp();
                const int twoL = 2 * L;
                const int cb0 = b * AW;  // first (w1, w2) combination of the block
                const int w1i0 = cb0 / twoL;
                int w1i = w1i0, w2i = cb0 - w1i0 * twoL;
                float ev = 0.f, t1 = 0.f;
                auto flush = [&]() {  // end of a w1 run (uniform over the warp)
                    if (w1i < twoL) {      // combinations past (2L)^2 are zero rows of B
                        t1 = fmaf(ev, yw[w1i], t1);
                        t2w[lane + (w1i - w1i0)] += ev * yu;
                    }
                    __syncwarp();
                    ev = 0.f;
                    w2i = 0;
                    ++w1i;
                };
                auto chunk = [&](const uint32_t* v, int c0) {
                    if (w2i + 32 <= twoL) {
                        // the 32 columns lie in one w1 run: fixed offsets from yw + w2i,
                        // four partial sums
                        const float* yq = yw + w2i;
                        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            p0 = fmaf(__uint_as_float(v[j]), yq[j], p0);
                            p1 = fmaf(__uint_as_float(v[j + 1]), yq[j + 1], p1);
                            p2 = fmaf(__uint_as_float(v[j + 2]), yq[j + 2], p2);
                            p3 = fmaf(__uint_as_float(v[j + 3]), yq[j + 3], p3);
                        }
                        ev += (p0 + p1) + (p2 + p3);
                        w2i += 32;
                        if (w2i == twoL || c0 + 32 == AW) flush();
                        return;
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        ev = fmaf(__uint_as_float(v[j]), yw[w2i], ev);
                        if (++w2i == twoL || c0 + j == AW - 1) flush();
                    }
                };
                // two 32-column loads in flight per wait
                for (int c0 = 0; c0 < AW; c0 += 64) {
                    uint32_t v0[32], v1[32];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + ab * 128u + (uint32_t)c0;
                    tmem_ld32(ta, v0);
                    tmem_ld32(ta + 32u, v1);
                    tmem_wait_ld();
                    chunk(v0, c0);
                    chunk(v1, c0 + 32);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.acc_empty[ab]);
                if (u0 + m < P.n) P.t1p[(int64_t)b * (P.nut * AU) + u0 + m] = t1;
                float* dst = P.t2p + (it * 4 + q) * P.t2d;
                for (int e = lane; e < P.t2d; e += 32) dst[e] = t2w[e];
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.empty[buf]);
                continue;
            }
            const float* yw = sm.yw[buf] + m;  // y(u + w1_0 + c)
            float t1 = 0.f;
            float* t2w = sm.t2w[q];
            float* pw = sm.pw[q];
            for (int e = lane; e < AU / 4 + AW; e += 32) t2w[e] = 0.f;
            __syncwarp();
            // per 32-column chunk: T1 per row; the products U[u, c] y(u) go to pw, and
            // lane l then sums anti-diagonals d = l and d = l + 32 of the chunk
            // (row r, column d - r), adding them at t2w[c0 + d]
            auto chunk = [&](const uint32_t* v, int c0) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float uval = __uint_as_float(v[j]);
                    t1 = fmaf(uval, yw[c0 + j], t1);
                    pw[lane * 33 + j] = uval * yu;
                }
                __syncwarp();
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                for (int r = 0; r < 32; r += 2) {
                    // address 32 r + l (+ 32): bank l, no conflicts
                    const float pa = pw[r * 33 + (r <= lane ? lane - r : lane + 32 - r)];
                    const float pb = pw[(r + 1) * 33 + (r + 1 <= lane ? lane - r - 1 : lane + 31 - r)];
                    if (r <= lane) s0 += pa; else s1 += pa;
                    if (r + 1 <= lane) s2 += pb; else s3 += pb;
                }
                t2w[c0 + lane] += s0 + s2;
                t2w[c0 + 32 + lane] += s1 + s3;
                __syncwarp();
            };
            for (int c0 = 0; c0 < AW; c0 += 64) {
                uint32_t v0[32], v1[32];
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + ab * 128u + (uint32_t)c0;
                tmem_ld32(ta, v0);
                tmem_ld32(ta + 32u, v1);
                tmem_wait_ld();
                chunk(v0, c0);
                chunk(v1, c0 + 32);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.acc_empty[ab]);  // this item's accumulator may be reused
            if (u0 + m < P.n) P.t1p[(int64_t)b * (P.nut * AU) + u0 + m] = t1;
            float* dst = P.t2p + (it * 4 + q) * P.t2d;
            for (int e = lane; e < P.t2d; e += 32) dst[e] = t2w[e];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[buf]);  // yu / yw of this buffer are no longer read
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

// Gs hi/lo per block of 128 B rows in the canonical K-major layout the kernel
// reads: byte (n % 8) * 16 + (n / 8) * 128 + (k / 8) * 2048 + (k % 8) * 2 of a
// plane, n = row - block start, k = last lag + L (K = kpad, zero beyond 2L).
// Rows: w1 (third order, nrows = 2L) or (w1, w2) combinations (fourth order,
// nrows = (2L)^2); Gs is row-major with 2L values per row.
template <int FMT>
__global__ void gs_layout_kernel(const float* __restrict__ Gs, int L, int kpad, int nb, int nrows,
                                 const float* __restrict__ gscale, uint8_t* __restrict__ out) {
    const int twoL = 2 * L;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nb * AW * kpad) return;
    const int b = (int)(e / ((int64_t)AW * kpad));
    const int r = (int)(e % ((int64_t)AW * kpad));
    const int n = r / kpad, k = r % kpad;
    const int w1i = b * AW + n;  // index w1 + L
    float v = 0.f;
    if (w1i < nrows && k < twoL) v = Gs[(int64_t)w1i * twoL + k];
    if (gscale) v *= gscale[0];  // a power of two: exact
    const uint32_t hl = pack2<FMT>(v, 0.0f);
    const float hv = unpack2<FMT>(hl).x;
    const uint16_t h = (uint16_t)(hl & 0xFFFFu), l = (uint16_t)(pack2<FMT>(v - hv, 0.0f) & 0xFFFFu);
    const size_t off = (size_t)(n % 8) * 16 + (size_t)(n / 8) * 128 + (size_t)(k / 8) * 2048 + (size_t)(k % 8) * 2;
    uint8_t* base = out + (size_t)b * 2 * B_BYTES;
    *reinterpret_cast<uint16_t*>(base + off) = h;
    *reinterpret_cast<uint16_t*>(base + B_BYTES + off) = l;
}

// g(j) = sum_b T1p[b][j] + (ORDER - 1) sum over the items (b, ut) covering j
// and their four warps (warp w's position d covers item position 32 w + d),
// in the order (b, ut, w); fourth order adds the c2 part
// sum_t gc2(t) (y(j + t) + y(j - t)), t in [-(2L-1), 2L-1].
// R = w1 values per block (AW for third order); a block's first lag is w1b.
// Compensated FP32 sum (TwoSum per addition): FP64 runs at a small fraction
// of the FP32 rate on this part.
struct CSum {
    float hi = 0.f, lo = 0.f;
    __device__ void add(float v) {
        const float s = hi + v;
        const float bv = s - hi;
        lo += (hi - (s - bv)) + (v - bv);
        hi = s;
    }
    __device__ float value() const { return hi + lo; }
};

// Gather: GJ samples j per CTA, GG thread groups per sample splitting the
// blocks b (b = g, g + GG, ...) and the c2 lags; the groups' compensated sums
// are then added in group order.  Third order has at most two blocks: one
// group.
constexpr int GATHER_THREADS = 256;
template <int ORDER>
__host__ __device__ constexpr int gather_groups() { return ORDER == 4 ? 4 : 1; }
// sc: {series scale, Gs scale} of split-FP16 operands (nullptr: unscaled); the
// contraction's sums carry their product, divided out here (exact: powers of two)
template <int ORDER>
__global__ void __launch_bounds__(GATHER_THREADS) adjoint_tc_gather_kernel(
    const float* __restrict__ t1p, const float* __restrict__ t2p, int64_t n, int L, int nb, int64_t nut, int R,
    const double* __restrict__ gc2, const float* __restrict__ y, const float* __restrict__ sc,
    float* __restrict__ g) {
    // fourth order: gc2 as FP32 and the CTA's samples y(j0 - T .. j0 + GJ - 1 + T)
    __shared__ float gcs[ORDER == 4 ? 4 * 64 : 1];
    __shared__ float ys[ORDER == 4 ? GATHER_THREADS / gather_groups<ORDER>() + 4 * 64 : 1];
    __shared__ int w1bs[ORDER == 4 ? 128 : 1];  // first lag of each block (nb <= 128 for L <= 64)
    constexpr int GG = gather_groups<ORDER>(), GJ = GATHER_THREADS / GG;
    __shared__ float2 part[GG][GJ];
    const int jj = threadIdx.x % GJ, grp = threadIdx.x / GJ;
    const int64_t j0 = (int64_t)blockIdx.x * GJ;
    const int64_t j = j0 + jj;
    const int T = 2 * L - 1;
    if constexpr (ORDER == 4) {
        for (int b = threadIdx.x; b < nb; b += GATHER_THREADS) w1bs[b] = (b * AW) / (2 * L) - L;
        for (int i = threadIdx.x; i < 2 * T + 1; i += GATHER_THREADS) gcs[i] = (float)gc2[i];
        for (int i = threadIdx.x; i < GJ + 2 * T; i += GATHER_THREADS) {
            const int64_t a = j0 - T + i;
            ys[i] = (a >= 0 && a < n) ? y[a] : 0.0f;
        }
        __syncthreads();
    }
    const int E = AU + R - 1, D = 32 + R - 1;
    CSum t1, t2, v;
    if (j < n) {
        for (int b = grp; b < nb; b += GG) {
            t1.add(t1p[(int64_t)b * (nut * AU) + j]);
            const int64_t w1b = (ORDER == 3) ? (int64_t)b * AW - L : (int64_t)w1bs[b];
            int64_t lo = j - w1b - (E - 1);
            lo = lo <= 0 ? 0 : ceil_div(lo, AU);
            int64_t hi = (j - w1b) >= 0 ? (j - w1b) / AU : -1;
            if (hi > nut - 1) hi = nut - 1;
            for (int64_t ut = lo; ut <= hi; ++ut) {
                const int64_t e = j - ut * AU - w1b;  // position in the item
                if (e < 0 || e >= E) continue;
                const float* it = t2p + (((int64_t)b * nut + ut) * 4) * D;
                for (int w = 0; w < 4; ++w) {
                    const int64_t d = e - 32 * w;
                    if (d >= 0 && d < D) t2.add(it[w * D + d]);
                }
            }
        }
        const float inv = sc ? 1.0f / (sc[0] * sc[1]) : 1.0f;
        v.add(t1.hi * inv);
        v.add(t1.lo * inv);
        v.add((float)(ORDER - 1) * t2.hi * inv);
        v.add((float)(ORDER - 1) * t2.lo * inv);
        if constexpr (ORDER == 4) {
            const float* yj = ys + T + jj;  // yj[t] = y(j + t), |t| <= T
            for (int t = -T + grp; t <= T; t += GG) v.add(gcs[t + T] * (yj[t] + yj[-t]));
        }
    }
    if constexpr (GG == 1) {
        if (j < n) g[j] = v.value();
        return;
    }
    part[grp][jj] = make_float2(v.hi, v.lo);
    __syncthreads();
    if (grp != 0 || j >= n) return;
    CSum r;
    for (int q = 0; q < GG; ++q) {
        r.add(part[q][jj].x);
        r.add(part[q][jj].y);
    }
    g[j] = r.value();
}

bool adjoint_tc_supported(int L) { return L >= 1 && L <= AMAXK / 2; }
static int adj_rows(int order, int L) { return order == 4 ? 4 * L * L : 2 * L; }
static int adj_nb(int order, int L) { return (adj_rows(order, L) + AW - 1) / AW; }
// w1 values a block of 128 rows touches: all 128 for third order; for fourth
// order at most (AW - 1) / 2L + 2 runs, and never more than 2L
static int adj_r(int order, int L) {
    if (order == 3) return AW;
    const int r = (AW - 1) / (2 * L) + 2;
    return r < 2 * L ? r : 2 * L;
}
size_t adjoint_tc_gs_bytes(int L, int order) { return (size_t)adj_nb(order, L) * 2 * B_BYTES; }
size_t adjoint_tc_t2_floats(int L, int64_t n, int order) {
    return (size_t)adj_nb(order, L) * (size_t)ceil_div(n, AU) * 4 * (size_t)(32 + adj_r(order, L) - 1);
}
size_t adjoint_tc_t1_floats(int L, int64_t n, int order) {
    return (size_t)adj_nb(order, L) * (size_t)ceil_div(n, AU) * AU;
}

template <int ORDER, int FMT>
static cudaError_t launch_adjoint_tc_order(const float* y32, const uint16_t* hi, const uint16_t* lo, int64_t n, int L,
                                           const float* Gs, uint8_t* gsb, float* t1p, float* t2p, const double* gc2,
                                           float* g, int* status, uint64_t limit_ns, int G, const float* sc,
                                           cudaStream_t st) {
    const int kpad = ((2 * L + 15) / 16) * 16;
    const int nb = adj_nb(ORDER, L), R = adj_r(ORDER, L);
    const int64_t nut = ceil_div(n, AU);
    const int64_t tot = (int64_t)nb * AW * kpad;
    gs_layout_kernel<FMT><<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Gs, L, kpad, nb, adj_rows(ORDER, L),
                                                                       sc ? sc + 1 : nullptr, gsb);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    AdjTcParams p{y32, 32 + R - 1, hi, lo, gsb, t1p, t2p, n, L, kpad, nb, nut, status, limit_ns};
    const size_t smem = sizeof(AdjSmem);
    // a per-device (per-context) attribute: set on every launch
    e = cudaFuncSetAttribute(adjoint_tc_kernel<ORDER, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t items = (int64_t)nb * nut;
    const int grid = (int)(items < G ? items : G);
    adjoint_tc_kernel<ORDER, FMT><<<grid, 192, smem, st>>>(p);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_tc_gather_kernel<ORDER><<<(unsigned)ceil_div(n, GATHER_THREADS / gather_groups<ORDER>()), GATHER_THREADS,
                                      0, st>>>(
        t1p, t2p, n, L, nb, nut, R, gc2, y32 + L, sc, g);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_adjoint_tc(const float* y32, const uint16_t* hi, const uint16_t* lo, int64_t n, int L,
                              const float* Gs, uint8_t* gsb, float* t1p, float* t2p, float* g, int* status,
                              uint64_t limit_ns, int G, cudaStream_t st, int fmt, const float* sc) {
    if (fmt == FMT_F16)
        return launch_adjoint_tc_order<3, FMT_F16>(y32, hi, lo, n, L, Gs, gsb, t1p, t2p, nullptr, g, status, limit_ns,
                                                   G, sc, st);
    return launch_adjoint_tc_order<3, FMT_BF16>(y32, hi, lo, n, L, Gs, gsb, t1p, t2p, nullptr, g, status, limit_ns, G,
                                                nullptr, st);
}

cudaError_t launch_adjoint4_tc(const float* y32, const uint16_t* hi, const uint16_t* lo, int64_t n, int L,
                               const float* Gs4, uint8_t* gsb, float* t1p, float* t2p, const double* gc2, float* g,
                               int* status, uint64_t limit_ns, int G, cudaStream_t st, int fmt, const float* sc) {
    if (fmt == FMT_F16)
        return launch_adjoint_tc_order<4, FMT_F16>(y32, hi, lo, n, L, Gs4, gsb, t1p, t2p, gc2, g, status, limit_ns, G,
                                                   sc, st);
    return launch_adjoint_tc_order<4, FMT_BF16>(y32, hi, lo, n, L, Gs4, gsb, t1p, t2p, gc2, g, status, limit_ns, G,
                                                nullptr, st);
}

}  // namespace hos
