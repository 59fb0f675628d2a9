// adjoint_tc.cu -- the adjoint contractions of the bispectrum and trispectrum
// estimators on the tensor cores (tcgen05, split-bf16 or split-FP16 of
// power-of-two scaled operands, FP32 accumulate), with both gradient terms
// taken in the epilogue.
//
// Third order (adjoint3_tm_kernel, below): U[u, w1] = sum_w2 y(u + w2) Gs(w1, w2)
// gives the gradient T1 + 2 T2 with
//   T1(u) = sum_w1 U[u, w1] y(u + w1),   T2(j) = sum_w1 U[j - w1, w1] y(j - w1);
// it runs transposed, Gs resident in tensor memory (its own comment block).
//
// Fourth order (adjoint_tc_kernel<4>, shared-memory operands).  With Gs the
// symmetrised lag-domain gradient of c4 and
// E(u, w1) = sum_{w2,w3} Gs(w1, w2, w3) y(u + w2) y(u + w3), the fourth-moment
// part of the gradient is T1 + 3 T2 with
//   T1(u) = sum_w1 E(u, w1) y(u + w1),   T2(j) = sum_w1 E(j - w1, w1) y(j - w1).
// One MMA (M = 128 rows u, N = 128 combinations (w1, w2) of one block, K = 16
// lags w3) computes D[u, (w1, w2)] = sum_w3 y(u + w3) Gs(w1, w2, w3):
//   A = Hankel X[u, w3] = y(u + w3): the interleaved 1-D window of the forward
//       kernel (8 copies shifted by one sample, 16-byte blocks), read straight
//       by the descriptor (LBO = SBO = 128 bytes) -- never expanded;
//   B = Gs rows of one block of 128 combinations, w2 fastest, K-major
//       canonical layout, loaded once per block and kept in shared memory;
//   D = two FP32 TMEM accumulators (128 columns each), so the epilogue drains
//       one item while the MMAs fill the next.
// The epilogue forms E(u, w1) = sum_w2 D[u, (w1, w2)] y(u + w2) one w1 run at
// a time (a run split between two blocks gives two partial E's, which T1 and
// T2 take linearly) and adds E y(u + w1) to T1 and E y(u) to the warp's T2
// positions u + w1.
//
// Work items (block b, 128-sample tile of u), b-major, split into equal
// contiguous ranges over the persistent CTAs.  Every sum runs in a fixed
// order and every wait is bounded.
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
    float yw[NBUF][AU + AW];   // y(u0 - L + t)
    float yu[NBUF][AU + 4];    // y(u0 + t - sh) from a 16-byte aligned start, sh = L & 3
    float t2w[4][AU / 4 + AW];  // each warp's anti-diagonal sums (private to the warp)
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
    static_assert(ORDER == 4, "third order runs on adjoint3_tm_kernel");
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
            const int64_t u0 = ((it0 + k) % P.nut) * AU;
            const int buf = (int)(k % NBUF);
            if (!warp_wait(&sm.empty[buf], (uint32_t)((k / NBUF) & 1) ^ 1u, abort, P.status, lim, 2000)) return false;
            // window of y(u0 - L + t): plane index u0 (multiple of 128, 16-byte aligned for bf16)
            const uint32_t wsamp = (uint32_t)(AU + K + 16);
            // yw = y(u0 - L + t) (plane index u0)
            const int64_t yw0 = u0;
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

// ---------------------------------------------------------------------------
// Third order with Gs resident in tensor memory.  The same contraction,
// transposed: D[w1, u] = sum_w2 Gs(w1, w2) y(u + w2), M = 128 lags w1 of one
// block, N = 128 samples u of an item, K = 16 lags w2 per step:
//   A = the block's Gs rows (hi and lo), stored into TMEM once per block by
//       the epilogue warps (TMEM lane m holds row w1 = w1b + m);
//   B = the Hankel matrix X[w2, u] = y(u + w2), the same interleaved window
//       read by descriptor (LBO = SBO = 128 bytes);
//   D = two FP32 accumulators of 128 columns.
// Only B is read from shared memory: 4 KB per MMA where the shared-memory
// form reads 8.  TMEM: Gs hi at column 0, lo at 128 (at most 128 columns
// each), accumulators at 256 and 384.
// Eight epilogue warps: warp (q, h) = (warp % 4, warp / 4) takes TMEM lanes
// 32 q .. 32 q + 31 (lags w1b + 32 q + lane) and the 64 columns 64 h ..:
//   T1(u) = sum_w1 D[w1, u] y(u + w1): each lane's products, reduced across
//           the warp by a butterfly per 32-column chunk (lane l ends with the
//           chunk's column l); the four lane quadrants' sums are then added
//           in quadrant order;
//   T2(j) = sum_w1 D[w1, j - w1] y(j - w1): lane r writes its products
//           D[r, c] y(u0 + c) at row r, position r + c of a zero-filled
//           32 x 96 array, so that each position's column sum is one
//           anti-diagonal; lanes read four positions per 16-byte load.  The
//           two column halves' diagonals are added per quadrant.
// Pairs of FP32 products and sums use the packed f32x2 instructions (each
// half rounded as its scalar instruction would be).
// Both results land in the layouts of the shared-memory form (t1p[b][u]; per
// quadrant q a T2 window at item position 32 q + d), so the gather is the
// same.
// ---------------------------------------------------------------------------
namespace {

constexpr int TM_EPI = 8;               // epilogue warps
constexpr int TM_THREADS = 32 * (TM_EPI + 2);
constexpr int YWC = AU + AW + 8;        // pitch of the shifted copies of yw (8 words mod 32)
constexpr int ZW = 96;                  // skewed row width: 64 columns + 31 lane offsets, rounded
constexpr int T2H = ZW;                 // one column half's diagonals
// Each item's sums are added up across warps one item later (so that no warp
// waits for the others right after its own work); a sum buffer is written
// again four items on, when every warp has passed the item that read it.
constexpr int RED = 4;

struct __align__(16) Adj3TmSmem {
    uint8_t win_hi[NBUF][AWIN * 16];
    uint8_t win_lo[NBUF][AWIN * 16];
    uint16_t lin_hi[NBUF][AWIN + 16];
    uint16_t lin_lo[NBUF][AWIN + 16];
    float yw[NBUF][AU + AW];    // staging: y(u0 + w1b + t), the y(u + w1) of T1
    float yu[NBUF][AU + 4];     // staging: y(u0 + t - sh) from a 16-byte aligned start, sh = L & 3
    float ywc[NBUF][4][YWC];    // ywc[s][t] = y(u0 + w1b + t + s): 16-byte loads at any lag
    float yua[NBUF][AU];        // yua[c] = y(u0 + c), 16-byte aligned
    float z[TM_EPI][32 * ZW];   // per warp: row r = lane r's T2 products at positions r .. r + 63, zero elsewhere
    float t2w[RED][4][2][T2H];  // [item % RED][quadrant][column half] anti-diagonal sums
    float t1s[RED][4][AU];      // [item % RED][quadrant] T1 column sums
    uint64_t full[NBUF], empty[NBUF], tma_bar[NBUF], acc_full[2], acc_empty[2], gs_full, gs_empty, t1_bar[RED],
        drain;
    uint32_t tmem_base;
    int abort;
};

// packed pairs: (x0, x1) op (y0, y1), each half rounded to nearest
HOS_DEV void mul2(float& r0, float& r1, float x0, float x1, float y0, float y1) {
    asm("{\n\t.reg .b64 a, b, c;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mul.rn.f32x2 c, a, b;\n\tmov.b64 {%0, %1}, c;\n\t}"
        : "=f"(r0), "=f"(r1)
        : "f"(x0), "f"(x1), "f"(y0), "f"(y1));
}
HOS_DEV void add2(float& s0, float& s1, float x0, float x1) {
    asm("{\n\t.reg .b64 a, b;\n\tmov.b64 a, {%0, %1};\n\tmov.b64 b, {%2, %3};\n\t"
        "add.rn.f32x2 a, a, b;\n\tmov.b64 {%0, %1}, a;\n\t}"
        : "+f"(s0), "+f"(s1)
        : "f"(x0), "f"(x1));
}

}  // namespace

// Gs rows for the TMEM form: per block b and row n (w1 index b * 128 + n), the
// hi plane's kh words then the lo plane's, word w holding lags 2w and 2w + 1
// (index w2 + L) of the row, zero past 2L; kh = 2L rounded up to 64, halved.
template <int FMT>
__global__ void gs_rows_kernel(const float* __restrict__ Gs, int L, int kh, int nb, int nrows,
                               const float* __restrict__ gscale, uint32_t* __restrict__ out) {
    const int twoL = 2 * L;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nb * AW * kh) return;
    const int64_t row = e / kh;  // b * 128 + n
    const int w = (int)(e % kh);
    const int k0 = 2 * w;
    float v0 = 0.f, v1 = 0.f;
    if (row < nrows) {
        if (k0 < twoL) v0 = Gs[row * twoL + k0];
        if (k0 + 1 < twoL) v1 = Gs[row * twoL + k0 + 1];
    }
    if (gscale) {  // a power of two: exact
        v0 *= gscale[0];
        v1 *= gscale[0];
    }
    const uint32_t h = pack2<FMT>(v0, v1);
    const float2 f = unpack2<FMT>(h);
    out[(row * 2) * kh + w] = h;
    out[(row * 2 + 1) * kh + w] = pack2<FMT>(v0 - f.x, v1 - f.y);
}

template <int FMT>
__global__ void __launch_bounds__(TM_THREADS, 1) adjoint3_tm_kernel(const AdjTcParams P) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    Adj3TmSmem& sm = *reinterpret_cast<Adj3TmSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = P.L, K = P.kpad;
    const int kh = ((K + 63) / 64) * 32;  // words (TMEM columns) per Gs plane row
    const uint32_t idesc = make_idesc(FMT, AW, AU);
    const int64_t items = (int64_t)P.nb * P.nut;
    const int64_t it0 = range_begin(blockIdx.x, items, gridDim.x), it1 = range_begin(blockIdx.x + 1, items, gridDim.x);
    // the first item's block and u tile; later ones advance without a division
    const int b_first = (int)(it0 / P.nut);
    const int64_t ut_first = it0 % P.nut;
    constexpr uint32_t GS_LO = 128u, ACC0 = 256u;
    constexpr int PRODUCER = TM_EPI, ISSUER = TM_EPI + 1;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&sm.full[i], 1);            // one elected arrival per arriving warp
            mbar_init(&sm.empty[i], 1 + TM_EPI);  // MMA commit + the epilogue warps
            mbar_init(&sm.tma_bar[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.acc_full[i], 1);
            mbar_init(&sm.acc_empty[i], TM_EPI);
        }
        for (int i = 0; i < RED; ++i) mbar_init(&sm.t1_bar[i], TM_EPI);
        mbar_init(&sm.gs_full, TM_EPI);
        mbar_init(&sm.gs_empty, 1);
        mbar_init(&sm.drain, 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < TM_EPI * 32 * ZW; i += blockDim.x) (&sm.z[0][0])[i] = 0.f;
    if (warp == ISSUER) {
        tmem_alloc(&sm.tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int* abort = &sm.abort;
    const uint64_t lim = P.limit_ns;

    if (warp == PRODUCER) {
        // ---------------------------------------------------------- producer
        bool ok = true;
        const int64_t cnt = it1 - it0;
        const int ysh = L & 3;
        // items whose copies run ahead; the buffer item k + PD reuses was freed by
        // item k + PD - NBUF = k - 2
        constexpr int PD = NBUF - 2;
        int64_t issued = 0, landed = 0;
        int ib = b_first;  // block and u tile of the next item to issue
        int64_t iut = ut_first;
        auto issue = [&](int64_t k) -> bool {
            const int64_t u0 = iut * AU;
            const int buf = (int)(k % NBUF);
            if (!warp_wait(&sm.empty[buf], (uint32_t)((k / NBUF) & 1) ^ 1u, abort, P.status, lim, 2000)) return false;
            // window of y(u0 - L + t) (plane index u0, 16-byte aligned); yw = y(u0 + w1b + t),
            // w1b = 128 b - L (plane index u0 + 128 b); yu from an aligned start
            const uint32_t wsamp = (uint32_t)(AU + K + 16);
            fence_proxy_async_smem();  // this buffer's earlier generic-proxy accesses, before the copies
            __syncwarp();
            if (lane == 0) {
                expect_bytes(&sm.tma_bar[buf], 2 * wsamp * 2 + (AU + AW) * 4 + (AU + 4) * 4);
                bulk_copy(sm.lin_hi[buf], P.hi + u0, wsamp * 2, &sm.tma_bar[buf]);
                bulk_copy(sm.lin_lo[buf], P.lo + u0, wsamp * 2, &sm.tma_bar[buf]);
                bulk_copy(sm.yw[buf], P.y32 + u0 + (int64_t)ib * AW, (AU + AW) * 4, &sm.tma_bar[buf]);
                bulk_copy(sm.yu[buf], P.y32 + ((L + u0) & ~(int64_t)3), (AU + 4) * 4, &sm.tma_bar[buf]);
            }
            issued = k + 1;
            if (++iut == P.nut) {
                iut = 0;
                ++ib;
            }
            return true;
        };
        for (int64_t k = 0; k < PD && k < cnt && ok; ++k) ok = issue(k);
        for (int64_t k = 0; k < cnt && ok; ++k) {
            const int buf = (int)(k % NBUF);
            ok = warp_wait(&sm.tma_bar[buf], (uint32_t)((k / NBUF) & 1), abort, P.status, lim, 1000);
            if (!ok) break;
            landed = k + 1;
            // interleave: block (q, r) <- samples [8q + r, 8q + r + 8)
            const int nblocks = (int)(((AU + K) / 8 + 2) * 8);
            const uint32_t* sh = reinterpret_cast<const uint32_t*>(sm.lin_hi[buf]);
            const uint32_t* sl = reinterpret_cast<const uint32_t*>(sm.lin_lo[buf]);
            for (int blk = lane; blk < nblocks; blk += 32) {
                const int w0 = blk >> 1;
                const uint32_t sft = (blk & 1) * 16;
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
            // the epilogue's operands: four shifted copies of yw (the last group of
            // copy s reads up to s words past yw, inside the buffer; those land at
            // t + s >= AU + AW, which no lane reads) and y(u0 + c) aligned
            {
                const float* y0 = sm.yw[buf];
                for (int g = lane; g < (AU + AW) / 4; g += 32) {
                    const float4 u = *reinterpret_cast<const float4*>(y0 + 4 * g);
                    const float4 v = (g + 1 < (AU + AW) / 4) ? *reinterpret_cast<const float4*>(y0 + 4 * g + 4)
                                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                    *reinterpret_cast<float4*>(sm.ywc[buf][0] + 4 * g) = u;
                    *reinterpret_cast<float4*>(sm.ywc[buf][1] + 4 * g) = make_float4(u.y, u.z, u.w, v.x);
                    *reinterpret_cast<float4*>(sm.ywc[buf][2] + 4 * g) = make_float4(u.z, u.w, v.x, v.y);
                    *reinterpret_cast<float4*>(sm.ywc[buf][3] + 4 * g) = make_float4(u.w, v.x, v.y, v.z);
                }
                for (int t = lane; t < AU; t += 32) sm.yua[buf][t] = sm.yu[buf][ysh + t];
            }
            fence_proxy_async_smem();  // every lane's window writes, for the MMA's reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.full[buf]);
            if (k + PD < cnt) ok = issue(k + PD);
        }
        // copies issued ahead of a failure still land in this CTA's shared memory:
        // wait for them (bounded, whatever the abort flag says) before the CTA exits
        if (!ok && lane == 0) {
            volatile int keep_waiting = 0;
            for (int64_t k = landed; k < issued; ++k)
                mbar_wait(&sm.tma_bar[k % NBUF], (uint32_t)((k / NBUF) & 1), &keep_waiting, P.status, lim);
        }
        __syncwarp();
    } else if (warp == ISSUER && lane == 0) {
        // ---------------------------------------------------------- MMA issuer
        int cur_b = -1, b = b_first;
        int64_t ut = ut_first;
        uint32_t nbl = 0;
        bool ok = true;
        const uint32_t wh0 = smem_u32(sm.win_hi[0]), wl0 = smem_u32(sm.win_lo[0]);
        for (int64_t k = 0; k < it1 - it0 && ok; ++k) {
            if (b != cur_b) {
                // the previous block's MMAs are all issued: their completion frees Gs
                if (cur_b >= 0) mma_commit(&sm.gs_empty);
                ok = mbar_wait(&sm.gs_full, nbl & 1, abort, P.status, lim);
                if (!ok) break;
                tc_fence_after();
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
            const uint32_t d = tmem + ACC0 + ab * 128u;
            const uint32_t wh = wh0 + (uint32_t)buf * (AWIN * 16), wl = wl0 + (uint32_t)buf * (AWIN * 16);
            uint32_t acc = 0;
            for (int ks = 0; ks < K / 16; ++ks) {
                // K = lags w2 (-L + 16 ks ..): window offset 16 ks samples = 2 groups of 128 B
                const uint64_t bh = make_sdesc(wh + (uint32_t)ks * 256u, 128, 128);
                const uint64_t bl = make_sdesc(wl + (uint32_t)ks * 256u, 128, 128);
                const uint32_t ah = tmem + (uint32_t)ks * 8u;  // 16 lags = 8 packed columns
                mma_ts<false>(d, ah, bh, idesc, acc);
                acc = 1;
                mma_ts<false>(d, ah, bl, idesc, 1);
                mma_ts<false>(d, ah + GS_LO, bh, idesc, 1);
            }
            mma_commit(&sm.empty[buf]);
            mma_commit(&sm.acc_full[ab]);
            if (++ut == P.nut) {
                ut = 0;
                ++b;
            }
        }
        mma_commit(&sm.drain);
        {   // every MMA must have completed before TMEM is freed, also after an
            // abort: wait whatever the abort flag says, bounded (at least 0.2 s)
            volatile int keep_waiting = 0;
            mbar_wait(&sm.drain, 0, &keep_waiting, P.status, lim > 200000000ull ? lim : 200000000ull);
        }
    } else if (warp < TM_EPI) {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;       // TMEM lane quadrant
        const int hf = warp >> 2;     // column half
        const int m = q * 32 + lane;  // row: lag w1 = w1b + m
        const int cb = 64 * hf;       // first column
        const uint32_t lrow = (uint32_t)(q * 32) << 16;
        float* zr = sm.z[warp] + lane * (ZW + 1);  // this lane's row, shifted by the lane
        const float* zc = sm.z[warp] + 4 * lane;   // positions 4 lane .. 4 lane + 3 of row 0
        int cur_b = -1, b = b_first;
        int64_t ut = ut_first;
        uint32_t nbl = 0;
        bool ok = true;
        // the cross-warp sums of item k (block bk, first sample u0k): T1 of columns
        // 32 q + 16 hf .. + 15 (the four quadrants added in order) and quadrant q's
        // T2 window entries [80 hf, 80 hf + 80) (half 1 starts 64 positions later)
        auto finish = [&](int64_t k, int bk, int64_t u0k) -> bool {
            const int sl = (int)(k % RED);
            if (!warp_wait(&sm.t1_bar[sl], (uint32_t)((k / RED) & 1), abort, P.status, lim, 200)) return false;
            if (lane < 16) {
                const int c = 32 * q + 16 * hf + lane;
                const float t1 = ((sm.t1s[sl][0][c] + sm.t1s[sl][1][c]) + sm.t1s[sl][2][c]) + sm.t1s[sl][3][c];
                if (u0k + c < P.n) P.t1p[(int64_t)bk * (P.nut * AU) + u0k + c] = t1;
            }
            const float* h0 = sm.t2w[sl][q][0];
            const float* h1 = sm.t2w[sl][q][1];
            float* dst = P.t2p + ((it0 + k) * 4 + q) * P.t2d;
            const int e1 = (80 * hf + 80 < P.t2d) ? 80 * hf + 80 : P.t2d;
            for (int e = 80 * hf + lane; e < e1; e += 32) {
                const float x0 = e < T2H ? h0[e] : 0.f;
                const float x1 = e >= 64 ? h1[e - 64] : 0.f;
                dst[e] = x0 + x1;
            }
            return true;
        };
        int prev_b = 0;
        int64_t prev_u0 = 0;
        for (int64_t k = 0; k < it1 - it0 && ok; ++k) {
            const int64_t u0 = ut * AU;
            if (b != cur_b) {
                // a new block: once every MMA on the previous one has completed, store
                // row m of its Gs into TMEM lane m (column half hf: plane hf)
                ok = warp_wait(&sm.gs_empty, (nbl & 1) ^ 1, abort, P.status, lim, 2000);
                if (!ok) break;
                tc_fence_after();
                const uint4* src =
                    reinterpret_cast<const uint4*>(P.gsb) + (((size_t)b * AW + m) * 2 + hf) * (size_t)(kh / 4);
                for (int c = 0; c < kh; c += 32) {
                    uint32_t v[32];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint4 w = src[c / 4 + i];
                        v[4 * i] = w.x;
                        v[4 * i + 1] = w.y;
                        v[4 * i + 2] = w.z;
                        v[4 * i + 3] = w.w;
                    }
                    tmem_st32(tmem + lrow + (uint32_t)hf * GS_LO + (uint32_t)c, v);
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.gs_full);
                cur_b = b;
                ++nbl;
            }
            const int buf = (int)(k % NBUF);
            const uint32_t ab = (uint32_t)(k & 1);
            const int sl = (int)(k % RED);
            ok = warp_wait(&sm.full[buf], (uint32_t)((k / NBUF) & 1), abort, P.status, lim, 2000);  // this item's windows
            if (!ok) break;
            ok = warp_wait(&sm.acc_full[ab], (k >> 1) & 1, abort, P.status, lim, 5000);
            if (!ok) break;
            tc_fence_after();
            uint32_t v0[32], v1[32];
            tmem_ld32(tmem + lrow + ACC0 + ab * 128u + (uint32_t)cb, v0);
            tmem_ld32(tmem + lrow + ACC0 + ab * 128u + (uint32_t)cb + 32u, v1);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.acc_empty[ab]);  // this warp's columns are read
            // T1 products D y(u + w1) into a0 / a1 (yw[c] = y(u0 + cb + c + w1), from the copy
            // that puts it on a 16-byte boundary); T2 products D y(u) into this lane's row
            float a0[32], a1[32];
            {
                const float* yw = sm.ywc[buf][m & 3] + (m & ~3) + cb;
                const float* yu = sm.yua[buf] + cb;
#pragma unroll
                for (int g = 0; g < 16; ++g) {
                    const float4 w4 = *reinterpret_cast<const float4*>(yw + 4 * g);
                    const float4 u4 = *reinterpret_cast<const float4*>(yu + 4 * g);
                    const uint32_t* v = g < 8 ? v0 + 4 * g : v1 + 4 * (g - 8);
                    float* a = g < 8 ? a0 + 4 * g : a1 + 4 * (g - 8);
                    const float d0 = __uint_as_float(v[0]), d1 = __uint_as_float(v[1]);
                    const float d2 = __uint_as_float(v[2]), d3 = __uint_as_float(v[3]);
                    mul2(a[0], a[1], d0, d1, w4.x, w4.y);
                    mul2(a[2], a[3], d2, d3, w4.z, w4.w);
                    float p0, p1, p2, p3;
                    mul2(p0, p1, d0, d1, u4.x, u4.y);
                    mul2(p2, p3, d2, d3, u4.z, u4.w);
                    zr[4 * g] = p0;
                    zr[4 * g + 1] = p1;
                    zr[4 * g + 2] = p2;
                    zr[4 * g + 3] = p3;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[buf]);  // this buffer's y copies are no longer read
            // butterflies over the lanes (both chunks, independent chains): after the
            // step of width s, lane l keeps the half of the columns whose bit s matches its own
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const bool up = (lane & s) != 0;
#pragma unroll
                for (int i = 0; i < s; ++i) {
                    const float x0 = up ? a0[i] : a0[i + s], k0 = up ? a0[i + s] : a0[i];
                    const float x1 = up ? a1[i] : a1[i + s], k1 = up ? a1[i + s] : a1[i];
                    a0[i] = k0 + __shfl_xor_sync(0xffffffffu, x0, s);
                    a1[i] = k1 + __shfl_xor_sync(0xffffffffu, x1, s);
                }
            }
            sm.t1s[sl][q][cb + lane] = a0[0];       // columns cb + lane and cb + 32 + lane,
            sm.t1s[sl][q][cb + 32 + lane] = a1[0];  // summed over the warp's 32 lags
            // anti-diagonals: lane l < 24 sums positions 4 l .. 4 l + 3 over the 32 rows
            if (lane < ZW / 4) {
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 8
                for (int r = 0; r < 32; ++r) {
                    const float4 z4 = *reinterpret_cast<const float4*>(zc + r * ZW);
                    add2(s0, s1, z4.x, z4.y);
                    add2(s2, s3, z4.z, z4.w);
                }
                *reinterpret_cast<float4*>(&sm.t2w[sl][q][hf][4 * lane]) = make_float4(s0, s1, s2, s3);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.t1_bar[sl]);  // this warp's sums of item k are in shared memory
            // the previous item's cross-warp sums
            if (k > 0) {
                ok = finish(k - 1, prev_b, prev_u0);
                if (!ok) break;
            }
            prev_b = b;
            prev_u0 = u0;
            if (++ut == P.nut) {
                ut = 0;
                ++b;
            }
        }
        if (ok && it1 > it0) ok = finish(it1 - it0 - 1, prev_b, prev_u0);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == ISSUER) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 512);
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

// third order, Gs in tensor memory
template <int FMT>
static cudaError_t launch_adjoint3_tm(const float* y32, const uint16_t* hi, const uint16_t* lo, int64_t n, int L,
                                      const float* Gs, uint8_t* gsb, float* t1p, float* t2p, float* g, int* status,
                                      uint64_t limit_ns, int G, const float* sc, cudaStream_t st) {
    const int kpad = ((2 * L + 15) / 16) * 16;
    const int kh = ((kpad + 63) / 64) * 32;
    const int nb = adj_nb(3, L);
    const int64_t nut = ceil_div(n, AU);
    const int64_t tot = (int64_t)nb * AW * kh;
    gs_rows_kernel<FMT><<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Gs, L, kh, nb, adj_rows(3, L),
                                                                     sc ? sc + 1 : nullptr,
                                                                     reinterpret_cast<uint32_t*>(gsb));
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    AdjTcParams p{y32, 32 + AW - 1, hi, lo, gsb, t1p, t2p, n, L, kpad, nb, nut, status, limit_ns};
    // at least 116 KB, so that one CTA (and one 512-column TMEM allocation) lands on each SM
    const size_t smem = sizeof(Adj3TmSmem) > 118784 ? sizeof(Adj3TmSmem) : 118784;
    e = cudaFuncSetAttribute(adjoint3_tm_kernel<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t items = (int64_t)nb * nut;
    const int grid = (int)(items < G ? items : G);
    adjoint3_tm_kernel<FMT><<<grid, TM_THREADS, smem, st>>>(p);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_tc_gather_kernel<3><<<(unsigned)ceil_div(n, GATHER_THREADS), GATHER_THREADS, 0, st>>>(
        t1p, t2p, n, L, nb, nut, AW, nullptr, y32 + L, sc, g);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_adjoint_tc(const float* y32, const uint16_t* hi, const uint16_t* lo, int64_t n, int L,
                              const float* Gs, uint8_t* gsb, float* t1p, float* t2p, float* g, int* status,
                              uint64_t limit_ns, int G, cudaStream_t st, int fmt, const float* sc) {
    if (fmt == FMT_F16)
        return launch_adjoint3_tm<FMT_F16>(y32, hi, lo, n, L, Gs, gsb, t1p, t2p, g, status, limit_ns, G, sc, st);
    return launch_adjoint3_tm<FMT_BF16>(y32, hi, lo, n, L, Gs, gsb, t1p, t2p, g, status, limit_ns, G, nullptr, st);
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
