// hos_internal.cuh -- shared definitions of the sm_103a kernels and the host
// runtime: geometry of the lag tiles, the stream-K work split, workspace
// layout, PTX wrappers (mbarrier, tcgen05, TMEM) and bounded waits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hos.h"

#define HOS_DEV __device__ __forceinline__
#define HOS_HD __host__ __device__ __forceinline__

namespace hos {

// ---------------------------------------------------------------------------
// Geometry of the c3 contraction.
//
// The lag square [-L, L-1]^2 (lag index i = w1 + L, j = w2 + L) is cut into
// row blocks of TILE_M (=128) lags w1.  Because c3(w1,w2) = c3(w2,w1), row
// block a computes only the columns j >= row_c0[a] = 128a (from its own
// diagonal block on); the reduction fills the rest from the mirror.  Each row
// block's column range is cut into tiles of at most tile_n (the widest, 256)
// columns; the last tile of a row is narrower (a multiple of 32 columns).  At
// L = 256 the four row blocks have 512, 384, 256 and 128 columns: 1280 columns
// of 128 rows against the 1536 of whole 256-wide tiles.
//
// Work unit = (series, tile, chunk of kc samples of the time index i), ordered
// series-major, then tile, then chunk.  A unit's cost is its tile's width in
// 32-column steps (tile_w32), the MMA work it carries.  The G persistent CTAs
// take contiguous, equal ranges of the cost axis (stream-K weighted by cost):
// CTA g runs the units whose cost interval starts inside its range.  Within a
// range, a CTA accumulates consecutive chunks of one (series, tile) in FP32, at
// most `flush` chunks, then writes one FP32 partial tile ("part") to a slot.
// Slots: one per (series, tile, flush-window) -- the part that starts at the
// window's first chunk -- plus one per CTA for a part that starts at the
// CTA's first unit inside a window.  The FP64-class reduction sums, in a fixed
// order, the main slot and the CTA slots of every window.
// ---------------------------------------------------------------------------
constexpr int TILE_M = 128;
constexpr int KC = 1024;         // most samples per chunk (shared-memory sizing); plans use geo.kc <= KC
constexpr int MAX_TILES_M = 16;  // L <= 1024
constexpr int MAX_TILES = 256;   // tiles of one plan

struct C3Geom {
    int L;
    int kc;         // samples per chunk (multiple of 64, <= KC)
    int tile_n;     // widest tile, 32..256, power of two (the TMEM accumulator width)
    int tiles_m;    // row blocks: ceil(2L / 128)
    int ntiles;     // tiles computed (after the symmetric and zero-window skips)
    int ktot;       // cost of one chunk of every tile: sum of tile_w32
    int flush;      // chunks per flush window
    int G;          // CTAs of the contraction
    int pad_tail;   // zero samples after the last chunk of a series
    int sym;        // lag set: 0 rows w1 in [-L, L) with the swap (w2, w1) (C3_SWAP);
                    // 1 or 2 the six-fold fundamental set (C3_SIX, C3_SIX_BAND)
    uint16_t row_c0[MAX_TILES_M];    // first column (lag index) computed in row block a
    uint8_t row_t0[MAX_TILES_M];     // first tile of row block a (its tiles are consecutive)
    uint8_t tile_a[MAX_TILES];       // row block of tile t
    uint8_t tile_c32[MAX_TILES];     // first column of tile t / 32
    uint8_t tile_w32[MAX_TILES];     // width of tile t / 32 (cost of one of its chunks)
    uint16_t tile_kpre[MAX_TILES + 1];  // sum of tile_w32 over the tiles before t
};

// Per-series layout produced on the device by the plan kernel.
//   off[S+1]  : input offsets
//   pad[S+1]  : start of each series' zero-padded block in the sample planes;
//               sample i of series s sits at pad[s] + L + i
//   unit[S+1] : prefix of work-unit cost  (ktot * nchunks(s))
//   win[S+1]  : prefix of flush windows (ntiles * ceil(nchunks(s) / flush))
//   mean[S]   : FP64 mean removed from each series
//   scale[S]  : power-of-two scale of each series' FP16 planes (nullptr: 1)
struct SeriesView {
    const int64_t* off;
    const int64_t* pad;
    const int64_t* unit;
    const int64_t* win;
    const double* mean;
    int S;
    const float* scale = nullptr;
};

// Operand formats of the tensor-core contraction.
enum { FMT_BF16 = 0, FMT_F16 = 1, FMT_TF32 = 2 };

HOS_HD int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
HOS_HD int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// first cost position of CTA g (ranges [range_begin(g), range_begin(g+1)))
HOS_HD int64_t range_begin(int64_t g, int64_t U, int64_t G) { return (g * U) / G; }

// One series' share of the plan: its padded block length in the sample
// planes (L zeros, the chunks, pad_tail zeros, rounded to 64 samples), the
// cost of its work units and its flush windows over all tiles.
struct SeriesPlan {
    int64_t plen, cost, wins;
};
HOS_HD SeriesPlan series_plan(int64_t len, int L, int ntiles, int ktot, int flush, int kc, int pad_tail) {
    const int64_t nch = ceil_div(len, kc);
    SeriesPlan r;
    r.plen = round_up((int64_t)L + nch * kc + pad_tail, 64);
    r.cost = (int64_t)ktot * nch;
    r.wins = (int64_t)ntiles * ceil_div(nch, flush);
    return r;
}

// Deterministic walk of one CTA's cost range, split into parts at (series,
// tile) boundaries and at flush-window boundaries.
struct Part {
    int s;           // series
    int t;           // computed-tile index
    int64_t c0, c1;  // chunk range [c0, c1) of the series
    int64_t slot;    // partial slot
};

struct Walk {
    int64_t u, ue, U, total_win;  // u: cost position from which the next unit may start
    int s, S, g;
    int flush, ntiles, kc;
    const int64_t* unit;
    const int64_t* win;
    const int64_t* off;
    const C3Geom* geo;

    HOS_HD void init(const C3Geom& geom, const SeriesView& sv, int gidx, int G) {
        geo = &geom;
        S = sv.S;
        unit = sv.unit;
        win = sv.win;
        off = sv.off;
        flush = geom.flush;
        ntiles = geom.ntiles;
        kc = geom.kc;
        g = gidx;
        U = unit[S];
        total_win = win[S];
        u = range_begin(gidx, U, G);
        ue = range_begin(gidx + 1, U, G);
        // series containing u: last s with unit[s] <= u
        int lo = 0, hi = S;  // invariant unit[lo] <= u < unit[hi] (when u < U)
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (unit[mid] <= u) lo = mid; else hi = mid;
        }
        s = lo;
    }
    HOS_HD bool next(Part& p) {
        for (;;) {
            if (u >= ue) return false;
            while (s < S - 1 && unit[s + 1] <= u) ++s;
            if (u >= unit[s + 1]) return false;  // past the last unit
            const int64_t len = off[s + 1] - off[s];
            const int64_t nch = ceil_div(len, kc);
            const int64_t r = u - unit[s];
            int t = 0;  // last tile whose cost range starts at or before r
            while (t + 1 < ntiles && nch * geo->tile_kpre[t + 1] <= r) ++t;
            const int64_t k = geo->tile_w32[t];
            const int64_t tb = unit[s] + nch * geo->tile_kpre[t];  // cost start of (s, t)
            const int64_t c = ceil_div(u - tb, k);                 // first chunk starting at or after u
            if (c >= nch) {  // u inside the tile's last chunk: go on at the next tile
                u = tb + nch * k;
                continue;
            }
            if (tb + c * k >= ue) return false;
            const int64_t f = c / flush;
            const int64_t wend = ((f + 1) * flush < nch) ? (f + 1) * flush : nch;
            const int64_t cap = ceil_div(ue - tb, k);  // chunks of this tile starting before ue
            const int64_t c1 = wend < cap ? wend : cap;
            const int64_t nwin = ceil_div(nch, flush);
            p.s = s;
            p.t = t;
            p.c0 = c;
            p.c1 = c1;
            p.slot = (c % flush == 0) ? (win[s] + (int64_t)t * nwin + f) : (total_win + g);
            u = tb + c1 * k;
            return true;
        }
    }
};

// ---------------------------------------------------------------------------
// Workspace layout (all offsets 256-byte aligned), computed on the host.
// ---------------------------------------------------------------------------
struct WsLayout {
    size_t status;      // int32 status word (+ pad)
    size_t ser;         // 4*(S+1) int64 + S double
    size_t planes_f32;  // y as float (A-operand source, SIMT path)
    size_t plane_hi;    // hi plane (bf16 or tf32-rounded f32)
    size_t plane_lo;    // lo plane
    size_t partials;    // FP32 partial tiles
    size_t grid;        // real transform input / lag-domain scratch
    size_t cplx;        // complex scratch (backward)
    size_t misc;        // small arrays: twiddles, c2, T1/T2, gs
    size_t total;
    int64_t plane_len;  // samples per plane (all series, padded)
    int64_t n_slots;    // partial slots
};

// ---------------------------------------------------------------------------
// Device status word and bounded waits.
// ---------------------------------------------------------------------------
HOS_DEV uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

HOS_DEV void record_status(int* status, int code) { atomicCAS(status, 0, code); }

HOS_DEV uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

HOS_DEV void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

HOS_DEV void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

HOS_DEV void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

// Test the phase; the thread may be suspended up to hint_ns waiting for it.
HOS_DEV bool mbar_try(uint64_t* bar, uint32_t parity, uint32_t hint_ns = 0) {
    uint32_t ok;
    if (hint_ns) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    }
    return ok != 0;
}

// Test the phase without suspending the thread.
HOS_DEV bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// hint_ns of a wait that polls with test_wait and never suspends
constexpr uint32_t WAIT_SPIN = 0xFFFFFFFFu;

// Wait for the phase with the given parity to complete.  Gives up (returning
// false) when another thread of the CTA has raised `abort`, or after
// `limit_ns` nanoseconds, in which case it raises `abort` and records
// HOS_ERR_TIMEOUT in the device status word.  hint_ns: 0 lets try_wait
// suspend the thread for the system's own time limit, WAIT_SPIN polls with
// test_wait (no suspension), other values are try_wait's suspend-time hint.
HOS_DEV bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status, uint64_t limit_ns,
                       uint32_t hint_ns = 0) {
    if (hint_ns == WAIT_SPIN ? mbar_test(bar, parity) : mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        if (hint_ns == WAIT_SPIN ? mbar_test(bar, parity) : mbar_try(bar, parity, hint_ns)) return true;
        if ((it & 7u) == 0) {
            if (*abort) return false;
            if (global_timer_ns() - t0 > limit_ns) {
                *abort = 1;
                record_status(status, HOS_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

// Warp-wide wait: lane 0 polls, the warp then synchronises (which orders the
// memory the barrier protects for every lane) and shares the outcome.
HOS_DEV bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status, uint64_t limit_ns,
                       uint32_t hint_ns = 0) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort, status, limit_ns, hint_ns);
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

HOS_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// tcgen05 / TMEM wrappers (cta_group::1).
// ---------------------------------------------------------------------------
HOS_DEV void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
HOS_DEV void tmem_relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
HOS_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
HOS_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
HOS_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f16 or kind::tf32
template <bool TF32>
HOS_DEV void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc, uint32_t accumulate) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// D[tmem] (+)= A[smem] * B[smem]^T
template <bool TF32>
HOS_DEV void mma_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc, uint32_t accumulate) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// Arrive on an mbarrier when every tcgen05 operation issued so far by this
// thread has completed.
HOS_DEV void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Instruction descriptor: FP32 accumulate, A and B K-major, M = 128.
//   bits 4-5 D format (1 = F32); 7-9 A format; 10-12 B format
//   (kind::f16: 0 = F16, 1 = BF16; kind::tf32: 2 = TF32); 17-22 N>>3; 24-28 M>>4.
HOS_HD uint32_t make_idesc(int fmt_kind, int M, int N) {
    const uint32_t fmt = fmt_kind == FMT_TF32 ? 2u : (fmt_kind == FMT_BF16 ? 1u : 0u);
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle, K-major:
//   bits 0-13 start >> 4; 16-29 leading (K-direction) core-matrix stride >> 4;
//   32-45 stride (M/N-direction, 8-row group) >> 4; 46-47 version = 1.
HOS_DEV uint64_t make_sdesc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// 32 lanes x 32 bits, 32 consecutive columns: thread t <-> lane (base + t).
HOS_DEV void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}
HOS_DEV void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

HOS_DEV void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}
HOS_DEV void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// bf16x2 pack, round to nearest even; `lo` goes to the low half.
HOS_DEV uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
// f16x2 pack, round to nearest even; `lo` goes to the low half.
HOS_DEV uint32_t pack_f16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
// The two halves of a packed pair as floats (exact: every f16 and bf16 value is a float).
template <int FMT>
HOS_DEV float2 unpack2(uint32_t v) {
    if constexpr (FMT == FMT_BF16) {
        return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xFFFF0000u));
    } else {
        float a, b;
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
            : "=f"(a), "=f"(b)
            : "r"(v));
        return make_float2(a, b);
    }
}
template <int FMT>
HOS_DEV uint32_t pack2(float lo, float hi) {
    if constexpr (FMT == FMT_BF16) return pack_bf16x2(lo, hi);
    else return pack_f16x2(lo, hi);
}
// tf32 rounding (nearest, ties away), result as an f32 bit pattern
HOS_DEV uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Parzen lag window in double (u = |w| / L).
HOS_HD double parzen(int w, int L) {
    double u = (w < 0 ? -w : w) / (double)L;
    if (u <= 0.5) return 1.0 - 6.0 * u * u + 6.0 * u * u * u;
    if (u <= 1.0) {
        double v = 1.0 - u;
        return 2.0 * v * v * v;
    }
    return 0.0;
}
HOS_HD double lag_window2(int w1, int w2, int L, int kind) {
    if (kind == HOS_WIN_PARZEN) return parzen(w1, L) * parzen(w2, L);
    if (kind == HOS_WIN_PARZEN_SYM) return parzen(w1, L) * parzen(w2, L) * parzen(w1 - w2, L);
    return 1.0;  // RECT: every computed lag has |w| <= L-1 except w = -L
}
HOS_HD double lag_window3(int w1, int w2, int w3, int L, int kind) {
    if (kind == HOS_WIN_PARZEN) return parzen(w1, L) * parzen(w2, L) * parzen(w3, L);
    return 1.0;
}
// RECT excludes the row/column w = -L that the 2L-wide lag range carries.
HOS_HD bool rect_excluded(int w, int L) { return w == -L; }

// ---------------------------------------------------------------------------
// Lag symmetry of the third-order sample cumulant.  With y zero outside the
// series (or part), c3(w1, w2) = (1/n) sum_i y(i) y(i+w1) y(i+w2) is a sum over
// every integer i, so c3(w1, w2) = c3(w2, w1) (swap the factors) and
// c3(w1, w2) = c3(-w1, w2 - w1) (shift i by w1): six lag pairs per value.
// A time slice's partial sum (i over the slice only) keeps the swap but not
// the shift.
// ---------------------------------------------------------------------------
enum { C3_SWAP = 0, C3_SIX = 1, C3_SIX_BAND = 2 };

// The six lag pairs with the value of c3(w1, w2) (some coincide on the lines
// w1 = 0, w2 = 0 and w1 = w2).
HOS_HD void c3_orbit(int w1, int w2, int (&o1)[6], int (&o2)[6]) {
    o1[0] = w1;      o2[0] = w2;
    o1[1] = w2;      o2[1] = w1;
    o1[2] = -w1;     o2[2] = w2 - w1;
    o1[3] = w2 - w1; o2[3] = -w1;
    o1[4] = -w2;     o2[4] = w1 - w2;
    o1[5] = w1 - w2; o2[5] = -w2;
}

// The fundamental set the six-fold plans compute: w1 in [0, L) and w2 in
// [w1, w1 + L).  Every lag pair of (-L, L)^2 has exactly one of its six images
// in it.  C3_SIX_BAND (a window that also vanishes for |w1 - w2| >= L, which
// is constant on the six images) keeps only w2 < L: the other pairs' values
// are weighted by zero wherever they land.
HOS_HD bool c3_fundamental(int L, int sym, int w1, int w2) {
    return w1 >= 0 && w1 < L && w2 >= w1 && w2 < (sym == C3_SIX_BAND ? L : w1 + L);
}

}  // namespace hos
