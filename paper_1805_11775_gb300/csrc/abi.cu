// abi.cu -- the C ABI (include/hos.h): argument validation, tile geometry,
// workspace carving, and the stream-ordered launch sequence of each entry
// point.  No device memory is allocated here: every buffer is carved from the
// caller's workspace.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.cuh"

namespace hos {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static const char* g_last_contraction = "none";
static char g_last_plan[160] = "none";

// Records the contraction plan of the last call (hos_last_plan).
static void note_plan(const C3Geom& g, int products) {
    int w256 = 0, wmin = 1 << 30;
    for (int t = 0; t < g.ntiles; ++t) {
        const int w = 32 * g.tile_w32[t];
        if (w == 256) ++w256;
        if (w < wmin) wmin = w;
    }
    // cols: the tiles' widths added up (each tile has 128 rows)
    snprintf(g_last_plan, sizeof(g_last_plan),
             "tile_n=%d tiles=%d cols=%d (256-wide %d, narrowest %d) flush=%d kc=%d ctas=%d products=%d", g.tile_n,
             g.ntiles, 32 * g.ktot, w256, g.ntiles ? wmin : 0, g.flush, g.kc, g.G, products);
}

// ---- host-side fault injection ----------------------------------------------------
// HOS_FAULT (read at every entry): "workspace" makes each entry point report
// HOS_ERR_WORKSPACE after its argument checks; "cuda" makes the first CUDA
// call of each entry point report a failure without making it.  Nothing
// reaches the GPU in either case.
static bool fault_is(const char* what) {
    const char* f = std::getenv("HOS_FAULT");
    return f && std::strcmp(f, what) == 0;
}

// ---- current context ----------------------------------------------------------
// Identifier of the calling thread's current CUDA context (unique for the life
// of the process; a reset device gets a new one), or 0 when there is none yet
// or the driver cannot say.  The driver entry points are looked up through the
// runtime, so the library does not link the driver library itself.
using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);

uint64_t current_context_id() {
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || ctx == nullptr) return 0;
    unsigned long long id = 0;
    if (get_id(ctx, &id) != 0) return 0;
    return (uint64_t)id + 1;  // never 0 for a live context
}

// ---- tracing ------------------------------------------------------------------
constexpr int MAX_STAGES = 8;
constexpr int MAX_DEVICES = 64;
static std::mutex g_prof_mu;
static bool g_prof_on = false;
// Events belong to the device (context) they were created on: one set per
// device, remade when the device's context has changed.
static cudaEvent_t g_ev[MAX_DEVICES][MAX_STAGES + 1];
static uint64_t g_ev_ctx[MAX_DEVICES] = {0};
static int g_prof_dev = 0;  // device of the last traced call
static int g_prof_n = 0;    // events recorded by the last call
static const char* g_cur_names[MAX_STAGES];

// Stage events (when profiling is on) and an NVTX range per stage (always;
// no-ops unless a tool is attached).
struct Tracer {
    cudaStream_t st;
    int n = 0;
    bool on;
    bool range_open = false;
    cudaEvent_t* ev = nullptr;
    explicit Tracer(cudaStream_t s) : st(s) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        on = g_prof_on;
        if (!on) return;
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
            on = false;
            return;
        }
        // 0: no context made current yet (the first event creation makes the
        // device's primary context current) or the driver cannot say
        const uint64_t ctx = current_context_id();
        if (g_ev_ctx[dev] == 0 || (ctx != 0 && g_ev_ctx[dev] != ctx)) {
            for (int i = 0; i <= MAX_STAGES; ++i)
                if (cudaEventCreate(&g_ev[dev][i]) != cudaSuccess) {
                    on = false;
                    return;
                }
            const uint64_t now = current_context_id();
            g_ev_ctx[dev] = now ? now : ~0ull;
        }
        ev = g_ev[dev];
        g_prof_dev = dev;
        g_prof_n = 0;
    }
    ~Tracer() {
        if (range_open) nvtxRangePop();
    }
    void mark(const char* next_stage) {
        if (range_open) {
            nvtxRangePop();
            range_open = false;
        }
        if (next_stage && *next_stage) {
            nvtxRangePushA(next_stage);
            range_open = true;
        }
        if (!on || n > MAX_STAGES) return;
        cudaEventRecord(ev[n], st);
        if (n < MAX_STAGES) g_cur_names[n] = next_stage;
        ++n;
        g_prof_n = n;
    }
};

// ---- device properties -----------------------------------------------------------
static int sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    static int cache[64] = {0};
    if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    if (dev >= 0 && dev < 64) cache[dev] = n;
    return n;
}

// The partial-slot count the contraction's bounds checks use.  In the
// HOS_DEBUG_BOUNDS build, HOS_DEBUG_SHRINK_SLOTS=1 reports one slot, so that
// a test can watch the check stop a kernel (it records HOS_ERR_DEVICE_FAULT
// before any access and the kernel exits) without any access going astray.
static int64_t debug_slots(int64_t slots) {
#ifdef HOS_DEBUG_BOUNDS
    const char* v = std::getenv("HOS_DEBUG_SHRINK_SLOTS");
    if (v && std::strcmp(v, "1") == 0) return 1;
#endif
    return slots;
}

// The contraction's wait hints per role (producer, builders, epilogue, MMA
// issuer): try_wait suspend-time hints in ns, 0 = the system's own limit,
// WAIT_SPIN = poll without suspending.  HOS_C3_WAIT_HINTS="p,b,e,m" (ns, -1
// for a spin) overrides them.
static void wait_hints(uint32_t (&h)[4]) {
    h[0] = 2000;
    h[1] = 1000;
    h[2] = 20000;
    h[3] = 0;
    const char* v = std::getenv("HOS_C3_WAIT_HINTS");
    if (!v) return;
    for (int i = 0; i < 4 && *v; ++i) {
        char* end = nullptr;
        const long x = std::strtol(v, &end, 10);
        if (end == v) break;
        h[i] = x < 0 ? WAIT_SPIN : (uint32_t)x;
        v = (*end == ',') ? end + 1 : end;
    }
}

static uint64_t wait_limit_ns() {
    const char* v = getenv("HOS_WAIT_LIMIT_MS");
    long ms = v ? atol(v) : 4000;
    if (ms <= 0) ms = 4000;
    return (uint64_t)ms * 1000000ull;
}

// ---- validation and geometry ------------------------------------------------------
static int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
static int ilog2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return ((1 << l) == v) ? l : -1;
}

static hos_status check_params(const hos_params* p, int op) {
    if (!p) return HOS_ERR_INVALID_ARG;
    if (p->L < 1 || p->L > 1024) return p->L < 1 ? HOS_ERR_INVALID_ARG : HOS_ERR_UNSUPPORTED;
    if (p->nfft != 0 && (p->nfft < 2 * p->L || p->nfft > 4096)) return HOS_ERR_INVALID_ARG;
    {   // a grid size that is not a power of two uses the direct transform (<= 2048 points)
        const int nf = p->nfft ? p->nfft : 2 * p->L;
        if ((nf & (nf - 1)) != 0 && nf > 2048) return HOS_ERR_UNSUPPORTED;
    }
    if (p->precision < 0 || p->precision > 4) return HOS_ERR_INVALID_ARG;
    if (p->window < 0 || p->window > 2) return HOS_ERR_INVALID_ARG;
    if (p->segment_len < 0) return HOS_ERR_INVALID_ARG;
    if (p->tile_n != 0 && p->tile_n != 32 && p->tile_n != 64 && p->tile_n != 128 && p->tile_n != 256)
        return HOS_ERR_INVALID_ARG;
    if (p->flush_chunks < 0) return HOS_ERR_INVALID_ARG;
    if (p->chunk_len != 0 && (p->chunk_len < 64 || p->chunk_len > KC || p->chunk_len % 64 != 0))
        return HOS_ERR_INVALID_ARG;
    if (p->segment_overlap < 0) return HOS_ERR_INVALID_ARG;
    if (p->segment_overlap > 0) {
        const bool parts_op = (op == HOS_OP_BISPECTRUM || op == HOS_OP_TRISPECTRUM || op == HOS_OP_CUMULANT3 ||
                               op == HOS_OP_CUMULANT4);
        if (!parts_op || p->segment_len <= 0 || p->segment_overlap >= p->segment_len) return HOS_ERR_INVALID_ARG;
    }
    if (op == HOS_OP_TRISPECTRUM || op == HOS_OP_CUMULANT4 || op == HOS_OP_TRISPECTRUM_BATCHED ||
        op == HOS_OP_TRISPECTRUM_BACKWARD || op == HOS_OP_MOMENTS4_SLICE || op == HOS_OP_TRISPECTRUM_FROM_MOMENTS) {
        if (p->L > 64) return HOS_ERR_UNSUPPORTED;
        if (p->window == HOS_WIN_PARZEN_SYM) return HOS_ERR_UNSUPPORTED;
    }
    // time slices of the fourth order: tensor-core contraction, one part
    if (op == HOS_OP_MOMENTS4_SLICE && (p->precision == HOS_PREC_SIMT_FP32 || p->segment_len != 0))
        return p->segment_len != 0 ? HOS_ERR_INVALID_ARG : HOS_ERR_UNSUPPORTED;
    if ((op == HOS_OP_BISPECTRUM_BACKWARD || op == HOS_OP_TRISPECTRUM_BACKWARD) && p->segment_len != 0)
        return HOS_ERR_UNSUPPORTED;
    // the trispectrum adjoint runs on the tensor cores in split precision (bf16 or FP16) only
    if (op == HOS_OP_TRISPECTRUM_BACKWARD && p->precision != HOS_PREC_SPLIT_BF16 &&
        p->precision != HOS_PREC_SPLIT_FP16)
        return HOS_ERR_UNSUPPORTED;
    if ((op == HOS_OP_BISPECTRUM_BATCHED || op == HOS_OP_TRISPECTRUM_BATCHED) && p->segment_len != 0)
        return HOS_ERR_INVALID_ARG;
    return HOS_OK;
}

// Overlapping parts: parts of m = segment_len samples every m - overlap
// samples are copied one after another into the workspace tail and run as
// plain parts of m samples.  `on` is false when there is nothing to expand
// (no overlap, or n <= m: one part).
struct OverlapPlan {
    bool on = false;
    int64_t K = 1, m = 0, step = 0, n2 = 0;
};

static OverlapPlan overlap_plan(const hos_params* p, int64_t n) {
    OverlapPlan o;
    if (!p || p->segment_overlap <= 0 || p->segment_len <= 0 || n <= p->segment_len) return o;
    o.on = true;
    o.m = p->segment_len;
    o.step = o.m - p->segment_overlap;
    o.K = (n - o.m) / o.step + 1;
    o.n2 = o.K * o.m;
    return o;
}

// Tiles of the lag square.  c3(w1,w2) = c3(w2,w1), so row block a (128 lags
// w1) needs only the columns from its own diagonal block on, j >= 128a.
// Full width (the default): the row's tiles are N columns wide and start at
// the multiple of N at or below 128a, so the diagonal block's lower part is
// computed too.  Diagonal start (HOS_TILE_SCHEME=diagonal): the row starts at
// 128a and its last tile is narrower (a multiple of 32); fewer MMA columns,
// but on GB300 a 128-column tile's chunk takes about as long as a 256-column
// one, so full width is faster.
// skip_zero_window: leave out tiles where the window is zero at every lag
// (PARZEN_SYM: d(w1 - w2) = 0 for |w1 - w2| >= L); the transform grid is
// zero-filled there.  Returns the tile count (may exceed MAX_TILES: nothing is
// written past it).
static int build_tiles(C3Geom& g, int L, int N, bool skip_zero_window, int* zero_skipped) {
    const int twoL = 2 * L;
    const char* scheme = std::getenv("HOS_TILE_SCHEME");
    const bool diagonal = scheme && std::strcmp(scheme, "diagonal") == 0;
    int cnt = 0, k = 0, zs = 0;
    if (g.sym != C3_SWAP) {
        // six-fold: rows w1 in [0, L), each row block's columns from its first
        // row's diagonal w2 = w1 to its last row's w1 + L - 1 (L - 1 under the
        // band), in tiles of the full width N (a narrower tile costs the MMA
        // issue of a full one)
        for (int a = 0; a < g.tiles_m; ++a) {
            const int r0 = -L + a * TILE_M;
            const int b_lo = r0 > 0 ? r0 : 0, b_hi = (r0 + TILE_M < L) ? r0 + TILE_M : L;
            g.row_c0[a] = 0;
            g.row_t0[a] = (uint8_t)cnt;
            if (b_lo >= b_hi) continue;
            const int c_end = (g.sym == C3_SIX_BAND ? L : b_hi - 1 + L) + L;  // last column + 1
            const int c0 = ((b_lo + L) / 32) * 32;
            g.row_c0[a] = (uint16_t)c0;
            for (int c = c0; c < c_end; c += N) {
                if (cnt < MAX_TILES) {
                    g.tile_a[cnt] = (uint8_t)a;
                    g.tile_c32[cnt] = (uint8_t)(c / 32);
                    g.tile_w32[cnt] = (uint8_t)(N / 32);
                    g.tile_kpre[cnt] = (uint16_t)k;
                }
                k += N / 32;
                ++cnt;
            }
        }
        if (cnt <= MAX_TILES) g.tile_kpre[cnt] = (uint16_t)k;
        g.ktot = k;
        if (zero_skipped) *zero_skipped = 0;
        return cnt;
    }
    for (int a = 0; a < g.tiles_m; ++a) {
        const int c0 = diagonal ? a * TILE_M : (a * TILE_M / N) * N;
        g.row_c0[a] = (uint16_t)c0;
        g.row_t0[a] = (uint8_t)cnt;
        for (int c = c0; c < twoL;) {
            const int rem = (int)round_up(twoL - c, 32);
            const int w = diagonal ? (rem < N ? rem : N) : N;
            bool zero = false;
            if (skip_zero_window) {
                const int w1lo = -L + a * TILE_M, w1hi = w1lo + TILE_M - 1;
                const int w2lo = -L + c, w2hi = w2lo + w - 1;
                int gap = w1lo - w2hi;
                if (w2lo - w1hi > gap) gap = w2lo - w1hi;
                zero = gap >= L;  // min |w1 - w2| over the tile
            }
            if (zero) {
                ++zs;
            } else {
                if (cnt < MAX_TILES) {
                    g.tile_a[cnt] = (uint8_t)a;
                    g.tile_c32[cnt] = (uint8_t)(c / 32);
                    g.tile_w32[cnt] = (uint8_t)(w / 32);
                    g.tile_kpre[cnt] = (uint16_t)k;
                }
                k += w / 32;
                ++cnt;
            }
            c += w;
        }
    }
    if (cnt <= MAX_TILES) g.tile_kpre[cnt] = (uint16_t)k;
    g.ktot = k;
    if (zero_skipped) *zero_skipped = zs;
    return cnt;
}

// batched: many short series, whose estimates (symmetric returns: B near 0)
// are the least well conditioned, so the FP32-class paths take the shorter
// FP32 sums below.
static C3Geom make_geom(const hos_params* p, int G, bool skip_zero_window = false, int* zero_skipped = nullptr,
                        bool batched = false, int sym = C3_SWAP) {
    C3Geom g;
    memset(&g, 0, sizeof(g));
    const int twoL = 2 * p->L;
    g.L = p->L;
    g.sym = sym;
    int N = p->tile_n ? p->tile_n : next_pow2(twoL);
    if (N < 32) N = 32;
    if (N > 256) N = 256;
    g.tiles_m = (twoL + TILE_M - 1) / TILE_M;
    // tile_n is a hint: narrow tiles over a wide lag square are widened until
    // the plan has at most MAX_TILES tiles
    while (build_tiles(g, p->L, N, skip_zero_window, zero_skipped) > MAX_TILES && N < 256) N *= 2;
    g.tile_n = N;
    g.ntiles = build_tiles(g, p->L, N, skip_zero_window, zero_skipped);
    // The tensor cores' FP32 accumulation loses a little on every MMA step, one-sidedly,
    // so its error grows with the steps one partial accumulates.  The 3xTF32 path
    // (8 samples per step) hands its partial to the reduction after every
    // 1024-sample chunk; split-bf16 (16 samples per step, 1e-4 target) and SIMT
    // (FP32 FFMA, round to nearest) after 16 chunks.
    // Plain TF32 is limited by its 10-bit factors, not by the accumulation.
    // The error of the tensor cores' FP32 accumulation grows with the MMA
    // steps one partial holds (measured: about 1e-8 of the result per step,
    // for every operand format).  The FP32-class paths (1e-5 target) hand a
    // partial to the reduction every chunk (3xTF32: 384 MMA steps) or every
    // two chunks (split FP16: 192 steps a chunk); batched, every 192 steps
    // (3xTF32: 512-sample chunks; split FP16: every chunk).
    int flush_auto = 16, kc_auto = KC;
    if (p->precision == HOS_PREC_FP32) {
        flush_auto = 1;
        if (batched) kc_auto = 512;
    }
    if (p->precision == HOS_PREC_SPLIT_FP16) flush_auto = batched ? 1 : 2;
    g.flush = p->flush_chunks ? p->flush_chunks : flush_auto;
    g.kc = p->chunk_len ? p->chunk_len : kc_auto;
    g.G = G;
    // zero samples after a series: every sample a tile's windows read (the
    // SIMT kernel reads all N columns of a tile, the tensor cores its width)
    int reach = g.tiles_m * TILE_M;
    for (int t = 0; t < g.ntiles; ++t)
        if (32 * g.tile_c32[t] + N > reach) reach = 32 * g.tile_c32[t] + N;
    g.pad_tail = reach + 64;
    return g;
}

static int contraction_ctas(int precision) { return precision == HOS_PREC_SIMT_FP32 ? 4 * sm_count() : sm_count(); }

static bool tf32_kind(int precision) { return precision == HOS_PREC_FP32 || precision == HOS_PREC_TF32; }
// operand format of the tensor-core contraction
static int tc_format(int precision) {
    return tf32_kind(precision) ? FMT_TF32 : (precision == HOS_PREC_SPLIT_FP16 ? FMT_F16 : FMT_BF16);
}
// products per lag term on the tensor cores: hi*hi + hi*lo + lo*hi, or hi*hi alone (plain TF32)
static int tc_products(int precision) { return precision == HOS_PREC_TF32 ? 1 : 3; }
static int plane_split(int precision) {
    if (precision == HOS_PREC_SPLIT_BF16) return 1;
    if (precision == HOS_PREC_SPLIT_FP16) return 3;
    return tf32_kind(precision) ? 2 : 0;
}
static int plane_elt(int precision) {
    if (precision == HOS_PREC_SPLIT_BF16 || precision == HOS_PREC_SPLIT_FP16) return 2;
    return tf32_kind(precision) ? 4 : 0;
}
// The FP16 planes put each series' largest |y| at 2^7 (third order: products
// of two samples up to 2^14) or 2^4 (fourth order: three samples, 2^12),
// inside FP16's range (65504) with the lo halves mostly normal.
constexpr int FP16_TOP3 = 7, FP16_TOP4 = 4;
static const char* contraction_name(int order, int precision) {
    const bool o3 = order == 3;
    switch (precision) {
        case HOS_PREC_TF32: return o3 ? "c3_tcgen05_tf32" : "m4_tcgen05_tf32";
        case HOS_PREC_FP32: return o3 ? "c3_tcgen05_3xtf32" : "m4_tcgen05_3xtf32";
        case HOS_PREC_SPLIT_FP16: return o3 ? "c3_tcgen05_split_fp16" : "m4_tcgen05_split_fp16";
        default: return o3 ? "c3_tcgen05_split_bf16" : "m4_tcgen05_split_bf16";
    }
}

static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// Slices of each series' FP64 sum (mean removal): 8192 samples per slice, at
// most 256 (finer slices measured no faster on the 2^21-sample series).
static int mean_slices(int64_t len, int S) {
    (void)S;
    const int64_t k = ceil_div(len > 0 ? len : 1, 8192);
    return (int)(k > 256 ? 256 : (k < 1 ? 1 : k));
}

struct Layout {
    size_t status, off, pad, unit, win, mean, mpart, scale, smax, bnd, xr, ilen, wtab, y32, hi, lo, partials, grid, tw,
        total;
    int64_t plane_len, slots;
    int nslices;
    int groups;
};

// Carve the workspace.  S series (parts), n_total samples, longest max_len.
static Layout make_layout(int op, const hos_params* p, const C3Geom& g, int64_t n_total, int S, int64_t max_len) {
    Layout l;
    memset(&l, 0, sizeof(l));
    const int Nf = p->nfft ? p->nfft : 2 * p->L;
    l.nslices = mean_slices(max_len, S);
    l.plane_len = n_total + (int64_t)S * ((int64_t)p->L + KC + g.pad_tail + 64);
    const int64_t chunks = ceil_div(n_total, g.kc) + S;
    l.slots = (int64_t)g.ntiles * (chunks / g.flush + S + 1) + g.G;
    l.groups = (op == HOS_OP_BISPECTRUM_BATCHED) ? S : 1;
    size_t o = 0;
    l.status = o; o = al256(o + 256);
    l.off = o; o = al256(o + 8 * (size_t)(S + 1));
    l.pad = o; o = al256(o + 8 * (size_t)(S + 1));
    l.unit = o; o = al256(o + 8 * (size_t)(S + 1));
    l.win = o; o = al256(o + 8 * (size_t)(S + 1));
    l.mean = o; o = al256(o + 8 * (size_t)S);
    l.mpart = o; o = al256(o + 8 * (size_t)S * l.nslices);
    l.scale = o; o = al256(o + 4 * (size_t)S);
    l.smax = o; o = al256(o + 4 * (size_t)S);
    l.bnd = o; o = al256(o + 8 * (size_t)(g.G + 1));
    l.xr = o; o = al256(o + sizeof(TileRec) * (size_t)S * g.ntiles);
    l.ilen = o; o = al256(o + 8 * (size_t)S);
    l.wtab = o; o = al256(o + 4 * (size_t)(4 * p->L));
    l.y32 = o; o = al256(o + 4 * (size_t)l.plane_len);
    const int elt = plane_elt(p->precision);
    l.hi = o; o = al256(o + (size_t)elt * l.plane_len + 64);
    l.lo = o; o = al256(o + (size_t)elt * l.plane_len + 64);
    l.partials = o; o = al256(o + 4 * (size_t)l.slots * TILE_M * g.tile_n);
    const bool spectrum = (op == HOS_OP_BISPECTRUM || op == HOS_OP_BISPECTRUM_BATCHED);
    l.grid = o; o = al256(o + (spectrum ? 4 * (size_t)l.groups * Nf * Nf : 0));
    l.tw = o; o = al256(o + 8 * (size_t)Nf);
    l.total = o;
    return l;
}

// Everything a call needs to know before launching, computed in one place so
// that hos_workspace_size and the entry points agree.
struct Plan {
    C3Geom g;
    Layout l;
    int zero_tiles;  // tiles left out because the window is zero on them
    int S;           // series (batched) or parts (one series cut by segment_len)
    int64_t seg;     // part length, 0 = one part
    int64_t max_len; // longest series / part
    int Nf;
};

static hos_status make_plan(int op, const hos_params* p, int64_t n_total, int S_in, int64_t max_len_in, Plan& P) {
    hos_status s = check_params(p, op);
    if (s != HOS_OK) return s;
    P.Nf = p->nfft ? p->nfft : 2 * p->L;
    int64_t U_known = -1;
    if (op == HOS_OP_BISPECTRUM_BATCHED) {
        P.S = S_in;
        P.seg = 0;
        P.max_len = max_len_in;
    } else {
        P.seg = (p->segment_len > 0 && p->segment_len < n_total) ? p->segment_len : 0;
        const int64_t S64 = P.seg ? ceil_div(n_total, P.seg) : 1;
        if (S64 > 65535) return HOS_ERR_UNSUPPORTED;
        P.S = (int)S64;
        P.max_len = P.seg ? P.seg : n_total;
        // exact chunk count: full parts plus the (possibly shorter) last one
        const int64_t last = n_total - (P.S - 1) * (P.seg ? P.seg : 0);
        const int kc = p->chunk_len ? p->chunk_len : KC;  // make_geom's chunk length
        U_known = (P.S - 1) * ceil_div(P.max_len, kc) + ceil_div(last, kc);
    }
    if (P.S > 65535) return HOS_ERR_UNSUPPORTED;
    int G = contraction_ctas(p->precision);
    P.zero_tiles = 0;
    const bool windowed = (op == HOS_OP_BISPECTRUM || op == HOS_OP_BISPECTRUM_BATCHED);
    // The windowed spectra of whole series or parts compute the six-fold
    // fundamental set (a third fewer MMAs at L = 256, half at L = 128); the raw
    // cumulant (every lag of the square, w = -L included) and time slices
    // (whose partial sums keep only the swap symmetry) the swap plan.
    // HOS_TILE_SCHEME=swap (or =diagonal) selects the swap plan for measurement.
    // The six-fold plan is taken where it needs fewer tile columns than the
    // swap plan (its rows start at a 32-column boundary, so at small L it can
    // need more; on a tie the swap plan saves the unfold pass).
    const char* scheme = std::getenv("HOS_TILE_SCHEME");
    const bool band = p->window == HOS_WIN_PARZEN_SYM;
    P.g = make_geom(p, G, windowed && band, &P.zero_tiles, op == HOS_OP_BISPECTRUM_BATCHED, C3_SWAP);
    if (windowed && !scheme) {
        const C3Geom six = make_geom(p, G, false, nullptr, op == HOS_OP_BISPECTRUM_BATCHED,
                                     band ? C3_SIX_BAND : C3_SIX);
        if (six.ktot < P.g.ktot) {
            P.g = six;
            P.zero_tiles = 0;
        }
    }
    if (U_known >= 0) {
        const int64_t U = U_known * P.g.ntiles;
        if (U < G) P.g.G = (int)(U > 0 ? U : 1);
    }
    P.l = make_layout(op, p, P.g, n_total, P.S, P.max_len);
    return HOS_OK;
}

template <typename T>
static T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(reinterpret_cast<uint8_t*>(ws) + off);
}

#define HOS_CUDA_TRY(expr)                         \
    do {                                           \
        if (fault_is("cuda")) return HOS_ERR_CUDA;   \
        cudaError_t e__ = (expr);                  \
        if (e__ != cudaSuccess) return HOS_ERR_CUDA; \
    } while (0)

static LineGeom line_geom(int N, int64_t nlines, int64_t inner, int64_t outer, int64_t elem) {
    LineGeom g;
    g.N = N;
    g.log2N = ilog2_exact(N);
    g.nlines = nlines;
    g.inner = inner;
    g.outer_stride = outer;
    g.elem_stride = elem;
    g.half_out = 0;
    g.herm = 0;
    int lpb = (g.log2N >= 0) ? 4096 / N : 2048 / N;
    // few lines: fewer per CTA so that the grid covers the SMs
    const int64_t spread = nlines / (2 * (int64_t)sm_count());
    if (spread < lpb) lpb = (int)(spread > 0 ? spread : 1);
    if (lpb < 1) lpb = 1;
    if (lpb > nlines) lpb = (int)(nlines > 0 ? nlines : 1);
    g.lpb = lpb;
    return g;
}

// A time slice of a longer series (hos_cumulant3_slice).
struct SliceArgs {
    int64_t halo_before, halo_after;  // neighbour samples around the slice in the input
    const double* d_sum;              // FP64 sum of the whole series (device)
    int64_t n_total;                  // length of the whole series
};

constexpr double kBispecScale = 1.0 / (4.0 * 3.14159265358979323846 * 3.14159265358979323846);  // (2 pi)^-2

// hos_series_sum's workspace: off {0, n} (256 B), then one FP64 partial per slice
static int sum_slices(int64_t n) { return mean_slices(n, 1); }
static size_t sum_ws_bytes(int64_t n) { return 256 + al256(8 * (size_t)sum_slices(n)); }

// hos_bispectrum_from_cumulant's workspace: window table, grid, twiddles
struct FromC3Layout {
    int Nf;
    size_t wtab, grid, tw, total;
};
static FromC3Layout from_c3_layout(const hos_params* p) {
    FromC3Layout l;
    l.Nf = p->nfft ? p->nfft : 2 * p->L;
    size_t o = 0;
    l.wtab = o; o = al256(o + 4 * (size_t)(4 * p->L));
    l.grid = o; o = al256(o + 4 * (size_t)l.Nf * l.Nf);
    l.tw = o; o = al256(o + 8 * (size_t)l.Nf);
    l.total = o;
    return l;
}

// hos_trispectrum_from_moments's workspace: grid, twiddles
struct FromM4Layout {
    int Nf;
    size_t grid, tw, total;
};
static FromM4Layout from_m4_layout(const hos_params* p) {
    FromM4Layout l;
    l.Nf = p->nfft ? p->nfft : 2 * p->L;
    size_t o = 0;
    l.grid = o; o = al256(o + 4 * (size_t)l.Nf * l.Nf * l.Nf);
    l.tw = o; o = al256(o + 8 * (size_t)l.Nf);
    l.total = o;
    return l;
}


// Steps shared by the c3 operations: plan, mean, planes, contraction, reduce.
static hos_status run_c3(int op, const void* x, int dtype, int64_t n, const int64_t* d_offsets, const Plan& P,
                         const hos_params* p, void* ws, size_t ws_bytes, cudaStream_t st, Tracer& tr, int red_mode,
                         float* grid_out, double* c3_out, const SliceArgs* sl = nullptr) {
    const C3Geom& g = P.g;
    const Layout& l = P.l;
    const int S = P.S;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < l.total ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    int* status = at<int>(ws, l.status);
    int64_t* off = at<int64_t>(ws, l.off);
    int64_t* pad = at<int64_t>(ws, l.pad);
    int64_t* unit = at<int64_t>(ws, l.unit);
    int64_t* win = at<int64_t>(ws, l.win);
    double* mean = at<double>(ws, l.mean);
    float* y32 = at<float>(ws, l.y32);
    void* hi = at<void>(ws, l.hi);
    void* lo = at<void>(ws, l.lo);
    float* partials = at<float>(ws, l.partials);

    tr.mark("prep");
    const int mode = (op == HOS_OP_BISPECTRUM_BATCHED) ? 1 : 0;
    HOS_CUDA_TRY(launch_plan_series(mode, n, P.seg, d_offsets, S, p->L, g.ntiles, g.ktot, g.flush, g.kc, g.pad_tail,
                                    off, pad, unit, win, st));
    const void* xs = x;
    if (sl) {  // the whole series' mean; the slice's first sample follows its halo
        HOS_CUDA_TRY(launch_slice_mean(sl->d_sum, sl->n_total, p->remove_mean, mean, st));
        xs = reinterpret_cast<const uint8_t*>(x) + sl->halo_before * (dtype == HOS_F64 ? 8 : 4);
    } else {
        HOS_CUDA_TRY(launch_mean(x, dtype, off, S, l.nslices, at<double>(ws, l.mpart), p->remove_mean, mean, st));
    }
    const int64_t maxpad = (int64_t)p->L + P.max_len + KC + g.pad_tail + 64;
    int bx = (int)ceil_div(maxpad, 256 * 4);
    if (bx < 1) bx = 1;
    if (bx > 65535) bx = 65535;
    float* scale = nullptr;
    if (p->precision == HOS_PREC_SPLIT_FP16) {
        scale = at<float>(ws, l.scale);
        HOS_CUDA_TRY(launch_series_scale(xs, dtype, off, mean, S, l.nslices, sl ? sl->halo_before : 0,
                                         sl ? sl->halo_after : 0, FP16_TOP3, at<unsigned>(ws, l.smax), scale, st));
    }
    HOS_CUDA_TRY(launch_planes(xs, dtype, off, pad, mean, p->L, plane_split(p->precision), y32, hi, lo, S, bx, st,
                               sl ? sl->halo_before : 0, sl ? sl->halo_after : 0, scale));

    SeriesView sv{off, pad, unit, win, mean, S, scale};
    tr.mark("contract");
    if (p->precision == HOS_PREC_SIMT_FP32) {
        C3SimtParams cp{g, sv, y32, partials};
        HOS_CUDA_TRY(launch_c3_simt(cp, g.G, st));
        g_last_contraction = "c3_simt_fp32";
        note_plan(g, 1);
    } else {
        C3TcParams cp{g, sv, y32, hi, lo, partials, status, wait_limit_ns(), tc_products(p->precision), l.plane_len,
                      debug_slots(l.slots), {}};
        wait_hints(cp.hint);
        HOS_CUDA_TRY(launch_c3_tc(tc_format(p->precision), 3, cp, g.G, st));
        g_last_contraction = contraction_name(3, p->precision);
        note_plan(g, tc_products(p->precision));
    }

    tr.mark("reduce");
    Reduce3Params rp;
    rp.geom = g;
    rp.ser = sv;
    rp.partials = partials;
    rp.window = p->window;
    rp.nfft = P.Nf;
    rp.mode = red_mode;
    rp.per_series_groups = (op == HOS_OP_BISPECTRUM_BATCHED) ? 1 : 0;
    rp.scale = kBispecScale;
    rp.grid = grid_out;
    rp.c3out = c3_out;
    rp.norm_len = sl ? sl->n_total : 0;
    const int groups = rp.per_series_groups ? S : 1;
    rp.tiles_out = partials;
    rp.n_slots = debug_slots(l.slots);
    rp.grid_floats = (red_mode == 0) ? (int64_t)groups * P.Nf * P.Nf : 0;
    rp.status = status;
    // grid entries no computed lag writes (lags past L when Nf > 2L, skipped
    // tiles) are zeroed first; the six-fold plans write every entry
    if (red_mode == 0 && g.sym == C3_SWAP && (P.Nf > 2 * p->L || P.zero_tiles > 0))
        HOS_CUDA_TRY(launch_zero_f32(grid_out, (int64_t)groups * P.Nf * P.Nf, st));
    HOS_CUDA_TRY(launch_reduce3(rp, groups, P.max_len, at<int64_t>(ws, l.bnd), at<TileRec>(ws, l.xr),
                                at<float2>(ws, l.ilen), at<float>(ws, l.wtab), st));
    return HOS_OK;
}

static hos_status run_dft2(float* grid, float2* out, int groups, int Nf, float2* tw, cudaStream_t st) {
    HOS_CUDA_TRY(launch_twiddles(Nf, tw, st));
    // The grid is real, so its 2-D transform is Hermitian: B(N-k2, N-k1) = conj B(k2, k1).
    // For N a power of two >= 8 the row pass writes columns 0..N/2 only and the
    // column pass transforms those columns and mirrors them into the rest.
    const bool herm = (Nf >= 8) && ((Nf & (Nf - 1)) == 0);
    // along the last axis (contiguous), real input
    LineGeom g1 = line_geom(Nf, (int64_t)groups * Nf, 1, Nf, 1);
    g1.half_out = herm ? 1 : 0;
    HOS_CUDA_TRY(launch_lines(true, grid, out, g1, tw, -1, 1.0f, st));
    // along the first axis, in place
    if (herm) {
        LineGeom g2 = line_geom(Nf, (int64_t)groups * (Nf / 2 + 1), Nf / 2 + 1, (int64_t)Nf * Nf, Nf);
        g2.herm = 1;
        HOS_CUDA_TRY(launch_lines(false, out, out, g2, tw, -1, 1.0f, st));
    } else {
        LineGeom g2 = line_geom(Nf, (int64_t)groups * Nf, Nf, (int64_t)Nf * Nf, Nf);
        HOS_CUDA_TRY(launch_lines(false, out, out, g2, tw, -1, 1.0f, st));
    }
    return HOS_OK;
}

// ---- fourth order --------------------------------------------------------------------
struct Plan4 {
    int S;
    bool batched;  // S independent series from caller offsets, one spectrum each
    int64_t seg, max_len, total_groups;
    int Nf, W3, npb, nslices, pad_tail;
    bool tc;    // tensor-core m4 (split-bf16 / 3xTF32) instead of FP32 SIMT
    C3Geom g4;  // tensor-core geometry: tiles = blocks of 128 lag pairs, columns = w3
    size_t status, off, pad, unit, win, mean, mpart, scale, smax, y32, hi, lo, bnd, xr, ilen, m4buf, c2, c2p, partials,
        grid, tw,
        total;
    int c2s;        // slices per part of the c2 sums
    int64_t slots;  // partial slots of the tensor-core contraction
    int64_t plane_len;
};

// Geometry of the tensor-core m4 contraction: tile t = pairs [128t, 128t+128)
// of the lag triangle w1 <= w2 (rows), all w3 in [-L, L) (columns).
static C3Geom make_geom4(const hos_params* p, int G) {
    C3Geom g;
    memset(&g, 0, sizeof(g));
    const int twoL = 2 * p->L;
    g.L = p->L;
    int N = next_pow2(twoL);
    if (N < 32) N = 32;
    g.tile_n = N;
    const int npairs = twoL * (twoL + 1) / 2;
    g.tiles_m = (npairs + TILE_M - 1) / TILE_M;  // blocks of pairs (row_c0 is unused)
    g.ntiles = g.tiles_m;
    for (int t = 0; t < g.ntiles; ++t) {
        g.tile_a[t] = (uint8_t)t;
        g.tile_c32[t] = 0;
        g.tile_w32[t] = (uint8_t)(N / 32);
        g.tile_kpre[t] = (uint16_t)(t * (N / 32));
    }
    g.tile_kpre[g.ntiles] = (uint16_t)(g.ntiles * (N / 32));
    g.ktot = g.ntiles * (N / 32);
    // c4 = m4 - sum c2*c2 cancels, which magnifies the tensor cores' one-sided
    // FP32 accumulation loss: partials go to the reduction after every
    // chunk, and 3xTF32 chunks are 128 samples (48 MMA steps)
    g.flush = p->flush_chunks ? p->flush_chunks : 1;
    // (the split FP16 path: 128-sample chunks, 24 MMA steps)
    g.kc = p->chunk_len ? p->chunk_len : ((p->precision == HOS_PREC_FP32 || p->precision == HOS_PREC_SPLIT_FP16) ? 128 : KC);
    g.G = G;
    g.pad_tail = 128 + N + 128;
    return g;
}

static hos_status make_plan4(int op, const hos_params* p, int64_t n, Plan4& P, int S_in = 1, int64_t max_len_in = 0) {
    hos_status s = check_params(p, op);
    if (s != HOS_OK) return s;
    const int L = p->L, twoL = 2 * L;
    P.Nf = p->nfft ? p->nfft : twoL;
    P.batched = (op == HOS_OP_TRISPECTRUM_BATCHED);
    int64_t last;
    if (P.batched) {
        if (p->precision == HOS_PREC_SIMT_FP32) return HOS_ERR_UNSUPPORTED;  // tensor-core path only
        if (S_in < 1 || S_in > 65535) return S_in < 1 ? HOS_ERR_INVALID_ARG : HOS_ERR_UNSUPPORTED;
        P.seg = 0;
        P.S = S_in;
        P.max_len = max_len_in;
        last = max_len_in;
    } else {
        P.seg = (p->segment_len > 0 && p->segment_len < n) ? p->segment_len : 0;
        const int64_t S64 = P.seg ? ceil_div(n, P.seg) : 1;
        if (S64 > 65535) return HOS_ERR_UNSUPPORTED;
        P.S = (int)S64;
        P.max_len = P.seg ? P.seg : n;
        last = n - (P.S - 1) * (P.seg ? P.seg : 0);
    }
    auto groups = [](int64_t len) { return ceil_div(ceil_div(len, KC), C4_CHUNK_GROUP); };
    P.total_groups = (P.S - 1) * groups(P.max_len) + groups(last);
    if (P.total_groups > 65535) return HOS_ERR_UNSUPPORTED;
    P.W3 = 16 * ((twoL + 15) / 16);
    const int npairs = twoL * (twoL + 1) / 2;
    P.npb = (npairs + C4_PAIRS_PER_CTA - 1) / C4_PAIRS_PER_CTA;
    P.pad_tail = 32 + 128 + 64 + 64;
    P.tc = (p->precision != HOS_PREC_SIMT_FP32);
    if (P.tc) {
        P.g4 = make_geom4(p, sm_count());
        // work units (tile, chunk); for caller offsets only an upper bound is known
        const int64_t U = P.batched ? (int64_t)P.g4.ntiles * (ceil_div(n, P.g4.kc) + P.S)
                                    : (int64_t)P.g4.ntiles *
                                          ((P.S - 1) * ceil_div(P.max_len, P.g4.kc) + ceil_div(last, P.g4.kc));
        if (U < P.g4.G) P.g4.G = (int)(U > 0 ? U : 1);
        P.pad_tail = P.g4.pad_tail;
    }
    P.nslices = mean_slices(P.max_len, P.S);
    const int64_t plane_len = n + (int64_t)P.S * ((int64_t)L + KC + P.pad_tail + 64);
    P.plane_len = plane_len;
    P.slots = 0;
    size_t o = 0;
    P.status = o; o = al256(o + 256);
    P.off = o; o = al256(o + 8 * (size_t)(P.S + 1));
    P.pad = o; o = al256(o + 8 * (size_t)(P.S + 1));
    P.unit = o; o = al256(o + 8 * (size_t)(P.S + 1));
    P.win = o; o = al256(o + 8 * (size_t)(P.S + 1));
    P.mean = o; o = al256(o + 8 * (size_t)P.S);
    P.mpart = o; o = al256(o + 8 * (size_t)P.S * P.nslices);
    P.scale = o; o = al256(o + 4 * (size_t)P.S);
    P.smax = o; o = al256(o + 4 * (size_t)P.S);
    P.y32 = o; o = al256(o + 4 * (size_t)plane_len);
    P.c2 = o; o = al256(o + 8 * (size_t)P.S * (4 * L - 1));
    P.c2s = c2_slices(P.S, P.max_len);
    P.c2p = o; o = al256(o + (P.c2s > 1 ? 8 * (size_t)P.S * (4 * L - 1) * P.c2s : 0));
    if (P.tc) {
        const C3Geom& g = P.g4;
        const int elt = plane_elt(p->precision);
        const int64_t chunks = ceil_div(n, g.kc) + P.S;
        const int64_t slots = (int64_t)g.ntiles * (chunks / g.flush + P.S + 1) + g.G;
        P.slots = slots;
        const size_t tsz = (size_t)TILE_M * g.tile_n;
        P.hi = o; o = al256(o + (size_t)elt * plane_len + 64);
        P.lo = o; o = al256(o + (size_t)elt * plane_len + 64);
        P.bnd = o; o = al256(o + 8 * (size_t)(g.G + 1));
        P.xr = o; o = al256(o + sizeof(TileRec) * (size_t)P.S * g.ntiles);
        P.ilen = o; o = al256(o + 8 * (size_t)P.S);
        P.partials = o; o = al256(o + 4 * (size_t)slots * tsz);
        P.m4buf = o; o = al256(o + 8 * (size_t)P.S * g.ntiles * tsz);
    } else {
        P.partials = o; o = al256(o + 4 * (size_t)P.total_groups * P.npb * C4_PAIRS_PER_CTA * P.W3);
    }
    const bool spectra = (op == HOS_OP_TRISPECTRUM || op == HOS_OP_TRISPECTRUM_BATCHED);
    P.grid = o; o = al256(o + (spectra ? 4 * (size_t)P.S * P.Nf * P.Nf * P.Nf : 0));
    P.tw = o; o = al256(o + 8 * (size_t)P.Nf);
    P.total = o;
    return HOS_OK;
}

// sl: a time slice of a longer series (the mean from the whole series' sum,
// halo samples around the slice serve as lags only, 1/n of the whole series;
// mode 2 writes the raw m4 cube and c2_out receives c2).
static hos_status run_c4(const void* x, int dtype, int64_t n, const Plan4& P, const hos_params* p, void* ws,
                         size_t ws_bytes, cudaStream_t st, Tracer& tr, int mode, double* c4out,
                         const int64_t* d_offsets = nullptr, const SliceArgs* sl = nullptr,
                         double* c2_out = nullptr) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < P.total ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    int64_t* off = at<int64_t>(ws, P.off);
    int64_t* pad = at<int64_t>(ws, P.pad);
    int64_t* unit = at<int64_t>(ws, P.unit);
    int64_t* win = at<int64_t>(ws, P.win);
    double* mean = at<double>(ws, P.mean);
    float* y32 = at<float>(ws, P.y32);
    tr.mark("prep");
    const int ntiles = P.tc ? P.g4.ntiles : 1;
    const int ktot = P.tc ? P.g4.ktot : 1;
    const int flush = P.tc ? P.g4.flush : C4_CHUNK_GROUP;
    const int kc = P.tc ? P.g4.kc : KC;
    HOS_CUDA_TRY(launch_plan_series(P.batched ? 1 : 0, n, P.seg, d_offsets, P.S, p->L, ntiles, ktot, flush, kc,
                                    P.pad_tail, off, pad, unit, win, st));
    if (sl) HOS_CUDA_TRY(launch_slice_mean(sl->d_sum, sl->n_total, p->remove_mean, mean, st));
    else HOS_CUDA_TRY(launch_mean(x, dtype, off, P.S, P.nslices, at<double>(ws, P.mpart), p->remove_mean, mean, st));
    const int64_t maxpad = (int64_t)p->L + P.max_len + KC + P.pad_tail + 64;
    int bx = (int)ceil_div(maxpad, 256 * 4);
    if (bx < 1) bx = 1;
    if (bx > 65535) bx = 65535;
    void* hi = P.tc ? at<void>(ws, P.hi) : nullptr;
    void* lo = P.tc ? at<void>(ws, P.lo) : nullptr;
    // a slice's input pointer is its first own sample; its halos lie before and after
    const void* xs = sl ? static_cast<const uint8_t*>(x) + sl->halo_before * (dtype == HOS_F64 ? 8 : 4) : x;
    float* scale = nullptr;
    if (P.tc && p->precision == HOS_PREC_SPLIT_FP16) {
        scale = at<float>(ws, P.scale);
        HOS_CUDA_TRY(launch_series_scale(xs, dtype, off, mean, P.S, P.nslices, sl ? sl->halo_before : 0,
                                         sl ? sl->halo_after : 0, FP16_TOP4, at<unsigned>(ws, P.smax), scale, st));
    }
    HOS_CUDA_TRY(launch_planes(xs, dtype, off, pad, mean, p->L, P.tc ? plane_split(p->precision) : 0, y32, hi, lo,
                               P.S, bx, st, sl ? sl->halo_before : 0, sl ? sl->halo_after : 0, scale));
    tr.mark("contract");
    C4ReduceArgs r;
    r.window = p->window;
    r.nfft = P.Nf;
    r.mode = mode;
    r.scale = 1.0 / (8.0 * 3.14159265358979323846 * 3.14159265358979323846 * 3.14159265358979323846);
    r.grid = at<float>(ws, P.grid);
    r.c4out = c4out;
    const int ngrids = P.batched ? P.S : 1;
    if (mode == 0 && P.Nf > 2 * p->L)
        HOS_CUDA_TRY(launch_zero_f32(r.grid, (int64_t)ngrids * P.Nf * P.Nf * P.Nf, st));
    if (!P.tc) {
        HOS_CUDA_TRY(launch_c4(y32, off, pad, win, P.S, p->L, C4_CHUNK_GROUP, P.total_groups, at<double>(ws, P.c2),
                               at<float>(ws, P.partials), r, st));
        g_last_contraction = "m4_simt_fp32";
        return HOS_OK;
    }
    double* c2 = at<double>(ws, P.c2);
    HOS_CUDA_TRY(launch_c2(y32, off, pad, P.S, p->L, P.c2s, c2, at<float2>(ws, P.c2p), st, sl ? 1 : 0,
                           sl ? sl->n_total : 0));
    SeriesView sv{off, pad, unit, win, mean, P.S, scale};
    C3TcParams cp{P.g4, sv, y32, hi, lo, at<float>(ws, P.partials), at<int>(ws, P.status), wait_limit_ns(),
                  tc_products(p->precision), P.plane_len, debug_slots(P.slots), {}};
    wait_hints(cp.hint);
    HOS_CUDA_TRY(launch_c3_tc(tc_format(p->precision), 4, cp, P.g4.G, st));
    g_last_contraction = contraction_name(4, p->precision);
    note_plan(P.g4, tc_products(p->precision));
    tr.mark("reduce");
    double* m4buf = at<double>(ws, P.m4buf);
    HOS_CUDA_TRY(launch_m4_tile_reduce(P.g4, sv, P.max_len, at<float>(ws, P.partials), at<int64_t>(ws, P.bnd),
                                       at<TileRec>(ws, P.xr), at<float2>(ws, P.ilen), m4buf, st,
                                       sl ? sl->n_total : 0));
    HOS_CUDA_TRY(launch_c4_assemble(m4buf, c2, off, P.S, p->L, P.g4.ntiles, P.g4.tile_n, r, P.batched ? 1 : 0, st));
    if (c2_out)
        HOS_CUDA_TRY(cudaMemcpyAsync(c2_out, c2, sizeof(double) * (size_t)(4 * p->L - 1), cudaMemcpyDeviceToDevice,
                                     st));
    return HOS_OK;
}

// 3-D transform of `grids` consecutive N^3 grids, one axis at a time.
static hos_status run_dft3(float* grid, float2* out, int Nf, float2* tw, cudaStream_t st, int grids = 1) {
    const int64_t N = Nf, N2 = N * N, G = grids;
    HOS_CUDA_TRY(launch_twiddles(Nf, tw, st));
    LineGeom g2 = line_geom(Nf, G * N2, 1, N, 1);  // along k3 (contiguous), real input
    HOS_CUDA_TRY(launch_lines(true, grid, out, g2, tw, -1, 1.0f, st));
    LineGeom g1 = line_geom(Nf, G * N2, N, N2, N);  // along k2
    HOS_CUDA_TRY(launch_lines(false, out, out, g1, tw, -1, 1.0f, st));
    LineGeom g0 = line_geom(Nf, G * N2, N2, N2 * N, N2);  // along k1
    HOS_CUDA_TRY(launch_lines(false, out, out, g0, tw, -1, 1.0f, st));
    return HOS_OK;
}

// ---- adjoint ----------------------------------------------------------------------------
struct PlanB {
    C3Geom g;
    int Nf, nslices;
    int64_t nctas;
    bool tc;  // tensor-core adjoint (split-bf16 or split FP16, L <= 128)
    size_t status, off, pad, unit, win, mean, mpart, sc, smx, y32, hi, lo, gc, gs, gsb, t1, t2p, gbuf, gmean, gmpart,
        tw, total;
};

static hos_status make_planb(const hos_params* p, int64_t n, PlanB& P) {
    hos_status s = check_params(p, HOS_OP_BISPECTRUM_BACKWARD);
    if (s != HOS_OK) return s;
    const int L = p->L, twoL = 2 * L;
    P.g = make_geom(p, 1);
    // the adjoint reads y(u + w1) windows up to 2L + 256 samples past a row tile
    if (P.g.pad_tail < twoL + 320) P.g.pad_tail = twoL + 320;
    P.tc = (p->precision == HOS_PREC_SPLIT_BF16 || p->precision == HOS_PREC_SPLIT_FP16) && adjoint_tc_supported(L);
    P.Nf = p->nfft ? p->nfft : twoL;
    P.nslices = mean_slices(n, 1);
    P.nctas = ceil_div(n, ADJ_ROWS_PER_CTA);
    const int64_t plane_len = n + ((int64_t)L + KC + P.g.pad_tail + 64);
    size_t o = 0;
    P.status = o; o = al256(o + 256);
    P.off = o; o = al256(o + 16);
    P.pad = o; o = al256(o + 16);
    P.unit = o; o = al256(o + 16);
    P.win = o; o = al256(o + 16);
    P.mean = o; o = al256(o + 8);
    P.mpart = o; o = al256(o + 8 * (size_t)P.nslices);
    P.sc = o; o = al256(o + 8);
    P.smx = o; o = al256(o + 8);
    P.y32 = o; o = al256(o + 4 * (size_t)plane_len);
    P.hi = o; o = al256(o + (P.tc ? 2 * (size_t)plane_len + 64 : 0));
    P.lo = o; o = al256(o + (P.tc ? 2 * (size_t)plane_len + 64 : 0));
    P.gc = o; o = al256(o + 8 * (size_t)P.Nf * P.Nf);
    P.gs = o; o = al256(o + 4 * (size_t)twoL * twoL);
    P.gsb = o; o = al256(o + (P.tc ? adjoint_tc_gs_bytes(L) : 0));
    P.t1 = o; o = al256(o + 4 * (P.tc ? adjoint_tc_t1_floats(L, n) : (size_t)P.nctas * ADJ_ROWS_PER_CTA));
    P.t2p = o; o = al256(o + 4 * (P.tc ? adjoint_tc_t2_floats(L, n) : (size_t)P.nctas * (ADJ_ROWS_PER_CTA + twoL)));
    P.gbuf = o; o = al256(o + 4 * (size_t)n);
    P.gmean = o; o = al256(o + 8);
    P.gmpart = o; o = al256(o + 8 * (size_t)P.nslices);
    P.tw = o; o = al256(o + 8 * (size_t)P.Nf);
    P.total = o;
    return HOS_OK;
}

// ---- trispectrum adjoint -------------------------------------------------------------
struct PlanB4 {
    C3Geom g;
    int Nf, nslices;
    size_t status, off, pad, unit, win, mean, mpart, sc, smx, y32, hi, lo, c2, c2p, gc, gs, gsb, gc2, t1, t2p, gbuf,
        gmean, gmpart, tw, total;
    int c2s;
};

static hos_status make_planb4(const hos_params* p, int64_t n, PlanB4& P) {
    hos_status s = check_params(p, HOS_OP_TRISPECTRUM_BACKWARD);
    if (s != HOS_OK) return s;
    const int L = p->L, twoL = 2 * L;
    P.g = make_geom(p, 1);
    // the adjoint reads windows up to 2L + 256 samples past a row tile
    if (P.g.pad_tail < twoL + 320) P.g.pad_tail = twoL + 320;
    P.Nf = p->nfft ? p->nfft : twoL;
    P.nslices = mean_slices(n, 1);
    const int64_t plane_len = n + ((int64_t)L + KC + P.g.pad_tail + 64);
    const int64_t N3 = (int64_t)P.Nf * P.Nf * P.Nf;
    size_t o = 0;
    P.status = o; o = al256(o + 256);
    P.off = o; o = al256(o + 16);
    P.pad = o; o = al256(o + 16);
    P.unit = o; o = al256(o + 16);
    P.win = o; o = al256(o + 16);
    P.mean = o; o = al256(o + 8);
    P.mpart = o; o = al256(o + 8 * (size_t)P.nslices);
    P.sc = o; o = al256(o + 8);
    P.smx = o; o = al256(o + 8);
    P.y32 = o; o = al256(o + 4 * (size_t)plane_len);
    P.hi = o; o = al256(o + 2 * (size_t)plane_len + 64);
    P.lo = o; o = al256(o + 2 * (size_t)plane_len + 64);
    P.c2 = o; o = al256(o + 8 * (size_t)(4 * L - 1));
    P.c2s = c2_slices(1, n);
    P.c2p = o; o = al256(o + (P.c2s > 1 ? 8 * (size_t)(4 * L - 1) * P.c2s : 0));
    P.gc = o; o = al256(o + 8 * (size_t)N3);
    P.gs = o; o = al256(o + 4 * (size_t)twoL * twoL * twoL);
    P.gsb = o; o = al256(o + adjoint_tc_gs_bytes(L, 4));
    P.gc2 = o; o = al256(o + 8 * (size_t)(4 * L - 1));
    P.t1 = o; o = al256(o + 4 * adjoint_tc_t1_floats(L, n, 4));
    P.t2p = o; o = al256(o + 4 * adjoint_tc_t2_floats(L, n, 4));
    P.gbuf = o; o = al256(o + 4 * (size_t)n);
    P.gmean = o; o = al256(o + 8);
    P.gmpart = o; o = al256(o + 8 * (size_t)P.nslices);
    P.tw = o; o = al256(o + 8 * (size_t)P.Nf);
    P.total = o;
    return HOS_OK;
}

// Run `core` on x, or, with overlapping parts, on the parts copied one after
// another into the workspace tail (as plain parts of segment_len samples).
using PartsCore = hos_status (*)(const void* x, int32_t dtype, int64_t n, const hos_params* p, void* out, void* ws,
                                 size_t ws_bytes, hos_stream_t stream);

static hos_status overlap_workspace(int32_t op, int64_t n, const hos_params* p, const OverlapPlan& o, size_t* inner,
                                    size_t* total) {
    hos_params p2 = *p;
    p2.segment_overlap = 0;
    size_t b = 0;
    hos_status s = hos_workspace_size(op, o.n2, 1, o.n2, &p2, &b);
    if (s != HOS_OK) return s;
    *inner = al256(b);
    *total = *inner + (size_t)o.n2 * sizeof(double);
    (void)n;
    return HOS_OK;
}

static hos_status with_overlap(int32_t op, const void* d_x, int32_t dtype, int64_t n, const hos_params* p, void* out,
                               void* ws, size_t ws_bytes, hos_stream_t stream, PartsCore core) {
    if (!d_x || !out || n < 1 || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    hos_status s = check_params(p, op);
    if (s != HOS_OK) return s;
    const OverlapPlan o = overlap_plan(p, n);
    hos_params p2 = *p;
    p2.segment_overlap = 0;
    if (!o.on) return core(d_x, dtype, n, &p2, out, ws, ws_bytes, stream);
    size_t inner = 0, total = 0;
    s = overlap_workspace(op, n, p, o, &inner, &total);
    if (s != HOS_OK) return s;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < total ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    void* xs = static_cast<uint8_t*>(ws) + inner;
    HOS_CUDA_TRY(launch_gather_parts(d_x, dtype, o.K, o.m, o.step, xs, reinterpret_cast<cudaStream_t>(stream)));
    return core(xs, dtype, o.n2, &p2, out, ws, inner, stream);
}

}  // namespace hos

using namespace hos;

extern "C" {

const char* hos_version(void) { return "hos-gb300 0.2 (sm_103a)"; }

const char* hos_status_string(int32_t s) {
    switch (s) {
        case HOS_OK: return "ok";
        case HOS_ERR_INVALID_ARG: return "invalid argument";
        case HOS_ERR_UNSUPPORTED: return "unsupported";
        case HOS_ERR_WORKSPACE: return "workspace too small or misaligned";
        case HOS_ERR_CUDA: return "CUDA error";
        case HOS_ERR_TIMEOUT: return "device wait timed out";
        case HOS_ERR_DEVICE_FAULT: return "device consistency check failed";
        default: return "unknown status";
    }
}

int64_t hos_launch_count(void) { return g_launches.load(); }
const char* hos_last_contraction(void) { return g_last_contraction; }
const char* hos_last_plan(void) { return g_last_plan; }

hos_status hos_workspace_size(int32_t op, int64_t n_total, int32_t n_series, int64_t max_len, const hos_params* p,
                              size_t* bytes) {
    if (!bytes || n_total < 0 || n_series < 1 || max_len < 0) return HOS_ERR_INVALID_ARG;
    if (op < 0 || op > HOS_OP_TRISPECTRUM_FROM_MOMENTS) return HOS_ERR_INVALID_ARG;
    if (op == HOS_OP_TRISPECTRUM_FROM_MOMENTS) {
        hos_status sf = check_params(p, op);
        if (sf != HOS_OK) return sf;
        *bytes = from_m4_layout(p).total;
        return HOS_OK;
    }
    if (p && p->segment_overlap != 0) {
        hos_status so = check_params(p, op);
        if (so != HOS_OK) return so;
        const OverlapPlan o = overlap_plan(p, n_total);
        if (o.on) {
            size_t inner = 0;
            return overlap_workspace(op, n_total, p, o, &inner, bytes);
        }
        hos_params p2 = *p;
        p2.segment_overlap = 0;
        return hos_workspace_size(op, n_total, n_series, max_len, &p2, bytes);
    }
    if (op == HOS_OP_TRISPECTRUM_BACKWARD) {
        PlanB4 P4;
        hos_status s4 = make_planb4(p, n_total, P4);
        if (s4 != HOS_OK) return s4;
        *bytes = P4.total;
        return HOS_OK;
    }
    if (op == HOS_OP_TRISPECTRUM || op == HOS_OP_CUMULANT4 || op == HOS_OP_TRISPECTRUM_BATCHED ||
        op == HOS_OP_MOMENTS4_SLICE) {
        Plan4 P4;
        hos_status s4 = make_plan4(op, p, n_total, P4, n_series, max_len);
        if (s4 != HOS_OK) return s4;
        *bytes = P4.total;
        return HOS_OK;
    }
    if (op == HOS_OP_BISPECTRUM_BACKWARD) {
        PlanB PB;
        hos_status sb = make_planb(p, n_total, PB);
        if (sb != HOS_OK) return sb;
        *bytes = PB.total;
        return HOS_OK;
    }
    if (op == HOS_OP_SERIES_SUM) {
        *bytes = sum_ws_bytes(n_total);
        return HOS_OK;
    }
    if (op == HOS_OP_BISPECTRUM_FROM_C3) {
        hos_status sf = check_params(p, op);
        if (sf != HOS_OK) return sf;
        *bytes = from_c3_layout(p).total;
        return HOS_OK;
    }
    Plan P;
    hos_status s = make_plan(op, p, n_total, n_series, max_len, P);
    if (s != HOS_OK) return s;
    *bytes = P.l.total;
    return HOS_OK;
}

hos_status hos_series_sum(const void* d_x, int32_t dtype, int64_t n, double* d_sum, void* ws, size_t ws_bytes,
                          hos_stream_t stream) {
    if (!d_x || !d_sum || n < 1 || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < sum_ws_bytes(n) ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HOS_CUDA_TRY(launch_series_sum(d_x, dtype, n, sum_slices(n), at<int64_t>(ws, 0), at<double>(ws, 256), d_sum,
                                   st));
    return HOS_OK;
}

hos_status hos_cumulant3_slice(const void* d_x, int32_t dtype, int64_t n_slice, int64_t halo_before,
                               int64_t halo_after, const double* d_sum, int64_t n_total, const hos_params* p,
                               double* d_c3, void* ws, size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_c3 || !d_sum || !p || n_slice < 1 || (dtype != HOS_F32 && dtype != HOS_F64))
        return HOS_ERR_INVALID_ARG;
    if (halo_before < 0 || halo_after < 0 || halo_before > p->L || halo_after > p->L) return HOS_ERR_INVALID_ARG;
    if (n_total < n_slice + halo_before + halo_after || p->segment_len != 0) return HOS_ERR_INVALID_ARG;
    Plan P;
    hos_status s = make_plan(HOS_OP_CUMULANT3_SLICE, p, n_slice, 1, n_slice, P);
    if (s != HOS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    const SliceArgs sl{halo_before, halo_after, d_sum, n_total};
    s = run_c3(HOS_OP_CUMULANT3_SLICE, d_x, dtype, n_slice, nullptr, P, p, ws, ws_bytes, st, tr, 1, nullptr, d_c3,
               &sl);
    tr.mark("");
    return s;
}

hos_status hos_bispectrum_from_cumulant(const double* d_c3, const hos_params* p, void* d_B, void* ws,
                                        size_t ws_bytes, hos_stream_t stream) {
    if (!d_c3 || !d_B) return HOS_ERR_INVALID_ARG;
    hos_status s = check_params(p, HOS_OP_BISPECTRUM_FROM_C3);
    if (s != HOS_OK) return s;
    const FromC3Layout l = from_c3_layout(p);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < l.total ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    tr.mark("reduce");
    float* grid = at<float>(ws, l.grid);
    if (l.Nf > 2 * p->L) HOS_CUDA_TRY(launch_zero_f32(grid, (int64_t)l.Nf * l.Nf, st));
    HOS_CUDA_TRY(launch_window_c3(d_c3, p->L, p->window, l.Nf, kBispecScale, at<float>(ws, l.wtab), grid, st));
    tr.mark("transform");
    s = run_dft2(grid, reinterpret_cast<float2*>(d_B), 1, l.Nf, at<float2>(ws, l.tw), st);
    tr.mark("");
    return s;
}

hos_status hos_moments4_slice(const void* d_x, int32_t dtype, int64_t n_slice, int64_t halo_before, int64_t halo_after,
                              const double* d_sum, int64_t n_total, const hos_params* p, double* d_m4, double* d_c2,
                              void* ws, size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_m4 || !d_c2 || !d_sum || !p || n_slice < 1 || (dtype != HOS_F32 && dtype != HOS_F64))
        return HOS_ERR_INVALID_ARG;
    if (halo_before < 0 || halo_after < 0 || halo_before > p->L || halo_after > 2 * p->L) return HOS_ERR_INVALID_ARG;
    if (n_total < n_slice + halo_before + halo_after) return HOS_ERR_INVALID_ARG;
    Plan4 P;
    hos_status s = make_plan4(HOS_OP_MOMENTS4_SLICE, p, n_slice, P);
    if (s != HOS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    const SliceArgs sl{halo_before, halo_after, d_sum, n_total};
    s = run_c4(d_x, dtype, n_slice, P, p, ws, ws_bytes, st, tr, 2, d_m4, nullptr, &sl, d_c2);
    tr.mark("");
    return s;
}

hos_status hos_trispectrum_from_moments(const double* d_m4, const double* d_c2, const hos_params* p, void* d_T,
                                        void* ws, size_t ws_bytes, hos_stream_t stream) {
    if (!d_m4 || !d_c2 || !d_T) return HOS_ERR_INVALID_ARG;
    hos_status s = check_params(p, HOS_OP_TRISPECTRUM_FROM_MOMENTS);
    if (s != HOS_OK) return s;
    const FromM4Layout l = from_m4_layout(p);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < l.total ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    tr.mark("reduce");
    float* grid = at<float>(ws, l.grid);
    if (l.Nf > 2 * p->L) HOS_CUDA_TRY(launch_zero_f32(grid, (int64_t)l.Nf * l.Nf * l.Nf, st));
    C4ReduceArgs r;
    r.window = p->window;
    r.nfft = l.Nf;
    r.mode = 0;
    r.scale = 1.0 / (8.0 * 3.14159265358979323846 * 3.14159265358979323846 * 3.14159265358979323846);
    r.grid = grid;
    r.c4out = nullptr;
    HOS_CUDA_TRY(launch_c4_from_moments(d_m4, d_c2, p->L, r, st));
    tr.mark("transform");
    s = run_dft3(grid, reinterpret_cast<float2*>(d_T), l.Nf, at<float2>(ws, l.tw), st);
    tr.mark("");
    return s;
}

// ---- the direct method (Algorithm DBS) ----------------------------------------------
struct DirectLayout {
    int64_t K, step;
    size_t mean, y, F, tw, R, Cw, total;
};

static hos_status direct_layout(int64_t n, int32_t M, int32_t M3, int32_t overlap, DirectLayout& l) {
    if (n < 1 || M < 2 || M3 < 1 || M3 > M || overlap < 0 || overlap >= M) return HOS_ERR_INVALID_ARG;
    const bool pow2 = (M & (M - 1)) == 0;
    if ((pow2 && M > 8192) || (!pow2 && M > 2048)) return HOS_ERR_UNSUPPORTED;
    // a row and its wrap in shared memory (16 B per point) next to 16 KB of run totals
    if ((size_t)(M + M3 - 1) * 16 + 16 * 1024 > 227 * 1024) return HOS_ERR_UNSUPPORTED;
    l.step = M - overlap;
    l.K = n >= M ? (n - M) / l.step + 1 : 0;
    if (l.K < 1) return HOS_ERR_INVALID_ARG;
    if (l.K > (1 << 24)) return HOS_ERR_UNSUPPORTED;
    const size_t MM = (size_t)M * M;
    size_t o = 0;
    l.mean = o; o = al256(o + 8 * (size_t)l.K);
    l.y = o; o = al256(o + 4 * (size_t)l.K * M);
    l.F = o; o = al256(o + 8 * (size_t)l.K * M);
    l.tw = o; o = al256(o + 8 * (size_t)M);
    l.R = o; o = al256(o + 8 * MM);
    l.Cw = o; o = al256(o + 8 * MM);
    l.total = o;
    return HOS_OK;
}

hos_status hos_bispectrum_direct_workspace_size(int64_t n, int32_t M, int32_t M3, int32_t overlap, size_t* bytes) {
    if (!bytes) return HOS_ERR_INVALID_ARG;
    DirectLayout l;
    hos_status s = direct_layout(n, M, M3, overlap, l);
    if (s != HOS_OK) return s;
    *bytes = l.total;
    return HOS_OK;
}

hos_status hos_bispectrum_direct(const void* d_x, int32_t dtype, int64_t n, int32_t M, int32_t M3, int32_t overlap,
                                 int32_t remove_mean, void* d_B, void* ws, size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_B || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    DirectLayout l;
    hos_status s = direct_layout(n, M, M3, overlap, l);
    if (s != HOS_OK) return s;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < l.total ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    tr.mark("prep");
    float* y = at<float>(ws, l.y);
    float2* F = at<float2>(ws, l.F);
    float2* tw = at<float2>(ws, l.tw);
    HOS_CUDA_TRY(launch_part_prep(d_x, dtype, l.K, M, l.step, remove_mean ? 1 : 0, at<double>(ws, l.mean), y, st));
    tr.mark("transform");
    HOS_CUDA_TRY(launch_twiddles(M, tw, st));
    LineGeom g = line_geom(M, l.K, 1, M, 1);
    HOS_CUDA_TRY(launch_lines(true, y, F, g, tw, -1, 1.0f, st));
    tr.mark("smooth");
    HOS_CUDA_TRY(launch_direct_smooth(F, (int)l.K, M, M3, at<float2>(ws, l.R), at<float2>(ws, l.Cw),
                                      reinterpret_cast<float2*>(d_B), st));
    tr.mark("");
    g_last_contraction = "direct_triple_product";
    return HOS_OK;
}

static hos_status bispectrum_core(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, void* d_B, void* ws,
                                  size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_B || n < 1 || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    Plan P;
    hos_status s = make_plan(HOS_OP_BISPECTRUM, p, n, 1, n, P);
    if (s != HOS_OK) return s;
    if (!ws || ws_bytes < P.l.total || fault_is("workspace")) return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    s = run_c3(HOS_OP_BISPECTRUM, d_x, dtype, n, nullptr, P, p, ws, ws_bytes, st, tr, 0, at<float>(ws, P.l.grid),
               nullptr);
    if (s != HOS_OK) return s;
    tr.mark("transform");
    s = run_dft2(at<float>(ws, P.l.grid), reinterpret_cast<float2*>(d_B), 1, P.Nf, at<float2>(ws, P.l.tw), st);
    tr.mark("");
    return s;
}

hos_status hos_bispectrum_batched(const void* d_x, int32_t dtype, const int64_t* d_offsets, int32_t S,
                                  int64_t n_total, int64_t max_len, const hos_params* p, void* d_B, void* ws,
                                  size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_B || !d_offsets || S < 1 || n_total < 0 || max_len < 0 || (dtype != HOS_F32 && dtype != HOS_F64))
        return HOS_ERR_INVALID_ARG;
    Plan P;
    hos_status s = make_plan(HOS_OP_BISPECTRUM_BATCHED, p, n_total, S, max_len, P);
    if (s != HOS_OK) return s;
    if (!ws || ws_bytes < P.l.total || fault_is("workspace")) return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    s = run_c3(HOS_OP_BISPECTRUM_BATCHED, d_x, dtype, n_total, d_offsets, P, p, ws, ws_bytes, st, tr, 0,
               at<float>(ws, P.l.grid), nullptr);
    if (s != HOS_OK) return s;
    tr.mark("transform");
    s = run_dft2(at<float>(ws, P.l.grid), reinterpret_cast<float2*>(d_B), S, P.Nf, at<float2>(ws, P.l.tw), st);
    tr.mark("");
    return s;
}

static hos_status cumulant3_core(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, void* out, void* ws,
                                 size_t ws_bytes, hos_stream_t stream) {
    double* d_c3 = static_cast<double*>(out);
    if (!d_x || !d_c3 || n < 1 || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    Plan P;
    hos_status s = make_plan(HOS_OP_CUMULANT3, p, n, 1, n, P);
    if (s != HOS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    s = run_c3(HOS_OP_CUMULANT3, d_x, dtype, n, nullptr, P, p, ws, ws_bytes, st, tr, 1, nullptr, d_c3);
    tr.mark("");
    return s;
}

static hos_status trispectrum_core(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, void* d_T,
                                   void* ws, size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_T || n < 1 || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    Plan4 P;
    hos_status s = make_plan4(HOS_OP_TRISPECTRUM, p, n, P);
    if (s != HOS_OK) return s;
    if (!ws || ws_bytes < P.total || fault_is("workspace")) return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    s = run_c4(d_x, dtype, n, P, p, ws, ws_bytes, st, tr, 0, nullptr);
    if (s != HOS_OK) return s;
    tr.mark("transform");
    s = run_dft3(at<float>(ws, P.grid), reinterpret_cast<float2*>(d_T), P.Nf, at<float2>(ws, P.tw), st);
    tr.mark("");
    return s;
}

hos_status hos_trispectrum_batched(const void* d_x, int32_t dtype, const int64_t* d_offsets, int32_t S,
                                   int64_t n_total, int64_t max_len, const hos_params* p, void* d_T, void* ws,
                                   size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_T || !d_offsets || S < 1 || n_total < 0 || max_len < 0 || (dtype != HOS_F32 && dtype != HOS_F64))
        return HOS_ERR_INVALID_ARG;
    Plan4 P;
    hos_status s = make_plan4(HOS_OP_TRISPECTRUM_BATCHED, p, n_total, P, S, max_len);
    if (s != HOS_OK) return s;
    if (!ws || ws_bytes < P.total || fault_is("workspace")) return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    s = run_c4(d_x, dtype, n_total, P, p, ws, ws_bytes, st, tr, 0, nullptr, d_offsets);
    if (s != HOS_OK) return s;
    tr.mark("transform");
    s = run_dft3(at<float>(ws, P.grid), reinterpret_cast<float2*>(d_T), P.Nf, at<float2>(ws, P.tw), st, P.S);
    tr.mark("");
    return s;
}

static hos_status cumulant4_core(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, void* out, void* ws,
                                 size_t ws_bytes, hos_stream_t stream) {
    double* d_c4 = static_cast<double*>(out);
    if (!d_x || !d_c4 || n < 1 || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    Plan4 P;
    hos_status s = make_plan4(HOS_OP_CUMULANT4, p, n, P);
    if (s != HOS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    s = run_c4(d_x, dtype, n, P, p, ws, ws_bytes, st, tr, 1, d_c4);
    tr.mark("");
    return s;
}
hos_status hos_bispectrum(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, void* d_B, void* ws,
                          size_t ws_bytes, hos_stream_t stream) {
    return with_overlap(HOS_OP_BISPECTRUM, d_x, dtype, n, p, d_B, ws, ws_bytes, stream, bispectrum_core);
}

hos_status hos_cumulant3(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, double* d_c3, void* ws,
                         size_t ws_bytes, hos_stream_t stream) {
    return with_overlap(HOS_OP_CUMULANT3, d_x, dtype, n, p, d_c3, ws, ws_bytes, stream, cumulant3_core);
}

hos_status hos_trispectrum(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, void* d_T, void* ws,
                           size_t ws_bytes, hos_stream_t stream) {
    return with_overlap(HOS_OP_TRISPECTRUM, d_x, dtype, n, p, d_T, ws, ws_bytes, stream, trispectrum_core);
}

hos_status hos_cumulant4(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, double* d_c4, void* ws,
                         size_t ws_bytes, hos_stream_t stream) {
    return with_overlap(HOS_OP_CUMULANT4, d_x, dtype, n, p, d_c4, ws, ws_bytes, stream, cumulant4_core);
}

hos_status hos_bispectrum_backward(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, const void* d_dB,
                                   void* d_dx, void* ws, size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_dB || !d_dx || n < 1 || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    PlanB P;
    hos_status s = make_planb(p, n, P);
    if (s != HOS_OK) return s;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < P.total ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    int64_t* off = at<int64_t>(ws, P.off);
    int64_t* pad = at<int64_t>(ws, P.pad);
    float* y32 = at<float>(ws, P.y32);
    const int L = p->L, Nf = P.Nf;
    tr.mark("prep");
    HOS_CUDA_TRY(launch_plan_series(0, n, 0, nullptr, 1, L, 1, 1, 16, KC, P.g.pad_tail, off, pad,
                                    at<int64_t>(ws, P.unit), at<int64_t>(ws, P.win), st));
    HOS_CUDA_TRY(launch_mean(d_x, dtype, off, 1, P.nslices, at<double>(ws, P.mpart), p->remove_mean,
                             at<double>(ws, P.mean), st));
    int bx = (int)ceil_div((int64_t)L + n + KC + P.g.pad_tail + 64, 256 * 4);
    if (bx > 65535) bx = 65535;
    void* hi = P.tc ? at<void>(ws, P.hi) : nullptr;
    void* lo = P.tc ? at<void>(ws, P.lo) : nullptr;
    // split FP16: sc = {series scale, Gs scale} (powers of two), the series' now
    const bool f16 = P.tc && p->precision == HOS_PREC_SPLIT_FP16;
    float* sc = f16 ? at<float>(ws, P.sc) : nullptr;
    if (f16)
        HOS_CUDA_TRY(launch_series_scale(d_x, dtype, off, at<double>(ws, P.mean), 1, P.nslices, 0, 0, FP16_TOP3,
                                         at<unsigned>(ws, P.smx), sc, st));
    HOS_CUDA_TRY(launch_planes(d_x, dtype, off, pad, at<double>(ws, P.mean), L, P.tc ? plane_split(p->precision) : 0,
                               y32, hi, lo, 1, bx, st, 0, 0, sc));
    tr.mark("transform");
    float2* tw = at<float2>(ws, P.tw);
    float2* gc = at<float2>(ws, P.gc);
    HOS_CUDA_TRY(launch_twiddles(Nf, tw, st));
    LineGeom g1 = line_geom(Nf, Nf, 1, Nf, 1);
    HOS_CUDA_TRY(launch_lines(false, d_dB, gc, g1, tw, +1, 1.0f, st));
    LineGeom g2 = line_geom(Nf, Nf, Nf, (int64_t)Nf * Nf, Nf);
    HOS_CUDA_TRY(launch_lines(false, gc, gc, g2, tw, +1, 1.0f, st));
    tr.mark("contract");
    // y(i) of the single series sits at pad[0] + L + i; pad[0] = 0 for one series
    const float* yS = y32 + L;
    const double scale = 1.0 / (4.0 * 3.14159265358979323846 * 3.14159265358979323846 * (double)n);
    float* g = at<float>(ws, P.gbuf);
    if (P.tc) {
        HOS_CUDA_TRY(launch_gs(gc, Nf, L, p->window, scale, at<float>(ws, P.gs), st));
        if (f16)
            HOS_CUDA_TRY(launch_flat_scale(at<float>(ws, P.gs), (int64_t)4 * L * L, FP16_TOP3,
                                           at<unsigned>(ws, P.smx) + 1, sc + 1, st));
        HOS_CUDA_TRY(launch_adjoint_tc(y32, reinterpret_cast<const uint16_t*>(hi), reinterpret_cast<const uint16_t*>(lo),
                                       n, L, at<float>(ws, P.gs), at<uint8_t>(ws, P.gsb), at<float>(ws, P.t1),
                                       at<float>(ws, P.t2p), g, at<int>(ws, P.status), wait_limit_ns(), sm_count(),
                                       st, f16 ? FMT_F16 : FMT_BF16, sc));
        g_last_contraction = f16 ? "adjoint_tcgen05_split_fp16" : "adjoint_tcgen05_split_bf16";
    } else {
        HOS_CUDA_TRY(launch_adjoint(yS, n, L, gc, Nf, p->window, scale, at<float>(ws, P.gs), at<float>(ws, P.t1),
                                    at<float>(ws, P.t2p), g, st));
        g_last_contraction = "adjoint_simt_fp32";
    }
    tr.mark("reduce");
    HOS_CUDA_TRY(launch_mean(g, HOS_F32, off, 1, P.nslices, at<double>(ws, P.gmpart), p->remove_mean,
                             at<double>(ws, P.gmean), st));
    HOS_CUDA_TRY(launch_adjoint_finish(g, n, at<double>(ws, P.gmean), p->remove_mean, dtype, d_dx, st));
    tr.mark("");
    return HOS_OK;
}

hos_status hos_trispectrum_backward(const void* d_x, int32_t dtype, int64_t n, const hos_params* p, const void* d_dT,
                                    void* d_dx, void* ws, size_t ws_bytes, hos_stream_t stream) {
    if (!d_x || !d_dT || !d_dx || n < 1 || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    PlanB4 P;
    hos_status s = make_planb4(p, n, P);
    if (s != HOS_OK) return s;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < P.total ||
        fault_is("workspace"))
        return HOS_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Tracer tr(st);
    int64_t* off = at<int64_t>(ws, P.off);
    int64_t* pad = at<int64_t>(ws, P.pad);
    float* y32 = at<float>(ws, P.y32);
    const int L = p->L, Nf = P.Nf;
    tr.mark("prep");
    HOS_CUDA_TRY(launch_plan_series(0, n, 0, nullptr, 1, L, 1, 1, 16, KC, P.g.pad_tail, off, pad,
                                    at<int64_t>(ws, P.unit), at<int64_t>(ws, P.win), st));
    HOS_CUDA_TRY(launch_mean(d_x, dtype, off, 1, P.nslices, at<double>(ws, P.mpart), p->remove_mean,
                             at<double>(ws, P.mean), st));
    int bx = (int)ceil_div((int64_t)L + n + KC + P.g.pad_tail + 64, 256 * 4);
    if (bx > 65535) bx = 65535;
    void* hi = at<void>(ws, P.hi);
    void* lo = at<void>(ws, P.lo);
    const bool f16 = p->precision == HOS_PREC_SPLIT_FP16;
    float* sc = f16 ? at<float>(ws, P.sc) : nullptr;
    if (f16)
        HOS_CUDA_TRY(launch_series_scale(d_x, dtype, off, at<double>(ws, P.mean), 1, P.nslices, 0, 0, FP16_TOP3,
                                         at<unsigned>(ws, P.smx), sc, st));
    HOS_CUDA_TRY(launch_planes(d_x, dtype, off, pad, at<double>(ws, P.mean), L, plane_split(p->precision), y32, hi, lo,
                               1, bx, st, 0, 0, sc));
    double* c2 = at<double>(ws, P.c2);
    HOS_CUDA_TRY(launch_c2(y32, off, pad, 1, L, P.c2s, c2, at<float2>(ws, P.c2p), st));
    tr.mark("transform");
    // adjoint transform: Gc(w mod N) = sum_k G(k) e^{+i 2 pi k.w / N}, one axis at a time
    float2* tw = at<float2>(ws, P.tw);
    float2* gc = at<float2>(ws, P.gc);
    const int64_t N = Nf, N2 = N * N;
    HOS_CUDA_TRY(launch_twiddles(Nf, tw, st));
    LineGeom g3 = line_geom(Nf, N2, 1, N, 1);  // along k3 (contiguous)
    HOS_CUDA_TRY(launch_lines(false, d_dT, gc, g3, tw, +1, 1.0f, st));
    LineGeom g2 = line_geom(Nf, N2, N, N2, N);  // along k2
    HOS_CUDA_TRY(launch_lines(false, gc, gc, g2, tw, +1, 1.0f, st));
    LineGeom g1 = line_geom(Nf, N2, N2, N2 * N, N2);  // along k1
    HOS_CUDA_TRY(launch_lines(false, gc, gc, g1, tw, +1, 1.0f, st));
    tr.mark("contract");
    const double pi = 3.14159265358979323846;
    const double scale = 1.0 / (8.0 * pi * pi * pi * (double)n);
    float* gs4 = at<float>(ws, P.gs);
    double* gc2 = at<double>(ws, P.gc2);
    float* g = at<float>(ws, P.gbuf);
    HOS_CUDA_TRY(launch_gs4(gc, Nf, L, p->window, scale, gs4, st));
    HOS_CUDA_TRY(launch_gc2(gs4, c2, L, gc2, st));
    if (f16)
        HOS_CUDA_TRY(launch_flat_scale(gs4, (int64_t)8 * L * L * L, FP16_TOP3, at<unsigned>(ws, P.smx) + 1, sc + 1,
                                       st));
    HOS_CUDA_TRY(launch_adjoint4_tc(y32, reinterpret_cast<const uint16_t*>(hi), reinterpret_cast<const uint16_t*>(lo),
                                    n, L, gs4, at<uint8_t>(ws, P.gsb), at<float>(ws, P.t1), at<float>(ws, P.t2p), gc2,
                                    g, at<int>(ws, P.status), wait_limit_ns(), sm_count(), st,
                                    f16 ? FMT_F16 : FMT_BF16, sc));
    g_last_contraction = f16 ? "adjoint4_tcgen05_split_fp16" : "adjoint4_tcgen05_split_bf16";
    tr.mark("reduce");
    HOS_CUDA_TRY(launch_mean(g, HOS_F32, off, 1, P.nslices, at<double>(ws, P.gmpart), p->remove_mean,
                             at<double>(ws, P.gmean), st));
    HOS_CUDA_TRY(launch_adjoint_finish(g, n, at<double>(ws, P.gmean), p->remove_mean, dtype, d_dx, st));
    tr.mark("");
    return HOS_OK;
}

// Host mirror of a contraction plan: the series layout, every CTA's walk, the
// slots its parts write, the reduction's view of those slots and the bounds
// and alignment of every bulk copy, run on the CPU with the same code the
// kernels use (series_plan, Walk, tile_record, cta_slot_used).
hos_status hos_check_plan(int32_t op, int64_t n_total, int32_t n_series, const int64_t* h_offsets,
                          const hos_params* p, int32_t ctas, char* msg, size_t msg_len) {
    auto fail = [&](const char* fmt, long long a, long long b, long long c) {
        if (msg && msg_len) snprintf(msg, msg_len, fmt, a, b, c);
        return HOS_ERR_DEVICE_FAULT;
    };
    if (msg && msg_len) msg[0] = 0;
    if (!p || n_total < 0 || n_series < 1 || ctas < 0) return HOS_ERR_INVALID_ARG;
    C3Geom g;
    int S = 0, order = 3;
    int64_t seg = 0, plane_len = 0, n_slots = 0;
    if (op == HOS_OP_BISPECTRUM || op == HOS_OP_BISPECTRUM_BATCHED) {
        if (op == HOS_OP_BISPECTRUM_BATCHED && !h_offsets) return HOS_ERR_INVALID_ARG;
        int64_t max_len = n_total;
        if (op == HOS_OP_BISPECTRUM_BATCHED) {
            max_len = 0;
            for (int s = 0; s < n_series; ++s) {
                if (h_offsets[s + 1] < h_offsets[s]) return HOS_ERR_INVALID_ARG;
                if (h_offsets[s + 1] - h_offsets[s] > max_len) max_len = h_offsets[s + 1] - h_offsets[s];
            }
        }
        Plan P;
        hos_status st = make_plan(op, p, n_total, n_series, max_len, P);
        if (st != HOS_OK) return st;
        g = P.g;
        S = P.S;
        seg = P.seg;
        plane_len = P.l.plane_len;
        n_slots = P.l.slots;
    } else if (op == HOS_OP_TRISPECTRUM) {
        Plan4 P;
        hos_status st = make_plan4(op, p, n_total, P);
        if (st != HOS_OK) return st;
        if (!P.tc) return HOS_ERR_UNSUPPORTED;
        g = P.g4;
        S = P.S;
        seg = P.seg;
        order = 4;
        plane_len = P.plane_len;
        n_slots = P.slots;
    } else {
        return HOS_ERR_UNSUPPORTED;
    }
    if (ctas > 0) {  // another CTA count: the per-CTA slots follow it
        n_slots += ctas - g.G;
        g.G = ctas;
    }
    if (g.ntiles > MAX_TILES || g.ntiles < 1) return fail("tile count %lld outside 1..%lld", g.ntiles, MAX_TILES, 0);
    // the plan kernel's layout
    std::vector<int64_t> off(S + 1), pad(S + 1), unit(S + 1), win(S + 1), bnd(g.G + 1);
    int64_t cp = 0, cu = 0, cw = 0;
    for (int s = 0; s < S; ++s) {
        int64_t o0, o1;
        if (op == HOS_OP_BISPECTRUM_BATCHED) {
            o0 = h_offsets[s];
            o1 = h_offsets[s + 1];
        } else {
            o0 = seg ? s * seg : 0;
            o1 = seg ? ((s + 1) * seg < n_total ? (s + 1) * seg : n_total) : n_total;
        }
        const SeriesPlan sp = series_plan(o1 - o0, p->L, g.ntiles, g.ktot, g.flush, g.kc, g.pad_tail);
        off[s] = o0;
        pad[s] = cp;
        unit[s] = cu;
        win[s] = cw;
        cp += sp.plen;
        cu += sp.cost;
        cw += sp.wins;
    }
    off[S] = (op == HOS_OP_BISPECTRUM_BATCHED) ? h_offsets[S] : n_total;
    pad[S] = cp;
    unit[S] = cu;
    win[S] = cw;
    if (pad[S] > plane_len) return fail("planes need %lld samples, the workspace holds %lld", pad[S], plane_len, 0);
    for (int q = 0; q <= g.G; ++q) bnd[q] = range_begin(q, unit[S], g.G);
    const SeriesView sv{off.data(), pad.data(), unit.data(), win.data(), nullptr, S};
    const int elt = plane_elt(p->precision);
    // coverage of every (series, tile, chunk); the writer of every slot
    std::vector<int64_t> tile0(S * (int64_t)g.ntiles + 1, 0);
    for (int s = 0; s < S; ++s)
        for (int t = 0; t < g.ntiles; ++t)
            tile0[(int64_t)s * g.ntiles + t + 1] = tile0[(int64_t)s * g.ntiles + t] + ceil_div(off[s + 1] - off[s], g.kc);
    std::vector<uint8_t> seen(tile0.back(), 0);
    std::vector<int32_t> slot_part(n_slots, -1);
    std::vector<int64_t> part_st;  // (s * ntiles + t) of each part
    for (int cta = 0; cta < g.G; ++cta) {
        Walk w;
        w.init(g, sv, cta, g.G);
        Part pt;
        int mid_window = 0;
        while (w.next(pt)) {
            if (pt.s < 0 || pt.s >= S || pt.t < 0 || pt.t >= g.ntiles)
                return fail("CTA %lld: part outside the plan (series %lld, tile %lld)", cta, pt.s, pt.t);
            const int64_t nch = ceil_div(off[pt.s + 1] - off[pt.s], g.kc);
            if (!(0 <= pt.c0 && pt.c0 < pt.c1 && pt.c1 <= nch) || (pt.c1 - 1) / g.flush != pt.c0 / g.flush)
                return fail("CTA %lld: bad chunk range [%lld, %lld)", cta, pt.c0, pt.c1);
            const int64_t st_idx = (int64_t)pt.s * g.ntiles + pt.t;
            for (int64_t c = pt.c0; c < pt.c1; ++c) {
                if (seen[tile0[st_idx] + c]++) return fail("chunk %lld of (series, tile) %lld run twice (CTA %lld)", c,
                                                           st_idx, cta);
                // bulk copies of the tensor-core producer (plane and y windows)
                const int64_t i0 = c * g.kc;
                const int col0 = 32 * g.tile_c32[pt.t], wt = 32 * g.tile_w32[pt.t];
                const int64_t wb = pad[pt.s] + i0 + col0, wend = wb + g.kc + wt + 16;
                const int64_t ab = (order == 3) ? pad[pt.s] + i0 + (int64_t)g.tile_a[pt.t] * TILE_M : pad[pt.s] + i0;
                if (wend > pad[pt.s + 1] || ab + g.kc + TILE_M > pad[pt.s + 1])
                    return fail("series %lld chunk %lld: a window reads past the series' block (tile %lld)", pt.s, c,
                                pt.t);
                if (elt && ((wb * elt) % 16 != 0 || ((g.kc + wt + 16) * elt) % 16 != 0 || (ab * 4) % 16 != 0))
                    return fail("series %lld chunk %lld tile %lld: a bulk copy is not 16-byte aligned", pt.s, c, pt.t);
            }
            const int64_t nwin = ceil_div(nch, g.flush);
            const int64_t want = (pt.c0 % g.flush == 0) ? win[pt.s] + (int64_t)pt.t * nwin + pt.c0 / g.flush
                                                        : win[S] + cta;
            if (pt.slot != want || pt.slot < 0 || pt.slot >= n_slots)
                return fail("CTA %lld: part slot %lld, expected %lld", cta, pt.slot, want);
            if (pt.c0 % g.flush != 0 && ++mid_window > 1)
                return fail("CTA %lld: %lld parts start inside a window", cta, mid_window, 0);
            if (slot_part[pt.slot] >= 0) return fail("slot %lld written twice (CTA %lld)", pt.slot, cta, 0);
            slot_part[pt.slot] = (int32_t)part_st.size();
            part_st.push_back(st_idx);
        }
    }
    for (size_t q = 0; q < seen.size(); ++q)
        if (seen[q] != 1) return fail("chunk %lld of the plan run %lld times", (long long)q, seen[q], 0);
    // the reduction reads every part exactly once, from its own (series, tile)
    std::vector<uint8_t> read(part_st.size(), 0);
    for (int s = 0; s < S; ++s)
        for (int t = 0; t < g.ntiles; ++t) {
            const TileRec r = tile_record(g, sv, bnd.data(), s, t);
            const int64_t st_idx = (int64_t)s * g.ntiles + t;
            for (int f = 0; f < r.nwin; ++f) {
                const int32_t q = slot_part[r.slot + f];
                if (q < 0 || part_st[q] != st_idx) return fail("(series, tile) %lld window %lld: main slot %lld unset",
                                                               st_idx, f, r.slot + f);
                ++read[q];
            }
            for (int cta = r.xlo; cta < r.xhi; ++cta) {
                if (!cta_slot_used(r, bnd.data(), cta, g.flush)) continue;
                const int32_t q = slot_part[win[S] + cta];
                if (q < 0 || part_st[q] != st_idx)
                    return fail("(series, tile) %lld: CTA %lld slot holds no part of it", st_idx, cta, 0);
                ++read[q];
            }
        }
    for (size_t q = 0; q < read.size(); ++q)
        if (read[q] != 1) return fail("part %lld read %lld times by the reduction", (long long)q, read[q], 0);
    if (order == 3) {
        // every lag pair of the square gets its value from exactly one computed
        // element: under the swap plan itself or its mirror (the reduction's rule),
        // under the six-fold plans its one image in the fundamental set
        const int L = g.L;
        // computed elements by (row w1 + L, column w2 + L)
        const int nr = TILE_M * g.tiles_m;
        int nc = 0;
        for (int t = 0; t < g.ntiles; ++t)
            if (32 * (g.tile_c32[t] + g.tile_w32[t]) > nc) nc = 32 * (g.tile_c32[t] + g.tile_w32[t]);
        std::vector<uint8_t> cov((size_t)nr * nc, 0);
        for (int t = 0; t < g.ntiles; ++t)
            for (int r = TILE_M * g.tile_a[t]; r < TILE_M * (g.tile_a[t] + 1); ++r)
                for (int c = 32 * g.tile_c32[t]; c < 32 * (g.tile_c32[t] + g.tile_w32[t]); ++c)
                    cov[(size_t)r * nc + c] = 1;
        auto computed = [&](int w1, int w2) {
            const int r = w1 + L, c = w2 + L;
            return r >= 0 && r < nr && c >= 0 && c < nc && cov[(size_t)r * nc + c] != 0;
        };
        for (int w1 = -L; w1 < L; ++w1)
            for (int w2 = -L; w2 < L; ++w2) {
                int src = 0;
                if (g.sym == C3_SWAP) {
                    if (computed(w1, w2)) ++src;
                    else if (w2 + L < (int)g.row_c0[(w1 + L) / TILE_M] && computed(w2, w1)) ++src;
                    // a tile the band window weights by zero is left out (the grid is zeroed)
                    if (src == 0 && p->window == HOS_WIN_PARZEN_SYM &&
                        lag_window2(w1, w2, L, HOS_WIN_PARZEN_SYM) == 0.0)
                        continue;
                } else {
                    if (w1 == -L || w2 == -L) continue;  // zero weight: the edge the reduction zeroes
                    int o1[6], o2[6];
                    c3_orbit(w1, w2, o1, o2);
                    int reps = 0;
                    for (int k2 = 0; k2 < 6; ++k2) {
                        bool dup = false;  // an image met before (the orbit repeats on three lines)
                        for (int j = 0; j < k2; ++j) dup = dup || (o1[j] == o1[k2] && o2[j] == o2[k2]);
                        if (dup || !c3_fundamental(L, C3_SIX, o1[k2], o2[k2])) continue;
                        ++reps;
                        if (c3_fundamental(L, g.sym, o1[k2], o2[k2]) && computed(o1[k2], o2[k2])) ++src;
                    }
                    if (reps != 1) return fail("lag (%lld, %lld): %lld images in the fundamental set", w1, w2, reps);
                    // the unfold finds that image from the signs of the lags
                    int sb, sa;
                    c3_sector_image(w1, w2, sb, sa);
                    if (!c3_fundamental(L, C3_SIX, sb, sa))
                        return fail("lag (%lld, %lld): sector image (%lld, ...) outside the fundamental set", w1, w2, sb);
                    if (c3_fundamental(L, g.sym, sb, sa)) {
                        // the unfold's tile of that image: its row block's first tile plus
                        // whole tile widths from the block's first column
                        const int r = sb + L, blk = r / TILE_M, c = sa + L;
                        const int t = g.row_t0[blk] + (c - g.row_c0[blk]) / g.tile_n;
                        if (t < 0 || t >= g.ntiles || g.tile_a[t] != blk || c < 32 * g.tile_c32[t] ||
                            c >= 32 * (g.tile_c32[t] + g.tile_w32[t]))
                            return fail("lag (%lld, %lld): the unfold looks in tile %lld, which does not hold it", w1,
                                        w2, t);
                    }
                    if (g.sym == C3_SIX_BAND && src == 0) {
                        // weighted by zero: |w1 - w2|, |w1| or |w2| reaches L on its image
                        if (lag_window2(w1, w2, L, HOS_WIN_PARZEN_SYM) == 0.0) continue;
                    }
                }
                if (src != 1) return fail("lag (%lld, %lld) of the square has %lld sources", w1, w2, src);
            }
    }
    if (msg && msg_len)
        snprintf(msg, msg_len, "ok: %d series, %d tiles (cost %d per chunk), %d CTAs, %lld parts", S, g.ntiles,
                 g.ktot, g.G, (long long)part_st.size());
    return HOS_OK;
}

hos_status hos_get_device_status(const void* ws, int32_t* status) {
    if (!ws || !status) return HOS_ERR_INVALID_ARG;
    int v = 0;
    if (cudaMemcpy(&v, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HOS_ERR_CUDA;
    *status = v;
    return HOS_OK;
}

hos_status hos_reset_device_status(void* ws, hos_stream_t stream) {
    if (!ws) return HOS_ERR_INVALID_ARG;
    if (cudaMemsetAsync(ws, 0, sizeof(int), reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return HOS_ERR_CUDA;
    return HOS_OK;
}

hos_status hos_selftest_timeout(void* ws, size_t ws_bytes, int32_t timeout_us, hos_stream_t stream) {
    if (!ws || ws_bytes < 256 || timeout_us < 1) return HOS_ERR_INVALID_ARG;
    if (launch_timeout_selftest(reinterpret_cast<int*>(ws), (uint64_t)timeout_us * 1000ull,
                                reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return HOS_ERR_CUDA;
    return HOS_OK;
}

hos_status hos_set_profiling(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = enable != 0;
    return HOS_OK;
}

hos_status hos_get_stage_times(float* ms, int32_t max_stages, int32_t* n_stages) {
    if (!ms || !n_stages) return HOS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int n = g_prof_n - 1;
    if (n < 0) n = 0;
    if (n > max_stages) n = max_stages;
    const cudaEvent_t* ev = g_ev[g_prof_dev];
    for (int i = 0; i < n; ++i) {
        if (cudaEventSynchronize(ev[i + 1]) != cudaSuccess) return HOS_ERR_CUDA;
        if (cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]) != cudaSuccess) return HOS_ERR_CUDA;
    }
    *n_stages = n;
    return HOS_OK;
}

const char* hos_stage_name(int32_t i) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (i < 0 || i >= MAX_STAGES || i >= g_prof_n) return "";
    return g_cur_names[i] ? g_cur_names[i] : "";
}

}  // extern "C"
