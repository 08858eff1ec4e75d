// C ABI of the SG-splatting rasterizer: argument checks, workspace layout and
// the launch sequence of the forward and backward passes.
#include "sg_internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

using namespace sgk;

namespace {
std::atomic<int64_t> &launch_counter();
}

void sgk::count_launches(int n) { launch_counter() += n; }

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(SG_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define SG_CUDA(call, where)                                 \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);  \
    } while (0)

// ---------------------------------------------------------------------------
// stage profiler: CUDA events recorded on the caller's stream
// ---------------------------------------------------------------------------
enum Stage {
    ST_SETUP = 0, ST_PRE, ST_DEPTH_SORT, ST_OFFSETS, ST_READ_PAIRS, ST_DUPLICATE, ST_TILE_SORT,
    ST_RANGES, ST_BLEND_FWD, ST_BWD_CLEAR, ST_BLEND_BWD, ST_PRE_BWD, ST_N
};
static_assert(ST_N == SG_PROFILE_STAGES, "stage count");
const char *const kStageNames[ST_N] = {"setup", "preprocess", "depth_sort", "pair_offsets",
                                       "read_pairs", "duplicate", "tile_sort", "tile_ranges",
                                       "blend_fwd", "bwd_clear", "blend_bwd", "preprocess_bwd"};

struct Profiler {
    std::mutex mu;
    int flags = 0;
    uint32_t stage_mask = 0xFFFFFFFFu;
    std::vector<cudaEvent_t> pool;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double ms[ST_N] = {};
    int64_t launches[ST_N] = {};
    int64_t evals[2] = {};
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};
Profiler &prof() { static Profiler p; return p; }

std::atomic<int64_t> &launch_counter() {
    static std::atomic<int64_t> c{0};
    return c;
}

// Brackets one stage with events when profiling is on.
struct StageTimer {
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageTimer(int st, cudaStream_t stream) : stage(st), s(stream) {
        Profiler &p = prof();
        if (!(p.flags & SG_PROFILE_EVENTS) || !((p.stage_mask >> st) & 1u)) return;
        std::lock_guard<std::mutex> g(p.mu);
        a = p.get();
        if (a) cudaEventRecord(a, s);
    }
    ~StageTimer() {
        if (!a) return;
        Profiler &p = prof();
        std::lock_guard<std::mutex> g(p.mu);
        cudaEvent_t b = p.get();
        if (!b) return;
        cudaEventRecord(b, s);
        p.pending.push_back({stage, a, b});
    }
};

// Process-wide kernel shape choices (sg_set_tuning); defaults from measurement
// (1M Gaussians at 1920x1080: both blends persistent, 4 and 8 pixels per thread).
constexpr sg_tuning kDefaultTuning = {4, 8, 1, 1, 0, 0, 0, {0}};
constexpr int kDefaultBatch = 64;
sg_tuning &tuning() {
    static sg_tuning t = kDefaultTuning;
    return t;
}

bool ppt_ok(int p) { return p == 1 || p == 2 || p == 4 || p == 8; }

constexpr size_t ALIGN = 256;
size_t al(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool dtype_ok(int dg, int dl, int ds) {
    return (dg == SG_F32 && dl == SG_F32 && ds == SG_F32) ||
           (dg == SG_F16 && dl == SG_F16 && (ds == SG_F16 || ds == SG_BF16));
}

int tile_bits_for(uint64_t n_tiles) {
    if (n_tiles <= 1) return 0;
    int b = 0;
    while ((1ull << b) < n_tiles) ++b;
    return b;
}

// Fills the batch table from host structs. Pointers of the scenes are
// validated only when check_ptrs is set (the query does not need them).
int build_batch(const sg_scene *scenes, int n_scenes, const sg_camera *cams, const int32_t *view_scene,
                int n_views, bool check_ptrs, Batch &b) {
    if (!scenes || !cams) return fail(SG_ERR_INVALID_ARG, "scene and cameras must not be NULL");
    if (n_views < 1 || n_views > SG_MAX_VIEWS)
        return fail(SG_ERR_INVALID_ARG, "n_views = %d outside [1, %d]", n_views, SG_MAX_VIEWS);
    if (n_scenes < 1 || n_scenes > SG_MAX_SCENES)
        return fail(SG_ERR_INVALID_ARG, "n_scenes = %d outside [1, %d]", n_scenes, SG_MAX_SCENES);
    std::memset(&b, 0, sizeof(Batch));
    b.n_views = n_views;
    b.n_scenes = n_scenes;
    uint64_t bwd_blk = 0;
    for (int s = 0; s < n_scenes; ++s) {
        const sg_scene &sc = scenes[s];
        if (sc.n < 0 || sc.n > (int64_t)INT32_MAX - PRE_THREADS)
            return fail(SG_ERR_INVALID_ARG, "scene %d: n = %lld out of range", s, (long long)sc.n);
        if (sc.n_lobes < 0 || sc.n_lobes > (int64_t)INT32_MAX)
            return fail(SG_ERR_INVALID_ARG, "scene %d: n_lobes = %lld out of range", s, (long long)sc.n_lobes);
        if (!dtype_ok(sc.dtype_geom, sc.dtype_lobe, sc.dtype_sharp))
            return fail(SG_ERR_INVALID_ARG, "scene %d: unsupported dtype combination (%d, %d, %d)", s,
                        sc.dtype_geom, sc.dtype_lobe, sc.dtype_sharp);
        if (s > 0 && (sc.dtype_geom != scenes[0].dtype_geom || sc.dtype_lobe != scenes[0].dtype_lobe ||
                      sc.dtype_sharp != scenes[0].dtype_sharp || sc.color_model != scenes[0].color_model))
            return fail(SG_ERR_INVALID_ARG, "scene %d: all scenes of a call must share storage types and colour model",
                        s);
        const bool sh3 = sc.color_model == SG_COLOR_SH3;
        if (sc.color_model != SG_COLOR_SG && !sh3)
            return fail(SG_ERR_INVALID_ARG, "scene %d: unknown colour model %d", s, sc.color_model);
        if (sh3 && (sc.n_lobes != 0 || sc.dtype_geom != SG_F32))
            return fail(SG_ERR_INVALID_ARG, "scene %d: the SH3 colour model takes binary32 geometry and no lobes", s);
        if (check_ptrs && sc.n > 0) {
            const void *req_sg[] = {sc.means, sc.scales, sc.quats, sc.opac, sc.gmask, sc.c0, sc.lobe_off};
            const void *req_sh[] = {sc.means, sc.scales, sc.quats, sc.opac, sc.gmask, sc.sh, sc.sh};
            for (const void *p : (sh3 ? req_sh : req_sg))
                if (!p || !aligned(p, 16))
                    return fail(SG_ERR_INVALID_ARG, "scene %d: a Gaussian array is NULL or not 16-byte aligned", s);
        }
        if (check_ptrs && sc.n_lobes > 0) {
            const void *req[] = {sc.axis, sc.sharp, sc.amp, sc.lmask};
            for (const void *p : req)
                if (!p || !aligned(p, 16))
                    return fail(SG_ERR_INVALID_ARG, "scene %d: a lobe array is NULL or not 16-byte aligned", s);
        }
        SceneDesc &d = b.scene[s];
        d.means = sc.means; d.scales = sc.scales; d.quats = sc.quats; d.opac = sc.opac;
        d.gmask = sc.gmask; d.c0 = sc.c0; d.lobe_off = sc.lobe_off;
        d.axis = sc.axis; d.sharp = sc.sharp; d.amp = sc.amp; d.lmask = sc.lmask;
        d.sh = sc.sh;
        d.color_model = sc.color_model;
        d.n = sc.n; d.n_lobes = sc.n_lobes;
        d.dtype_geom = sc.dtype_geom; d.dtype_lobe = sc.dtype_lobe; d.dtype_sharp = sc.dtype_sharp;
        d.blk_off = (uint32_t)bwd_blk;
        bwd_blk += div_up((uint64_t)sc.n, PRE_THREADS);
    }
    uint64_t tiles = 0, pix = 0, ent = 0;
    for (int v = 0; v < n_views; ++v) {
        const sg_camera &c = cams[v];
        const int s = view_scene ? view_scene[v] : 0;
        if (s < 0 || s >= n_scenes) return fail(SG_ERR_INVALID_ARG, "view %d: scene index %d", v, s);
        if (c.width < 1 || c.height < 1 || c.width > 16 * 65535 || c.height > 16 * 65535)
            return fail(SG_ERR_INVALID_ARG, "view %d: bad image size %dx%d", v, c.width, c.height);
        if (!(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.fx) || !std::isfinite(c.fy) ||
            !std::isfinite(c.cx) || !std::isfinite(c.cy) || !(c.near_plane >= 0.f))
            return fail(SG_ERR_INVALID_ARG, "view %d: bad intrinsics", v);
        for (int i = 0; i < 12; ++i)
            if (!std::isfinite(c.viewmat[i])) return fail(SG_ERR_INVALID_ARG, "view %d: non-finite viewmat", v);
        ViewDesc &d = b.view[v];
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        std::memcpy(d.V, c.viewmat, sizeof(d.V));
        // camera centre -R^T t (FP64 on the host)
        for (int i = 0; i < 3; ++i) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc -= (double)c.viewmat[4 * k + i] * (double)c.viewmat[4 * k + 3];
            d.campos[i] = (float)acc;
        }
        d.near_plane = c.near_plane;
        d.bg[0] = c.bg[0]; d.bg[1] = c.bg[1]; d.bg[2] = c.bg[2];
        d.W = c.width; d.H = c.height;
        d.tiles_x = (c.width + TILE - 1) / TILE;
        d.tiles_y = (c.height + TILE - 1) / TILE;
        d.scene = s;
        d.n = (int32_t)scenes[s].n;
        d.tile_off = (uint32_t)tiles;
        d.pix_off = pix;
        d.ent_off = ent;
        tiles += (uint64_t)d.tiles_x * d.tiles_y;
        pix += (uint64_t)c.width * c.height;
        ent += (uint64_t)scenes[s].n;
    }
    if (tiles >= (1ull << 31)) return fail(SG_ERR_INVALID_ARG, "too many tiles (%llu)", (unsigned long long)tiles);
    if (ent >= (1ull << 32) - 1)
        return fail(SG_ERR_INVALID_ARG, "too many (view, Gaussian) entries (%llu)", (unsigned long long)ent);
    if (bwd_blk >= (1ull << 31)) return fail(SG_ERR_INVALID_ARG, "too many blocks");
    b.n_tiles = (uint32_t)tiles;
    b.n_entries = ent;
    b.scene_blocks = (uint32_t)bwd_blk;
    uint32_t per_scene[SG_MAX_SCENES] = {};
    b.max_views_per_scene = 0;
    for (int v = 0; v < n_views; ++v) {
        const uint32_t c = ++per_scene[b.view[v].scene];
        b.max_views_per_scene = c > b.max_views_per_scene ? c : b.max_views_per_scene;
    }
    return SG_OK;
}

uint64_t n_pixels_of(const Batch &b) {
    uint64_t p = 0;
    for (int v = 0; v < b.n_views; ++v) p += (uint64_t)b.view[v].W * b.view[v].H;
    return p;
}

WsLayout make_layout(const Batch &b, uint64_t cap) {
    WsLayout L{};
    const uint64_t M = b.n_entries, T = b.n_tiles;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
    L.batch = take(sizeof(Batch));
    L.counters = take(CNT_N * sizeof(uint64_t));
    L.rec = take(M * sizeof(Rec));
    L.tiles_touched = take(M * 4);
    L.rect = take(M * 8);
    L.clamp = take(M);
    L.dup_flags = take(div_up(M, 256) * 8 + 8);   // the duplicate blocks' look-back words
    L.ranges = take(T * 8);
    L.order = take(T * 4);   // tile order of the persistent blends (forward and backward)
    L.order_scratch = take(TILE_ORDER_WORDS * 4);
    L.fixed_end = o;
    L.tile_bits = tile_bits_for(T);
    L.tile_passes = radix_passes(L.tile_bits);
    // the tile sort counts where one chunk's tile counters fit shared memory
    L.tile_counting = T >= 1 && T <= TC_MAX_TILES;
    L.tc_chunks = L.tile_counting ? tc_chunks(cap) : 0u;
    // Pairs: region A receives the duplicate's (tile, entry) pairs, region B the
    // tile sort's first output, and radix passes alternate between them; the
    // counting sort writes only the sorted entries, into B. The depth sort's
    // four buffers live in B: B is first written by the tile sort, after the
    // duplicate has read the depth order. The backward reads only the final
    // entries (B when counting, else A after an even number of passes, B after
    // an odd one).
    const size_t pairs4 = al(cap * 4), m4 = al(M * 4);
    // (the counting sort's keys are 16-bit)
    const size_t A = take(L.tile_counting ? al(cap * 2) + pairs4 : 2 * pairs4);
    const size_t B = take(std::max((L.tile_counting ? 1 : 2) * pairs4, 4 * m4));
    L.dkey0 = B;
    L.dval0 = B + m4;
    L.dkey1 = B + 2 * m4;
    L.dval1 = B + 3 * m4;
    if (L.tile_counting) {
        L.pkey_final = NO_OFFSET;
        L.pval_final = B;
        L.pkey_tmp = A;
        L.pval_tmp = A + al(cap * 2);
    } else {
        const size_t fin = L.tile_passes % 2 == 1 ? B : A, tmp = fin == A ? B : A;
        L.pkey_final = fin;
        L.pval_final = fin + pairs4;
        L.pkey_tmp = tmp;
        L.pval_tmp = tmp + pairs4;
    }
    // look-back flags of the depth sort's 4 passes, then those of the tile
    // sort's radix passes or the counting sort's [chunks][row] count matrix
    const uint64_t tile_words = L.tile_counting ? (uint64_t)L.tc_chunks * tc_row(T)
                                                : (uint64_t)L.tile_passes * div_up(cap, RS_TILE) * RS_RADIX;
    const uint64_t flag_words = std::max<uint64_t>(4 * div_up(M, RS_TILE) * RS_RADIX, tile_words);
    L.hist = take(flag_words * 4);
    L.scan_sums = take(SORT_AUX_BYTES);   // the depth sort's aux
    L.aux_tile = take(SORT_AUX_BYTES);
    L.total = o;
    L.M = M;
    L.n_tiles = T;
    L.cap = cap;
    return L;
}

uint64_t capacity_for(const Batch &b, size_t ws_bytes) {
    if (make_layout(b, 0).total > ws_bytes) return UINT64_MAX;   // not even the fixed part
    uint64_t lo = 0, hi = (1ull << 32) - 1;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        if (make_layout(b, mid).total <= ws_bytes) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Backward scratch: batch table, counters and the [9][M] 2D gradients (the
// persistent backward takes its tile order from the forward's workspace).
struct BwdLayout {
    size_t batch, counters, dg, total;
};

BwdLayout bwd_layout(const Batch &b) {
    BwdLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
    L.batch = take(sizeof(Batch));
    L.counters = take(CNT_N * sizeof(uint64_t));
    L.dg = take(9 * b.n_entries * sizeof(float));
    L.total = o;
    return L;
}

size_t bwd_bytes(const Batch &b) { return bwd_layout(b).total; }

// Blend shape of this call: pixels per thread from the tuning, and for the
// persistent form the resident grid, the work counter and the tile order.
int blend_shape(bool backward, const uint32_t *order, uint32_t *queue, BlendShape &sh) {
    const sg_tuning &t = tuning();
    sh.pixels_per_thread = backward ? t.bwd_pixels_per_thread : t.fwd_pixels_per_thread;
    sh.persistent = (backward ? t.bwd_persistent : t.fwd_persistent) != 0;
    sh.tile_order = sh.persistent ? order : nullptr;
    sh.queue = queue;
    const int nb = backward ? t.bwd_batch : t.fwd_batch;
    sh.batch = nb ? nb : kDefaultBatch;
    sh.grid = sh.persistent ? blend_persistent_grid(backward, sh.pixels_per_thread, sh.batch) : 0;
    if (sh.persistent && sh.grid <= 0)
        return fail(SG_ERR_CUDA, "persistent blend: occupancy query failed");
    return SG_OK;
}

void fill_sizes(const Batch &b, const WsLayout &L, uint64_t n_pairs, sg_sizes *out) {
    if (!out) return;
    out->n_entries = b.n_entries;
    out->n_tiles = b.n_tiles;
    out->n_pixels = n_pixels_of(b);
    out->n_pairs = n_pairs;
    out->pair_capacity = L.cap;
    out->ws_fixed_bytes = make_layout(b, 0).total;
    // pair buffers (32-bit keys and entries twice; the counting sort's 16-bit
    // keys and entries, then the sorted entries), plus the radix passes'
    // look-back words or, below the counting sort's chunk limit, its count
    // matrix rows
    out->ws_per_pair_bytes = L.tile_counting ? 10 + div_up(4 * tc_row(b.n_tiles), TC_CHUNK_TARGET) : 17;
    out->ws_bytes = L.total;
    out->bwd_ws_bytes = bwd_bytes(b);
}

// Per-thread pinned host words, mapped into the device, and an event for the
// plain form's read of the pair count: the scan's spine kernel stores the count
// and the depth sort's status there, and the host waits on the event after it.
struct CountReadback {
    uint64_t *host = nullptr;     // [0] pairs, [1] status
    uint64_t *dev_ptr = nullptr;  // the same words as the current device sees them
    cudaEvent_t ev = nullptr;
    int device = -1;
};

static cudaError_t count_readback(CountReadback *&out) {
    thread_local CountReadback rb;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!rb.host) {
        void *p = nullptr;
        e = cudaHostAlloc(&p, 64, cudaHostAllocPortable | cudaHostAllocMapped);
        if (e != cudaSuccess) return e;
        rb.host = static_cast<uint64_t *>(p);
    }
    if (!rb.ev || rb.device != dev) {
        if (rb.ev) cudaEventDestroy(rb.ev);
        rb.ev = nullptr;
        e = cudaEventCreateWithFlags(&rb.ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        void *dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, rb.host, 0);
        if (e != cudaSuccess) return e;
        rb.dev_ptr = static_cast<uint64_t *>(dp);
        rb.device = dev;
    }
    out = &rb;
    return cudaSuccess;
}

// Both forms queue the whole forward at once with grids sized by the pair
// capacity; the pair count stays on the device, which handles an overflow
// (no pairs are written, every tile list is empty). sync = true: the plain
// form also copies the count to the host behind an event and waits for that
// copy alone after queueing everything, to return SG_ERR_CAPACITY (or the
// depth sort's SG_ERR_TIMEOUT) and the count. sync = false: the batched form
// (overflow recorded in the device status, graph capturable).
int forward_impl(const sg_scene *scenes, int n_scenes, const sg_camera *cams, const int32_t *view_scene,
                 int n_views, void *ws, size_t ws_bytes, float *img, float *T_final, int32_t *last,
                 float *const *importance, sg_sizes *out, cudaStream_t stream, bool sync) {
    std::unique_ptr<Batch> hb(new Batch);
    int st = build_batch(scenes, n_scenes, cams, view_scene, n_views, true, *hb);
    if (st != SG_OK) return st;
    Batch &b = *hb;
    bool want_importance = false;
    if (importance) {
        for (int s = 0; s < n_scenes; ++s) {
            if (scenes[s].n > 0 && (!importance[s] || !aligned(importance[s], 4)))
                return fail(SG_ERR_INVALID_ARG, "importance[%d] is NULL or misaligned", s);
            b.scene[s].importance = importance[s];
            want_importance = want_importance || scenes[s].n > 0;
        }
    }
    if (!img || !T_final || !last) return fail(SG_ERR_INVALID_ARG, "output pointers must not be NULL");
    if (!aligned(img, 16) || !aligned(T_final, 16) || !aligned(last, 16))
        return fail(SG_ERR_INVALID_ARG, "outputs must be 16-byte aligned");
    if (!ws || !aligned(ws, ALIGN)) return fail(SG_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    const uint64_t cap = capacity_for(b, ws_bytes);
    if (cap == UINT64_MAX) {
        WsLayout L0 = make_layout(b, 0);
        fill_sizes(b, L0, 0, out);
        return fail(SG_ERR_WORKSPACE, "workspace of %zu bytes is below the fixed part (%zu bytes)", ws_bytes,
                    L0.total);
    }
    const WsLayout L = make_layout(b, cap);
    char *w = static_cast<char *>(ws);
    Batch *db = reinterpret_cast<Batch *>(w + L.batch);
    uint64_t *counters = reinterpret_cast<uint64_t *>(w + L.counters);
    Rec *rec = reinterpret_cast<Rec *>(w + L.rec);
    uint32_t *tt = reinterpret_cast<uint32_t *>(w + L.tiles_touched);
    uint2 *rect = reinterpret_cast<uint2 *>(w + L.rect);
    uint32_t *dkey0 = reinterpret_cast<uint32_t *>(w + L.dkey0);
    uint32_t *dval0 = reinterpret_cast<uint32_t *>(w + L.dval0);
    uint32_t *dkey1 = reinterpret_cast<uint32_t *>(w + L.dkey1);
    uint32_t *dval1 = reinterpret_cast<uint32_t *>(w + L.dval1);
    uint64_t *dup_flags = reinterpret_cast<uint64_t *>(w + L.dup_flags);
    uint2 *ranges = reinterpret_cast<uint2 *>(w + L.ranges);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + L.hist);
    uint64_t *sums = reinterpret_cast<uint64_t *>(w + L.scan_sums);
    const uint64_t M = L.M;

    const bool counting = (prof().flags & SG_PROFILE_COUNT) != 0;
    uint64_t *aux_tile = reinterpret_cast<uint64_t *>(w + L.aux_tile);
    {
        // the setup kernel also marks every tile range empty and clears both sorts' scratch
        ZeroRegions z;
        z.ptr[0] = reinterpret_cast<uint32_t *>(ranges);
        z.words[0] = 2 * L.n_tiles;
        z.even[0] = RANGE_EMPTY;
        z.ptr[1] = reinterpret_cast<uint32_t *>(sums);
        z.words[1] = SORT_AUX_BYTES / 4;
        z.ptr[2] = reinterpret_cast<uint32_t *>(aux_tile);
        z.words[2] = SORT_AUX_BYTES / 4;
        z.ptr[3] = reinterpret_cast<uint32_t *>(dup_flags);
        z.words[3] = 2 * div_up(M, 256);
        z.ptr[4] = reinterpret_cast<uint32_t *>(w + L.order_scratch);
        z.words[4] = TILE_ORDER_WORDS;
        StageTimer t(ST_SETUP, stream);
        SG_CUDA(launch_setup(b, db, counters, stream, z), "setup");
    }
    {
        StageTimer t(ST_PRE, stream);
        SG_CUDA(launch_preprocess(b, db, rec, tt, rect, dkey0, dval0, reinterpret_cast<uint8_t *>(w + L.clamp),
                                  stream),
                "preprocessSG");
    }
    {
        // depth digits, once per entry (result back in dkey0/dval0 after 4 passes)
        StageTimer t(ST_DEPTH_SORT, stream);
        // entries that reach no tile carry the drop key and are left out of the order
        SG_CUDA(launch_radix_sort(dkey0, dval0, dkey1, dval1, counters + CNT_ENTRIES, M, 32, hist, sums,
                                  stream, counters + CNT_STATUS, counters + CNT_VISIBLE, true),
                "depth sort");
    }
    CountReadback *rb = nullptr;   // plain form: where the duplicate leaves the pair count for the host
    if (sync) SG_CUDA(count_readback(rb), "pair count readback");
    // grids sized by the capacity (at most SORT_MAX_KEYS pairs); counts read on the device
    const uint64_t cap_dev = std::min<uint64_t>(cap, SORT_MAX_KEYS);
    uint64_t K = cap_dev;
    // duplicate into the buffer from which the tile sort ends in *_final: the
    // counting sort and an odd number of radix passes write the other buffer
    uint32_t *pk_final = L.tile_counting ? nullptr : reinterpret_cast<uint32_t *>(w + L.pkey_final);
    uint32_t *pv_final = reinterpret_cast<uint32_t *>(w + L.pval_final);
    uint32_t *pk_tmp = reinterpret_cast<uint32_t *>(w + L.pkey_tmp);
    uint32_t *pv_tmp = reinterpret_cast<uint32_t *>(w + L.pval_tmp);
    const bool dup_final = !L.tile_counting && (L.tile_passes % 2) == 0;
    uint32_t *k0 = dup_final ? pk_final : pk_tmp, *v0 = dup_final ? pv_final : pv_tmp;
    uint32_t *k1 = dup_final ? pk_tmp : pk_final, *v1 = dup_final ? pv_tmp : pv_final;
    {
        StageTimer t(ST_DUPLICATE, stream);
        // radix: also the tile sort's digit histograms and cleared look-back flags
        // the pair offsets come from the duplicate blocks' own look-back (no scan kernel)
        const int hp = L.tile_counting ? 0 : L.tile_passes;
        SG_CUDA(launch_duplicate(db, M, dval0, tt, rect, rec, counters, cap_dev, k0, v0, dup_flags,
                                 rb ? rb->dev_ptr : nullptr, stream, hp, hp ? aux_tile : nullptr,
                                 hp ? hist : nullptr, hp ? sort_flag_words(K, L.tile_bits) : 0, L.tile_counting),
                "duplicateWithKeys");
    }
    if (L.tile_counting) {
        StageTimer t(ST_TILE_SORT, stream);
        // also the tile ranges and the tile order's bucket counts; the plain
        // form's status word goes to the host word next to the pair count
        SG_CUDA(launch_tile_count_sort(reinterpret_cast<const uint16_t *>(k0), v0, v1, counters, cap_dev,
                                       (uint32_t)L.n_tiles, L.tc_chunks, hist,
                                       aux_tile, ranges, reinterpret_cast<uint32_t *>(w + L.order_scratch),
                                       rb ? rb->dev_ptr + 1 : nullptr, stream),
                "tile sort");
    } else {
        StageTimer t(ST_TILE_SORT, stream);
        // the last pass also bounds every tile's range in the sorted pairs
        // plain form: the sorts' merged status also goes to the host word next to the pair count
        SG_CUDA(launch_radix_sort(k0, v0, k1, v1, counters + CNT_WRITTEN, K, L.tile_bits, hist, aux_tile, stream,
                                  counters + CNT_STATUS, nullptr, true, ranges, L.n_tiles, true,
                                  rb ? rb->dev_ptr + 1 : nullptr, counters + CNT_STATUS,
                                  reinterpret_cast<uint32_t *>(w + L.order_scratch)),
                "tile sort");
    }
    if (sync) SG_CUDA(cudaEventRecord(rb->ev, stream), "read pairs");
    unsigned long long *evals =
        counting ? reinterpret_cast<unsigned long long *>(counters + CNT_EVALS) : nullptr;
    if (counting) SG_CUDA(cudaMemsetAsync(evals, 0, 8, stream), "clear counter");
    BlendShape shape{};
    st = blend_shape(false, reinterpret_cast<uint32_t *>(w + L.order),
                     reinterpret_cast<uint32_t *>(counters + CNT_QUEUE), shape);
    if (st != SG_OK) return st;
    shape.status = counters + CNT_STATUS;
    shape.importance = want_importance && !counting;
    if (shape.importance)
        for (int s = 0; s < n_scenes; ++s)
            if (scenes[s].n > 0)
                SG_CUDA(cudaMemsetAsync(importance[s], 0, (size_t)scenes[s].n * sizeof(float), stream),
                        "clear importance");
    {
        // built for every forward: the persistent backward walks tiles in this order too
        StageTimer t(ST_RANGES, stream);
        SG_CUDA(launch_tile_order(ranges, b.n_tiles, reinterpret_cast<uint32_t *>(w + L.order),
                                  reinterpret_cast<uint32_t *>(w + L.order_scratch), stream),
                "tile order");
    }
    {
        StageTimer t(ST_BLEND_FWD, stream);
        SG_CUDA(launch_blend_forward(db, b.n_tiles, ranges, pv_final, rec, img, T_final, last, shape, evals,
                                     stream),
                "blend forward");
    }
    if (counting) {
        uint64_t ne = 0;
        SG_CUDA(cudaMemcpyAsync(&ne, evals, 8, cudaMemcpyDeviceToHost, stream), "read counter");
        SG_CUDA(cudaStreamSynchronize(stream), "read counter");
        std::lock_guard<std::mutex> g(prof().mu);
        prof().evals[0] += (int64_t)ne;
    }
    if (sync) {
        SG_CUDA(cudaEventSynchronize(rb->ev), "read pairs");
        const volatile uint64_t *mirror = rb->host;
        const uint64_t n_pairs = mirror[0];
        if (mirror[1] == SG_ERR_TIMEOUT)
            return fail(SG_ERR_TIMEOUT, "a sort's bounded device wait expired (outputs unspecified)");
        if (n_pairs > cap_dev) {
            const WsLayout need = make_layout(b, n_pairs);
            fill_sizes(b, need, n_pairs, out);
            if (n_pairs > SORT_MAX_KEYS)
                return fail(SG_ERR_CAPACITY, "%llu pairs exceed the %llu one call can sort",
                            (unsigned long long)n_pairs, (unsigned long long)SORT_MAX_KEYS);
            return fail(SG_ERR_CAPACITY, "%llu pairs exceed the workspace capacity %llu (need %zu bytes)",
                        (unsigned long long)n_pairs, (unsigned long long)cap, need.total);
        }
        K = n_pairs;
    }
    fill_sizes(b, L, K, out);
    return SG_OK;
}

int backward_impl(const sg_scene *scenes, int n_scenes, const sg_camera *cams, const int32_t *view_scene,
                  int n_views, const void *ws, size_t ws_bytes, const float *T_final, const int32_t *last,
                  const float *d_img, void *bwd_ws, size_t bwd_ws_bytes, const sg_grads *grads,
                  cudaStream_t stream) {
    std::unique_ptr<Batch> hb(new Batch);
    int st = build_batch(scenes, n_scenes, cams, view_scene, n_views, true, *hb);
    if (st != SG_OK) return st;
    Batch &b = *hb;
    if (!grads) return fail(SG_ERR_INVALID_ARG, "grads must not be NULL");
    for (int s = 0; s < n_scenes; ++s) b.scene[s].grads = grads[s];
    if (!T_final || !last || !d_img) return fail(SG_ERR_INVALID_ARG, "T_final, last and d_img must not be NULL");
    if (!ws || !aligned(ws, ALIGN)) return fail(SG_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    if (!bwd_ws || !aligned(bwd_ws, ALIGN))
        return fail(SG_ERR_INVALID_ARG, "backward scratch NULL or not 256-byte aligned");
    if (bwd_ws_bytes < bwd_bytes(b))
        return fail(SG_ERR_WORKSPACE, "backward scratch of %zu bytes, %zu needed", bwd_ws_bytes, bwd_bytes(b));
    const uint64_t cap = capacity_for(b, ws_bytes);
    if (cap == UINT64_MAX) return fail(SG_ERR_WORKSPACE, "workspace smaller than its fixed part");
    const WsLayout L = make_layout(b, cap);
    const char *w = static_cast<const char *>(ws);
    const Rec *rec = reinterpret_cast<const Rec *>(w + L.rec);
    const uint32_t *tt = reinterpret_cast<const uint32_t *>(w + L.tiles_touched);
    const uint2 *ranges = reinterpret_cast<const uint2 *>(w + L.ranges);
    const uint32_t *pv_final = reinterpret_cast<const uint32_t *>(w + L.pval_final);
    char *bw = static_cast<char *>(bwd_ws);
    const BwdLayout BL = bwd_layout(b);
    Batch *db = reinterpret_cast<Batch *>(bw + BL.batch);
    uint64_t *counters = reinterpret_cast<uint64_t *>(bw + BL.counters);
    float *dg = reinterpret_cast<float *>(bw + BL.dg);
    const uint64_t M = L.M;

    const bool counting = (prof().flags & SG_PROFILE_COUNT) != 0;
    unsigned long long *evals =
        counting ? reinterpret_cast<unsigned long long *>(counters + CNT_EVALS) : nullptr;
    BlendShape shape{};
    // the forward's tile order (longest lists first)
    st = blend_shape(true, reinterpret_cast<const uint32_t *>(w + L.order),
                     reinterpret_cast<uint32_t *>(counters + CNT_QUEUE), shape);
    if (st != SG_OK) return st;
    shape.status = reinterpret_cast<const uint64_t *>(w + L.counters) + CNT_STATUS;   // the forward's
    {
        // the setup kernel also clears the 2D-gradient accumulators
        StageTimer t(ST_BWD_CLEAR, stream);
        ZeroRegions z;
        z.ptr[0] = reinterpret_cast<uint32_t *>(dg);
        z.words[0] = 9 * M;
        SG_CUDA(launch_setup(b, db, counters, stream, z), "setup");
    }
    {
        StageTimer t(ST_BLEND_BWD, stream);
        SG_CUDA(launch_blend_backward(db, b.n_tiles, ranges, pv_final, rec, T_final, last, d_img, dg, M, shape,
                                      evals, stream),
                "blend backward");
    }
    {
        StageTimer t(ST_PRE_BWD, stream);
        SG_CUDA(launch_preprocess_backward(b, db, tt, reinterpret_cast<const uint8_t *>(w + L.clamp), dg, M, stream), "preprocess backward");
    }
    if (counting) {
        uint64_t ne = 0;
        SG_CUDA(cudaMemcpyAsync(&ne, evals, 8, cudaMemcpyDeviceToHost, stream), "read counter");
        SG_CUDA(cudaStreamSynchronize(stream), "read counter");
        std::lock_guard<std::mutex> g(prof().mu);
        prof().evals[1] += (int64_t)ne;
    }
    return SG_OK;
}

}  // namespace

extern "C" {

int sg_profile_enable(int flags) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.flags = flags & (SG_PROFILE_EVENTS | SG_PROFILE_COUNT);
    return SG_OK;
}

int sg_profile_set_stages(uint32_t stage_mask) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.stage_mask = stage_mask;
    return SG_OK;
}

int sg_profile_read(double *ms, int64_t *launches, int64_t *pair_evals, int reset) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    int rc = SG_OK;
    for (auto &q : p.pending) {
        cudaError_t e = cudaEventSynchronize(q.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, q.a, q.b);
        if (e != cudaSuccess) rc = cuda_fail(e, "profile read");
        p.ms[q.stage] += t;
        p.launches[q.stage] += 1;
        p.pool.push_back(q.a);
        p.pool.push_back(q.b);
    }
    p.pending.clear();
    for (int i = 0; i < ST_N; ++i) {
        if (ms) ms[i] = p.ms[i];
        if (launches) launches[i] = p.launches[i];
    }
    if (pair_evals) { pair_evals[0] = p.evals[0]; pair_evals[1] = p.evals[1]; }
    if (reset) {
        for (int i = 0; i < ST_N; ++i) { p.ms[i] = 0.0; p.launches[i] = 0; }
        p.evals[0] = p.evals[1] = 0;
    }
    return rc;
}

int64_t sg_kernel_launches(void) { return launch_counter().load(); }

int sg_set_tuning(const sg_tuning *t) {
    if (!t) {
        tuning() = kDefaultTuning;
        set_sort_wait_polls(0);
        return SG_OK;
    }
    if (!ppt_ok(t->fwd_pixels_per_thread) || !ppt_ok(t->bwd_pixels_per_thread))
        return fail(SG_ERR_INVALID_ARG, "pixels per thread must be 1, 2, 4 or 8 (got %d, %d)",
                    t->fwd_pixels_per_thread, t->bwd_pixels_per_thread);
    if (t->sort_wait_polls < 0) return fail(SG_ERR_INVALID_ARG, "sort_wait_polls = %d < 0", t->sort_wait_polls);
    if (!(t->fwd_batch == 0 || t->fwd_batch == 32 || t->fwd_batch == 64 || t->fwd_batch == 128))
        return fail(SG_ERR_INVALID_ARG, "fwd_batch must be 0, 32, 64 or 128 (got %d)", t->fwd_batch);
    if (!(t->bwd_batch == 0 || t->bwd_batch == 32 || t->bwd_batch == 64))
        return fail(SG_ERR_INVALID_ARG, "bwd_batch must be 0, 32 or 64 (got %d)", t->bwd_batch);
    tuning() = *t;
    set_sort_wait_polls((uint32_t)t->sort_wait_polls);
    return SG_OK;
}

int sg_get_tuning(sg_tuning *t) {
    if (!t) return fail(SG_ERR_INVALID_ARG, "t must not be NULL");
    *t = tuning();
    return SG_OK;
}

const char *sg_profile_stage_name(int i) { return (i >= 0 && i < ST_N) ? kStageNames[i] : nullptr; }

int sg_version(void) { return SG_ABI_VERSION; }

const char *sg_last_error(void) { return g_err; }

int sg_workspace_query(const sg_scene *scene, const sg_camera *cams, int n_views, uint64_t pair_capacity,
                       sg_sizes *out) {
    if (!out) return fail(SG_ERR_INVALID_ARG, "out must not be NULL");
    std::unique_ptr<Batch> hb(new Batch);
    int st = build_batch(scene, 1, cams, nullptr, n_views, false, *hb);
    if (st != SG_OK) return st;
    if (pair_capacity >= (1ull << 32) - 1) return fail(SG_ERR_INVALID_ARG, "pair capacity too large");
    const WsLayout L = make_layout(*hb, pair_capacity);
    fill_sizes(*hb, L, 0, out);
    return SG_OK;
}

static int layout_of(const sg_scene *scenes, int n_scenes, const sg_camera *cams, const int32_t *view_scene,
                     int n_views, size_t ws_bytes, sg_ws_layout *out) {
    if (!out) return fail(SG_ERR_INVALID_ARG, "out must not be NULL");
    std::unique_ptr<Batch> hb(new Batch);
    int st = build_batch(scenes, n_scenes, cams, view_scene, n_views, false, *hb);
    if (st != SG_OK) return st;
    const uint64_t cap = capacity_for(*hb, ws_bytes);
    if (cap == UINT64_MAX) return fail(SG_ERR_WORKSPACE, "workspace smaller than its fixed part");
    const WsLayout L = make_layout(*hb, cap);
    out->rec = L.rec;
    out->tiles_touched = L.tiles_touched;
    out->rect = L.rect;
    out->depth_order = L.dval0;
    out->ranges = L.ranges;
    out->pair_tile = L.pkey_final;
    out->pair_entry = L.pval_final;
    out->total_bytes = L.total;
    return SG_OK;
}

int sg_workspace_layout(const sg_scene *scene, const sg_camera *cams, int n_views, size_t ws_bytes,
                        sg_ws_layout *out) {
    return layout_of(scene, 1, cams, nullptr, n_views, ws_bytes, out);
}

int sg_batched_workspace_layout(const sg_scene *scenes, int n_scenes, const sg_camera *cams,
                                const int32_t *view_scene, int n_views, size_t ws_bytes, sg_ws_layout *out) {
    if (!view_scene) return fail(SG_ERR_INVALID_ARG, "view_scene must not be NULL");
    return layout_of(scenes, n_scenes, cams, view_scene, n_views, ws_bytes, out);
}

int sg_render_forward(const sg_scene *scene, const sg_camera *cams, int n_views, void *ws, size_t ws_bytes,
                      float *img, float *T_final, int32_t *last, sg_sizes *out, void *stream) {
    g_err[0] = '\0';
    return forward_impl(scene, 1, cams, nullptr, n_views, ws, ws_bytes, img, T_final, last, nullptr, out,
                        static_cast<cudaStream_t>(stream), true);
}

int sg_render_forward_importance(const sg_scene *scene, const sg_camera *cams, int n_views, void *ws,
                                 size_t ws_bytes, float *img, float *T_final, int32_t *last, float *importance,
                                 sg_sizes *out, void *stream) {
    g_err[0] = '\0';
    float *const imp[1] = {importance};
    return forward_impl(scene, 1, cams, nullptr, n_views, ws, ws_bytes, img, T_final, last, imp, out,
                        static_cast<cudaStream_t>(stream), true);
}

int sg_render_backward(const sg_scene *scene, const sg_camera *cams, int n_views, const void *ws,
                       size_t ws_bytes, const float *T_final, const int32_t *last, const float *d_img,
                       void *bwd_ws, size_t bwd_ws_bytes, const sg_grads *grads, void *stream) {
    g_err[0] = '\0';
    return backward_impl(scene, 1, cams, nullptr, n_views, ws, ws_bytes, T_final, last, d_img, bwd_ws,
                         bwd_ws_bytes, grads, static_cast<cudaStream_t>(stream));
}

// Times every blend shape (pixels per thread 1, 2, 4, 8; one block per tile or
// persistent) on the caller's workload: each candidate runs `reps` forward and
// backward calls after one untimed pair; the forward and the backward pick
// their fastest shape independently (only the blend kernels differ between
// candidates, so whole-call times rank them). The choice is installed with
// sg_set_tuning and written to *chosen; times_ms (nullable) receives [2][8]
// mean milliseconds, forward then backward, candidate c = 2 * log2(P) + persistent.
int sg_autotune(const sg_scene *scene, const sg_camera *cams, int n_views, void *ws, size_t ws_bytes,
                float *img, float *T_final, int32_t *last, const float *d_img, void *bwd_ws,
                size_t bwd_ws_bytes, const sg_grads *grads, int reps, sg_tuning *chosen, float *times_ms,
                void *stream) {
    g_err[0] = '\0';
    if (!chosen) return fail(SG_ERR_INVALID_ARG, "chosen must not be NULL");
    if (reps < 1 || reps > 100) return fail(SG_ERR_INVALID_ARG, "reps = %d out of [1, 100]", reps);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const sg_tuning saved = tuning();
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto &x : ev) if (x) cudaEventDestroy(x);
            return cuda_fail(cudaGetLastError(), "autotune events");
        }
    float best_f = 1e30f, best_b = 1e30f;
    int bf = 0, bb = 0;
    int st = SG_OK;
    for (int c = 0; c < 8 && st == SG_OK; ++c) {
        sg_tuning t = saved;
        t.fwd_pixels_per_thread = t.bwd_pixels_per_thread = 1 << (c >> 1);
        t.fwd_persistent = t.bwd_persistent = c & 1;
        tuning() = t;
        float tf = 0.f, tb = 0.f;
        for (int r = 0; r <= reps && st == SG_OK; ++r) {
            sg_sizes sz{};
            cudaEventRecord(ev[0], s);
            st = forward_impl(scene, 1, cams, nullptr, n_views, ws, ws_bytes, img, T_final, last, nullptr, &sz, s,
                              true);
            if (st != SG_OK) break;
            cudaEventRecord(ev[1], s);
            st = backward_impl(scene, 1, cams, nullptr, n_views, ws, ws_bytes, T_final, last, d_img, bwd_ws,
                               bwd_ws_bytes, grads, s);
            if (st != SG_OK) break;
            cudaEventRecord(ev[2], s);
            const cudaError_t e = cudaEventSynchronize(ev[2]);
            if (e != cudaSuccess) { st = cuda_fail(e, "autotune"); break; }
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            cudaEventElapsedTime(&b, ev[1], ev[2]);
            if (r > 0) { tf += a; tb += b; }   // the first pair is untimed
        }
        if (st != SG_OK) break;
        tf /= (float)reps;
        tb /= (float)reps;
        if (times_ms) { times_ms[c] = tf; times_ms[8 + c] = tb; }
        if (tf < best_f) { best_f = tf; bf = c; }
        if (tb < best_b) { best_b = tb; bb = c; }
    }
    // then the batch sizes for the chosen shapes (forward 32 / 64 / 128, backward 32 / 64)
    sg_tuning t = saved;
    t.fwd_pixels_per_thread = 1 << (bf >> 1);
    t.fwd_persistent = bf & 1;
    t.bwd_pixels_per_thread = 1 << (bb >> 1);
    t.bwd_persistent = bb & 1;
    int best_fb = 64, best_bb = 64;
    best_f = best_b = 1e30f;
    for (int c = 0; c < 3 && st == SG_OK; ++c) {
        sg_tuning u = t;
        u.fwd_batch = 32 << c;
        u.bwd_batch = c < 2 ? 32 << c : 64;
        tuning() = u;
        float tf = 0.f, tb = 0.f;
        for (int r = 0; r <= reps && st == SG_OK; ++r) {
            sg_sizes sz{};
            cudaEventRecord(ev[0], s);
            st = forward_impl(scene, 1, cams, nullptr, n_views, ws, ws_bytes, img, T_final, last, nullptr, &sz, s,
                              true);
            if (st != SG_OK) break;
            cudaEventRecord(ev[1], s);
            st = backward_impl(scene, 1, cams, nullptr, n_views, ws, ws_bytes, T_final, last, d_img, bwd_ws,
                               bwd_ws_bytes, grads, s);
            if (st != SG_OK) break;
            cudaEventRecord(ev[2], s);
            const cudaError_t e = cudaEventSynchronize(ev[2]);
            if (e != cudaSuccess) { st = cuda_fail(e, "autotune"); break; }
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            cudaEventElapsedTime(&b, ev[1], ev[2]);
            if (r > 0) { tf += a; tb += b; }
        }
        if (st != SG_OK) break;
        if (tf < best_f) { best_f = tf; best_fb = u.fwd_batch; }
        if (c < 2 && tb < best_b) { best_b = tb; best_bb = u.bwd_batch; }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st != SG_OK) {
        tuning() = saved;
        return st;
    }
    t.fwd_batch = best_fb;
    t.bwd_batch = best_bb;
    tuning() = t;
    *chosen = t;
    return SG_OK;
}

int sg_batched_workspace_query(const sg_scene *scenes, int n_scenes, const sg_camera *cams,
                               const int32_t *view_scene, int n_views, uint64_t pair_capacity, sg_sizes *out) {
    if (!out) return fail(SG_ERR_INVALID_ARG, "out must not be NULL");
    if (!view_scene) return fail(SG_ERR_INVALID_ARG, "view_scene must not be NULL");
    std::unique_ptr<Batch> hb(new Batch);
    int st = build_batch(scenes, n_scenes, cams, view_scene, n_views, false, *hb);
    if (st != SG_OK) return st;
    if (pair_capacity >= (1ull << 32) - 1) return fail(SG_ERR_INVALID_ARG, "pair capacity too large");
    fill_sizes(*hb, make_layout(*hb, pair_capacity), 0, out);
    return SG_OK;
}

int sg_render_batched_forward(const sg_scene *scenes, int n_scenes, const sg_camera *cams,
                              const int32_t *view_scene, int n_views, void *ws, size_t ws_bytes, float *img,
                              float *T_final, int32_t *last, float *const *importance, void *stream) {
    g_err[0] = '\0';
    if (!view_scene) return fail(SG_ERR_INVALID_ARG, "view_scene must not be NULL");
    return forward_impl(scenes, n_scenes, cams, view_scene, n_views, ws, ws_bytes, img, T_final, last,
                        importance, nullptr, static_cast<cudaStream_t>(stream), false);
}

int sg_render_batched_backward(const sg_scene *scenes, int n_scenes, const sg_camera *cams,
                               const int32_t *view_scene, int n_views, const void *ws, size_t ws_bytes,
                               const float *T_final, const int32_t *last, const float *d_img, void *bwd_ws,
                               size_t bwd_ws_bytes, const sg_grads *grads, void *stream) {
    g_err[0] = '\0';
    if (!view_scene) return fail(SG_ERR_INVALID_ARG, "view_scene must not be NULL");
    return backward_impl(scenes, n_scenes, cams, view_scene, n_views, ws, ws_bytes, T_final, last, d_img, bwd_ws,
                         bwd_ws_bytes, grads, static_cast<cudaStream_t>(stream));
}

size_t sg_admm_workspace_bytes(int64_t n) { return admm_workspace_bytes(n); }

static int admm_check(int64_t n, const void *ws, size_t ws_bytes) {
    if (n < 0 || n >= (int64_t)UINT32_MAX) return fail(SG_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
    if (n > 0 && (!ws || !aligned(ws, ALIGN)))
        return fail(SG_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    if (ws_bytes < admm_workspace_bytes(n))
        return fail(SG_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, admm_workspace_bytes(n));
    return SG_OK;
}

int sg_admm_opacity_step(int64_t n, const float *opac, const float *importance, int64_t kappa, float *lambda,
                         float *opac_tilde, void *ws, size_t ws_bytes, void *stream) {
    g_err[0] = '\0';
    int st = admm_check(n, ws, ws_bytes);
    if (st != SG_OK) return st;
    if (n > 0 && (!opac || !lambda || !opac_tilde))
        return fail(SG_ERR_INVALID_ARG, "opac, lambda and opac_tilde must not be NULL");
    SG_CUDA(launch_admm_step(0, n, opac, importance, nullptr, kappa, lambda, opac_tilde, ws,
                             static_cast<cudaStream_t>(stream)),
            "ADMM opacity step");
    return SG_OK;
}

int sg_admm_sharpness_step(int64_t n_lobes, const float *sharp, const float *amp, int64_t kappa, float *lambda,
                           float *sharp_tilde, void *ws, size_t ws_bytes, void *stream) {
    g_err[0] = '\0';
    int st = admm_check(n_lobes, ws, ws_bytes);
    if (st != SG_OK) return st;
    if (n_lobes > 0 && (!sharp || !amp || !lambda || !sharp_tilde))
        return fail(SG_ERR_INVALID_ARG, "sharp, amp, lambda and sharp_tilde must not be NULL");
    SG_CUDA(launch_admm_step(1, n_lobes, sharp, nullptr, amp, kappa, lambda, sharp_tilde, ws,
                             static_cast<cudaStream_t>(stream)),
            "ADMM sharpness step");
    return SG_OK;
}

int sg_admm_penalty_grad(int64_t n, const float *x, const float *x_tilde, const float *lambda, float delta,
                         float *grad, void *stream) {
    g_err[0] = '\0';
    if (n < 0) return fail(SG_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!x || !x_tilde || !lambda || !grad))
        return fail(SG_ERR_INVALID_ARG, "x, x_tilde, lambda and grad must not be NULL");
    SG_CUDA(launch_penalty_grad(n, x, x_tilde, lambda, delta, grad, static_cast<cudaStream_t>(stream)),
            "ADMM penalty gradient");
    return SG_OK;
}

size_t sg_postprocess_workspace_bytes(int64_t n) { return post_workspace_bytes(n); }

static int post_check(const sg_scene *in, const void *ws, size_t ws_bytes) {
    if (!in) return fail(SG_ERR_INVALID_ARG, "scene must not be NULL");
    if (in->n < 0 || in->n >= (int64_t)INT32_MAX || in->n_lobes < 0 || in->n_lobes >= (int64_t)INT32_MAX)
        return fail(SG_ERR_INVALID_ARG, "sizes out of range");
    if (in->dtype_geom != SG_F32 || in->dtype_lobe != SG_F32 || in->dtype_sharp != SG_F32)
        return fail(SG_ERR_INVALID_ARG, "post-processing reads binary32 scenes only");
    if (in->n > 0) {
        const void *req[] = {in->means, in->scales, in->quats, in->opac, in->gmask, in->c0, in->lobe_off};
        for (const void *p : req)
            if (!p) return fail(SG_ERR_INVALID_ARG, "a Gaussian array is NULL");
    }
    if (in->n_lobes > 0 && (!in->axis || !in->sharp || !in->amp || !in->lmask))
        return fail(SG_ERR_INVALID_ARG, "a lobe array is NULL");
    if (!ws || !aligned(ws, ALIGN)) return fail(SG_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    if (ws_bytes < post_workspace_bytes(in->n))
        return fail(SG_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, post_workspace_bytes(in->n));
    return SG_OK;
}

int sg_postprocess_plan(const sg_scene *in, float tau_opacity, float tau_sharpness, void *ws, size_t ws_bytes,
                        int64_t *n_out, int64_t *l_out, void *stream) {
    g_err[0] = '\0';
    int st = post_check(in, ws, ws_bytes);
    if (st != SG_OK) return st;
    uint64_t totals[2] = {0, 0};
    SG_CUDA(launch_post_plan(*in, tau_opacity, tau_sharpness, ws, totals, static_cast<cudaStream_t>(stream)),
            "post-processing plan");
    if (n_out) *n_out = (int64_t)totals[0];
    if (l_out) *l_out = (int64_t)totals[1];
    return SG_OK;
}

int sg_postprocess_apply(const sg_scene *in, float tau_opacity, float tau_sharpness, const void *ws,
                         size_t ws_bytes, const sg_scene *out, void *stream) {
    g_err[0] = '\0';
    int st = post_check(in, ws, ws_bytes);
    if (st != SG_OK) return st;
    if (!out || !out->lobe_off) return fail(SG_ERR_INVALID_ARG, "out and out->lobe_off must not be NULL");
    if (out->n > 0) {
        const void *req[] = {out->means, out->scales, out->quats, out->opac, out->gmask, out->c0};
        for (const void *p : req)
            if (!p) return fail(SG_ERR_INVALID_ARG, "an output Gaussian array is NULL");
    }
    if (out->n_lobes > 0 && (!out->axis || !out->sharp || !out->amp || !out->lmask))
        return fail(SG_ERR_INVALID_ARG, "an output lobe array is NULL");
    SG_CUDA(launch_post_apply(*in, tau_opacity, tau_sharpness, ws, *out, out->n, out->n_lobes,
                              static_cast<cudaStream_t>(stream)),
            "post-processing apply");
    return SG_OK;
}

int sg_forward_status(const void *ws, uint64_t *n_pairs, int32_t *status, void *stream) {
    if (!ws || !aligned(ws, ALIGN)) return fail(SG_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    // the counters sit right after the batch table, whatever the sizes
    const uint64_t *counters = reinterpret_cast<const uint64_t *>(static_cast<const char *>(ws) + al(sizeof(Batch)));
    uint64_t host[CNT_N] = {};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SG_CUDA(cudaMemcpyAsync(host, counters, sizeof(host), cudaMemcpyDeviceToHost, s), "read status");
    SG_CUDA(cudaStreamSynchronize(s), "read status");
    if (n_pairs) *n_pairs = host[CNT_PAIRS];
    if (status) *status = (int32_t)host[CNT_STATUS];
    return SG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Backward with library-owned scratch, for callers that cannot allocate
// device memory while rendering
// ---------------------------------------------------------------------------
namespace {

// Scratch of sg_render_backward_noalloc: batch table, counters and the
// [9][M] per-entry 2D-gradient accumulators. Every device that loads the
// library holds it until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[SG_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device. In host code the
// array's name stands for the symbol, not for device memory, so the address is
// looked up once per device (with that device current) and cached.
int noalloc_scratch(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc backward: cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return fail(SG_ERR_INVALID_ARG, "no-alloc backward: device %d out of range", dev);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "no-alloc backward: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SG_OK;
}

}  // namespace

extern "C" int sg_render_backward_noalloc(const sg_scene *scene, const sg_camera *cams, int n_views,
                                          const void *ws, size_t ws_bytes, const float *T_final,
                                          const int32_t *last, const float *d_img, const sg_grads *grads,
                                          void *stream_) {
    g_err[0] = '\0';
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    Batch b;   // host table on the stack: no heap allocation either
    int st = build_batch(scene, 1, cams, nullptr, n_views, true, b);
    if (st != SG_OK) return st;
    if (!grads) return fail(SG_ERR_INVALID_ARG, "grads must not be NULL");
    b.scene[0].grads = grads[0];
    if (!T_final || !last || !d_img) return fail(SG_ERR_INVALID_ARG, "T_final, last and d_img must not be NULL");
    if (!ws || !aligned(ws, ALIGN)) return fail(SG_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    const size_t need = bwd_bytes(b);
    if (need > (size_t)SG_NOALLOC_SCRATCH_BYTES)
        return fail(SG_ERR_WORKSPACE,
                    "no-alloc backward needs %zu bytes of scratch for %llu entries; the static scratch holds "
                    "%zu bytes; use sg_render_backward with caller scratch",
                    need, (unsigned long long)b.n_entries, (size_t)SG_NOALLOC_SCRATCH_BYTES);
    const uint64_t cap = capacity_for(b, ws_bytes);
    if (cap == UINT64_MAX) return fail(SG_ERR_WORKSPACE, "workspace smaller than its fixed part");
    void *scratch = nullptr;
    st = noalloc_scratch(&scratch);
    if (st != SG_OK) return st;
    const WsLayout L = make_layout(b, cap);
    const char *w = static_cast<const char *>(ws);
    const Rec *rec = reinterpret_cast<const Rec *>(w + L.rec);
    const uint32_t *tt = reinterpret_cast<const uint32_t *>(w + L.tiles_touched);
    const uint2 *ranges = reinterpret_cast<const uint2 *>(w + L.ranges);
    const uint32_t *pv_final = reinterpret_cast<const uint32_t *>(w + L.pval_final);
    char *bw = static_cast<char *>(scratch);
    const BwdLayout BL = bwd_layout(b);
    Batch *db = reinterpret_cast<Batch *>(bw + BL.batch);
    uint64_t *counters = reinterpret_cast<uint64_t *>(bw + BL.counters);
    float *dg = reinterpret_cast<float *>(bw + BL.dg);
    const uint64_t M = L.M;
    BlendShape shape{};   // one block per tile: no tile order or work counter needed
    shape.pixels_per_thread = tuning().bwd_pixels_per_thread;
    shape.batch = tuning().bwd_batch ? tuning().bwd_batch : kDefaultBatch;
    shape.status = reinterpret_cast<const uint64_t *>(w + L.counters) + CNT_STATUS;   // the forward's
    // the setup kernel rewrites the table and counters and clears the accumulators
    ZeroRegions z;
    z.ptr[0] = reinterpret_cast<uint32_t *>(dg);
    z.words[0] = 9 * M;
    SG_CUDA(launch_setup(b, db, counters, stream, z), "setup");
    SG_CUDA(launch_blend_backward(db, b.n_tiles, ranges, pv_final, rec, T_final, last, d_img, dg, M, shape,
                                  nullptr, stream),
            "blend backward");
    SG_CUDA(launch_preprocess_backward(b, db, tt, reinterpret_cast<const uint8_t *>(w + L.clamp), dg, M, stream), "preprocess backward");
    return SG_OK;
}
