// Internal declarations shared by the kernel translation units of the
// SG-splatting rasterizer (sm_103a). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstddef>
#include <cstdint>

#include "../../include/sgsplat.h"

namespace sgk {

constexpr int TILE = SG_TILE;             // 16x16 pixel tiles
constexpr int BLEND_THREADS = TILE * TILE;
constexpr int PRE_THREADS = 256;

// Per-view camera and packing offsets. Built on the host, copied into the
// workspace by k_setup so that kernels take a single pointer.
struct ViewDesc {
    float fx, fy, cx, cy;
    float V[12];          // world->camera [R|t], row-major
    float campos[3];      // camera centre in world space (-R^T t)
    float near_plane;
    float bg[3];
    int32_t W, H, tiles_x, tiles_y;
    int32_t scene;        // index into Batch::scene
    int32_t n;            // Gaussians of that scene
    uint32_t tile_off;    // first global tile id of the view
    uint32_t pad1;
    uint32_t pad0;
    uint64_t pix_off;     // first pixel of the view in T_final / last (img: x3)
    uint64_t ent_off;     // first (view, Gaussian) entry of the view
};

struct SceneDesc {
    const void *means, *scales, *quats, *opac;
    const float *gmask, *c0;
    const int32_t *lobe_off;
    const void *axis, *sharp, *amp;
    const float *lmask;
    const float *sh;      // SH3 coefficients [3][16][N] (color_model SH3)
    float *importance;    // forward output: sum of alpha T per Gaussian (null: not wanted)
    sg_grads grads;
    int64_t n, n_lobes;
    int32_t dtype_geom, dtype_lobe, dtype_sharp, color_model;
    uint32_t blk_off;     // first block of the scene in the per-Gaussian preprocess grids
};

struct Batch {
    int32_t n_views, n_scenes;
    uint32_t n_tiles;
    uint32_t scene_blocks;   // blocks of 256 scene Gaussians over all scenes
    uint32_t max_views_per_scene;
    uint32_t pad0;
    uint64_t n_entries;
    ViewDesc view[SG_MAX_VIEWS];
    SceneDesc scene[SG_MAX_SCENES];
};

// One projected Gaussian: 48 bytes. The tile binning reads the first 24 bytes
// (one 32-byte sector), the blend the first 40.
struct __align__(16) Rec {
    float4 a;   // x, y, conic A, conic B
    float4 b;   // conic C, tile-binning bound t (tile_reach_threshold), o' = m_g * o, r
    float4 c;   // g, b, radius, depth
};

// Device counters kept in the workspace.
enum : int {
    CNT_ENTRIES = 0,   // (view, Gaussian) entries
    CNT_PAIRS = 1,     // (tile, Gaussian) pairs of the forward
    CNT_STATUS = 2,    // sg_status of the last batched forward
    CNT_EVALS = 3,     // pair evaluations (counting kernels)
    CNT_TILES = 4,     // tiles
    CNT_QUEUE = 5,     // persistent-blend work counter
    CNT_VISIBLE = 6,   // entries with at least one pair (the depth order's length)
    CNT_DUP_BLOCK = 7, // duplicate kernel: next logical block
    CNT_WRITTEN = 8,   // pairs the duplicate wrote (min(pairs, capacity)): the tile sort's count
    CNT_N = 10
};

// Radix sort / scan geometry.
constexpr int RS_THREADS = 256;
#ifndef SG_RS_ITEMS
#define SG_RS_ITEMS 12
#endif
constexpr int RS_ITEMS = SG_RS_ITEMS;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // 3072 keys per block
constexpr int RS_RADIX = 256;
constexpr int SCAN_TILE = 4096;

// Byte offsets of every workspace buffer (host computed, identical for the
// forward and the backward of one call).
struct WsLayout {
    size_t batch, counters, rec, tiles_touched, rect, clamp, dkey0, dval0, dkey1, dval1,
        dup_flags, ranges, order, order_scratch, scan_sums, hist, aux_tile, fixed_end;
    size_t pval_final, pkey_final, pval_tmp, pkey_tmp, total;
    uint64_t M, n_tiles, cap;
    int tile_bits, tile_passes;
    bool tile_counting;   // the tile sort counts (launch_tile_count_sort) instead of radix passes:
    uint32_t tc_chunks;   // its chunks; its count matrix takes the look-back flags' region and
                          // no sorted keys are kept (pkey_final = NO_OFFSET)
};

__host__ __device__ inline uint64_t div_up(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// A workspace buffer the layout does not hold.
constexpr size_t NO_OFFSET = ~(size_t)0;

// ---------------------------------------------------------------------------
// Tight tile binning. A pair (tile, Gaussian) can only blend where
// alpha = o' exp(-q / 2) >= 1/255, q = A dx^2 + 2 B dx dy + C dy^2 (the conic),
// i.e. inside the ellipse q <= 2 ln(255 o'). Of the tiles of the 3-sigma
// rectangle, only those whose box of pixel centres meets that ellipse get a
// pair; the others would be skipped at every pixel, so leaving them out changes
// no image and no gradient. The ellipse is enlarged (1 % + 0.01 in q, 0.02 px)
// so that binary32 rounding here or in the blend can only keep extra tiles.
// Preprocess counts the tiles and duplicate enumerates them with this same
// code (explicitly rounded operations), so the two agree exactly.
// ---------------------------------------------------------------------------
struct TileReach {
    float x, y, B, det, At, ymax, m, invA;
    int mode;   // 0: reaches nothing, 1: ellipse, 2: whole rectangle (degenerate conic)
};

// The tile binning is a decision recipe like cull and rectangle: every step is
// one binary32 operation with round-to-nearest (no contraction), so that a
// restatement in numpy float32 states exactly which tiles are kept. Its
// constants are exact binary32 values (hexadecimal literals).
constexpr float TR_C7 = 0x1.24924ap-3f;      // 1/7
constexpr float TR_C5 = 0x1.99999ap-3f;      // 1/5
constexpr float TR_C3 = 0x1.555556p-2f;      // 1/3
constexpr float TR_INV_LN2 = 0x1.715476p+0f; // 1/ln 2
constexpr float TR_LN2X2 = 0x1.62e430p+0f;   // 2 ln 2
constexpr float TR_GROW = 0x1.028f5cp+0f;    // 1.01
constexpr float TR_ADD = 0x1.47ae14p-7f;     // 0.01
constexpr float TR_PAD = 0x1.47ae14p-6f;     // 0.02 px

// log2 of a positive normal x: exponent plus ln(m) / ln 2 for the mantissa
// m in [1, 2), ln m = 2 atanh(s) with s = (m - 1) / (m + 1) <= 1/3, summed to
// s^7 (relative error below 1e-5, far inside the 1 % enlargement below).
__device__ __forceinline__ float log2_recipe(float x) {
    const uint32_t u = __float_as_uint(x);
    const float e = (float)((int)((u >> 23) & 255u) - 127);
    const float m = __uint_as_float((u & 0x007FFFFFu) | 0x3F800000u);
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float P = __fadd_rn(__fmul_rn(s2, TR_C7), TR_C5);
    P = __fadd_rn(__fmul_rn(P, s2), TR_C3);
    P = __fadd_rn(__fmul_rn(P, s2), 1.0f);
    const float lnm = __fmul_rn(__fmul_rn(2.0f, s), P);
    return __fadd_rn(e, __fmul_rn(lnm, TR_INV_LN2));
}

// Enlarged bound on q where alpha can reach 1/255: 2 ln(255 o') (1 + 1 %) + 0.01;
// negative when o' < 1/255 (alpha <= o' < 1/255 everywhere). Computed once per
// entry by preprocess and kept in its record.
__device__ __forceinline__ float tile_reach_threshold(float op) {
    if (!(op >= 1.0f / 255.0f)) return -1.0f;
    const float t0 = __fmul_rn(TR_LN2X2, log2_recipe(__fmul_rn(255.0f, op)));
    return __fadd_rn(__fmul_rn(t0, TR_GROW), TR_ADD);
}

__device__ __forceinline__ void tile_reach_init(float x, float y, float A, float B, float C, float t,
                                                TileReach &R) {
    R.x = x; R.y = y; R.B = B;
    R.det = R.At = R.ymax = R.m = R.invA = 0.f;
    if (!(t >= 0.f)) { R.mode = 0; return; }
    R.det = __fsub_rn(__fmul_rn(A, C), __fmul_rn(B, B));
    if (!(A > 0.f) || !(C > 0.f) || !(R.det > 0.f) || !isfinite(t) || !isfinite(R.det)) {
        R.mode = 2;
        return;
    }
    R.At = __fmul_rn(A, t);
    R.ymax = __fsqrt_rn(__fdiv_rn(R.At, R.det));
    const float xmax = __fsqrt_rn(__fdiv_rn(__fmul_rn(C, t), R.det));
    R.m = __fdiv_rn(__fmul_rn(B, xmax), C);   // dy of the right-most point is -m, of the left-most +m
    R.invA = __frcp_rn(A);
    R.mode = isfinite(R.ymax) && isfinite(R.m) && isfinite(R.At) && isfinite(R.invA) ? 1 : 2;
}

// Columns [c0, c1) of tile row ty (within [x0, x1)) that the enlarged ellipse
// reaches. Over the row's band of dy, the ellipse's right edge
// x_r(dy) = (-B dy + sqrt(A t - det dy^2)) / A is concave with its maximum at
// dy = -m (m = B xmax / C), the left edge convex with its minimum at dy = +m:
// both extremes are taken at those points clamped into the band.
__device__ __forceinline__ void tile_reach_row(const TileReach &R, int ty, int x0, int x1, int &c0, int &c1) {
    c0 = c1 = x0;
    if (R.mode == 0) return;
    if (R.mode == 2) { c1 = x1; return; }
    const float pad = TR_PAD;
    float lo = __fsub_rn(__fsub_rn((float)(ty * SG_TILE), R.y), pad);
    float hi = __fadd_rn(__fsub_rn((float)(ty * SG_TILE + SG_TILE - 1), R.y), pad);
    lo = fmaxf(lo, -R.ymax);
    hi = fminf(hi, R.ymax);
    if (!(lo <= hi)) return;
    const float dr = fminf(fmaxf(-R.m, lo), hi), dl = fminf(fmaxf(R.m, lo), hi);
    const float sr = __fsqrt_rn(fmaxf(0.f, __fsub_rn(R.At, __fmul_rn(R.det, __fmul_rn(dr, dr)))));
    const float sl = __fsqrt_rn(fmaxf(0.f, __fsub_rn(R.At, __fmul_rn(R.det, __fmul_rn(dl, dl)))));
    const float xr = __fadd_rn(__fadd_rn(R.x, __fmul_rn(__fsub_rn(sr, __fmul_rn(R.B, dr)), R.invA)), pad);
    const float xl = __fsub_rn(__fsub_rn(R.x, __fmul_rn(__fadd_rn(sl, __fmul_rn(R.B, dl)), R.invA)), pad);
    // tile tx is reached iff 16 tx <= xr and 16 tx + 15 >= xl (clamped to the rectangle first;
    // scaling by 1/16 is exact)
    const float fx0 = (float)(x0 * SG_TILE - SG_TILE), fx1 = (float)(x1 * SG_TILE);
    const float a = ceilf(__fmul_rn(__fsub_rn(fminf(fmaxf(xl, fx0), fx1), (float)(SG_TILE - 1)), 1.0f / SG_TILE));
    const float b = floorf(__fmul_rn(fminf(fmaxf(xr, fx0), fx1), 1.0f / SG_TILE));
    c0 = max(x0, (int)a);
    c1 = max(c0, min(x1, (int)b + 1));
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_inclusive(T x) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= (unsigned)o) x += y;
    }
    return x;
}

// exclusive scan over blockDim.x (multiple of 32, <= 1024) values; returns the
// exclusive prefix and writes the block total.
template <typename T>
__device__ __forceinline__ T block_exclusive(T x, T &total, T *sh /* >= 32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const T inc = warp_inclusive(x);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? sh[lane] : T(0);
        const T wi = warp_inclusive(w);
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    const T r = sh[warp] + inc - x;
    total = sh[32];
    __syncthreads();
    return r;
}

// Decoupled look-back words of 64 bits (the duplicate blocks, the ADMM
// selection): 2 status bits (aggregate, inclusive prefix) and a 62-bit count.
constexpr uint64_t DL_AGG = 1ull << 62, DL_INC = 2ull << 62, DL_VAL = (1ull << 62) - 1ull;

__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" : : "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive prefix of the counts of logical blocks [0, blk) (warp 0 of the
// block; all its lanes return it). The block has published its own count
// (DL_AGG) before it calls this, so successors never wait on a block that waits. Predecessors are read 32 at a time;
// a run of ready words ending in an inclusive prefix completes the sum. Unready
// words are polled at most spin_limit times; past that the status word gets
// SG_ERR_TIMEOUT and the (smaller) partial prefix is returned.
__device__ __forceinline__ uint64_t block_lookback64(uint64_t *__restrict__ dflags, uint64_t blk, uint64_t count,
                                                 uint32_t spin_limit, uint64_t *status) {
    const int lane = threadIdx.x & 31;
    uint64_t excl = 0;
    int64_t p = (int64_t)blk - 1;
    uint32_t spins = 0;
    while (p >= 0) {
        const int64_t q = p - lane;
        const uint64_t f = q >= 0 ? ld_relaxed64(dflags + q) : DL_INC;   // before block 0: prefix 0
        const uint32_t unready = __ballot_sync(0xffffffffu, (f & ~DL_VAL) == 0ull);
        const uint32_t inc = __ballot_sync(0xffffffffu, (f & DL_INC) != 0ull);
        const int first_unready = unready ? __ffs(unready) - 1 : 32;
        const int first_inc = inc ? __ffs(inc) - 1 : 32;
        if (first_inc < first_unready) {
            excl += warp_sum64(lane <= first_inc ? (f & DL_VAL) : 0ull);
            break;
        }
        excl += warp_sum64(lane < first_unready ? (f & DL_VAL) : 0ull);
        p -= first_unready;
        if (first_unready < 32) {
            if (++spins >= spin_limit) {
                if (lane == 0) atomicExch(reinterpret_cast<unsigned long long *>(status),
                                          (unsigned long long)SG_ERR_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
    }
    if (lane == 0) st_relaxed64(dflags + blk, DL_INC | ((excl + count) & DL_VAL));
    return excl;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch along the render chain. Each kernel of the
// chain is launched with programmatic stream serialisation, so the GPU may
// schedule its blocks while the kernel before it drains; its first statement
// waits until that kernel has completed and its writes are visible, so the
// chain keeps plain stream order. Right after the wait it lets the next kernel
// be scheduled in turn. Both instructions are no-ops for a kernel launched
// without the attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void chain_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chain_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                     cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chain(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                                Args &&...args) {
    return launch_chain_smem(kernel, grid, block, 0, s, static_cast<Args &&>(args)...);
}

// Process-wide count of kernels this library has launched (sg_kernel_launches).
void count_launches(int n);

// ---- launchers (host side, defined in the .cu files) ----
// Up to N device regions of 32-bit words that the setup kernel zeroes.
// Regions the setup kernel fills: word i of region r gets even[r] if i is
// even, else 0 (even[r] = 0: plain zeroing).
struct ZeroRegions {
    static constexpr int N = 5;
    uint32_t *ptr[N] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint64_t words[N] = {0, 0, 0, 0, 0};
    uint32_t even[N] = {0, 0, 0, 0, 0};
};
cudaError_t launch_setup(const Batch &b, Batch *dst, uint64_t *counters, cudaStream_t s,
                         const ZeroRegions &z = ZeroRegions());
// clamp [M]: bit ch set where colour channel ch was clamped by max(c, 0)
cudaError_t launch_preprocess(const Batch &hb, const Batch *db, Rec *rec, uint32_t *tiles_touched,
                              uint2 *rect, uint32_t *dkey, uint32_t *dval, uint8_t *clamp, cudaStream_t s);
cudaError_t launch_preprocess_backward(const Batch &hb, const Batch *db,
                                       const uint32_t *tiles_touched, const uint8_t *clamp, const float *dg,
                                       uint64_t M, cudaStream_t s);

// Exclusive scan of `in` (or of tiles_touched[idx[i]] when idx != null) into
// `out`, total written to *total. n items (host known), or min(n, *n_dev) when
// n_dev is given. mirror (nullable, host memory mapped into the device): also
// receives the total and *status_src in its first two words.
cudaError_t launch_scan(const uint32_t *in, const uint32_t *gather_idx, uint32_t *out,
                        uint64_t n, uint64_t *block_sums, uint64_t *total, cudaStream_t s,
                        const uint64_t *n_dev = nullptr, uint64_t *mirror = nullptr,
                        const uint64_t *status_src = nullptr);

// Stable LSD radix sort of (key, val) u32 pairs on bits [0, bits); item count read
// from *n_dev and clamped to max_n (the capacity the launch is sized for, below
// 2^30). Ping-pongs between (k0,v0) and (k1,v1); the sorted result ends in
// (k0,v0) when the pass count is even, else in (k1,v1).
// hist: 4 x RS_RADIX x ceil(max_n / RS_TILE) words of look-back flags (one region
// per pass, zeroed by the sort itself); aux: at least
// SORT_AUX_BYTES; status (nullable): set to SG_ERR_TIMEOUT if a look-back gave up.
// kept_out (nullable): drop mode — keys equal to SORT_DROP_KEY are left out, the
// sorted kept keys fill positions [0, *kept_out) and *kept_out receives their count.
constexpr size_t SORT_AUX_BYTES = 16384;
// Most keys one sort takes (its look-back words carry 30-bit counts).
constexpr uint64_t SORT_MAX_KEYS = (1ull << 30) - 1;
constexpr uint32_t SORT_DROP_KEY = 0xFFFFFFFFu;
// aux_zeroed: the caller has already zeroed the aux region in this stream.
// hist_ready: the caller has also written every pass's digit histogram into
// aux and zeroed the sort_flag_words(max_n, bits) look-back words of hist.
// status_mirror (nullable): receives *status after the sort (host memory mapped
// into the device, read by the host behind an event).
// skip_status (nullable): when it holds a status other than SG_OK (a bounded
// wait gave up, so the input may hold stale words the histograms do not count;
// or the pairs overflowed the capacity) the passes do nothing.
// ranges (nullable): keys are ids below n_ranges; the sort also writes each
// id's [first, last + 1) position range in the sorted output, (0, 0) for an id
// with no key. On entry every range must hold (RANGE_EMPTY, 0).
constexpr uint32_t RANGE_EMPTY = 0xFFFFFFFFu;
cudaError_t launch_radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                              const uint64_t *n_dev, uint64_t max_n, int bits, uint32_t *hist,
                              uint64_t *aux, cudaStream_t s, uint64_t *status = nullptr,
                              uint64_t *kept_out = nullptr, bool aux_zeroed = false, uint2 *ranges = nullptr,
                              uint64_t n_ranges = 0, bool hist_ready = false, uint64_t *status_mirror = nullptr,
                              const uint64_t *skip_status = nullptr, uint32_t *order_counts = nullptr);
int radix_passes(int bits);
// Bound on a sort block's polls of an unpublished predecessor before it gives
// up and records SG_ERR_TIMEOUT (0: the default, 2^20).
void set_sort_wait_polls(uint32_t polls);
uint32_t sort_wait_polls();
// Look-back flag words a sort of up to max_n keys of `bits` bits uses.
uint64_t sort_flag_words(uint64_t max_n, int bits);

// duplicateWithKeys over the depth-sorted entries. Every block of 256 entries
// finds the offset of its pairs by a decoupled look-back over its predecessors'
// pair counts (dup_flags: div_up(M, 256) zeroed 64-bit words, and
// counters[CNT_DUP_BLOCK] zeroed), so no separate scan runs. The last block
// writes the pair total to counters[CNT_PAIRS] (and to mirror[0], host memory
// mapped into the device, when given), min(total, cap) to counters[CNT_WRITTEN],
// and SG_ERR_CAPACITY to counters[CNT_STATUS] when the pairs exceed cap; pairs
// at positions >= cap are not written. A status of SG_ERR_TIMEOUT on entry
// (a sort gave up a bounded wait) makes the kernel write nothing.
// key16: the keys are written as uint16_t (tile ids below 2^16, for the
// counting tile sort; no digit histograms then), else as uint32_t.
cudaError_t launch_duplicate(const Batch *db, uint64_t M, const uint32_t *sorted_ent,
                             const uint32_t *tiles_touched, const uint2 *rect, const Rec *rec,
                             uint64_t *counters, uint64_t cap, void *pkey, uint32_t *pval,
                             uint64_t *dup_flags, uint64_t *mirror, cudaStream_t s, int hist_passes = 0,
                             uint64_t *sort_aux = nullptr, uint32_t *flags = nullptr, uint64_t flag_words = 0,
                             bool key16 = false);
// Tile sort by counting, for tile counts up to TC_MAX_TILES (one chunk's
// counters fit 48 KB of shared memory): a stable sort by tile of the
// duplicate's (tile, entry) pairs, the same order as launch_radix_sort's, in
// three kernels with no pass over the key bits; the keys (tile ids) are
// 16-bit, as the duplicate writes them for it. Only the entries are written
// (ovals, cap words): a pair's tile is the tile whose range holds it. The pair
// count is min(counters[CNT_WRITTEN], cap), none when counters[CNT_STATUS] is
// not SG_OK on entry. matrix: n_chunks x tc_row(n_tiles) words (no zeroing
// needed); words: zeroed, 8 + 8 * ceil(n_tiles / 32) bytes; ranges: every
// tile's [first, last + 1) in the output ((0, 0) when empty); order_counts:
// the tile order's zeroed bucket counts, incremented here; status_mirror
// (nullable): receives counters[CNT_STATUS] after the sort. cap below 2^32.
constexpr uint32_t TC_MAX_TILES = 12288;
#ifndef SG_TC_MAX_CHUNKS
#define SG_TC_MAX_CHUNKS 608
#endif
constexpr uint32_t TC_MAX_CHUNKS = SG_TC_MAX_CHUNKS;   // four one-warp placing blocks per SM
constexpr uint64_t TC_CHUNK_TARGET = 8192;            // pairs per chunk when the capacity is small
uint32_t tc_chunks(uint64_t cap);                      // chunks of a sort sized for cap pairs
uint64_t tc_row(uint64_t n_tiles);                     // words per row of the count matrix (multiple of 4)
cudaError_t launch_tile_count_sort(const uint16_t *keys, const uint32_t *vals, uint32_t *ovals,
                                   uint64_t *counters, uint64_t cap, uint32_t n_tiles, uint32_t n_chunks,
                                   uint32_t *matrix, uint64_t *words, uint2 *ranges, uint32_t *order_counts,
                                   uint64_t *status_mirror, cudaStream_t s);
// Tiles by descending list length (256 length buckets) into order[n_tiles].
// scratch: TILE_ORDER_WORDS zeroed words whose first 256 already hold the
// bucket counts (launch_radix_sort's order_counts, filled by its finish kernel).
constexpr int TILE_ORDER_WORDS = 512;
cudaError_t launch_tile_order(const uint2 *ranges, uint32_t n_tiles, uint32_t *order, uint32_t *scratch,
                              cudaStream_t s);

// Blend launch shape.
struct BlendShape {
    int pixels_per_thread;
    bool persistent;              // resident blocks pull tiles from *queue
    const uint32_t *tile_order;   // persistent: tiles in this order (null: natural order)
    uint32_t *queue;              // persistent: zeroed work counter
    int grid;                     // persistent: resident blocks
    bool importance;              // forward: accumulate SceneDesc::importance
    const uint64_t *status;       // the forward's status word: SG_ERR_TIMEOUT = lists unusable
    int batch;                    // Gaussians staged per shared-memory batch
};

cudaError_t launch_blend_forward(const Batch *db, uint32_t n_tiles, const uint2 *ranges,
                                 const uint32_t *pval, const Rec *rec, float *img,
                                 float *T_final, int32_t *last, const BlendShape &shape,
                                 unsigned long long *evals, cudaStream_t s);
cudaError_t launch_blend_backward(const Batch *db, uint32_t n_tiles, const uint2 *ranges,
                                  const uint32_t *pval, const Rec *rec, const float *T_final,
                                  const int32_t *last, const float *d_img, float *dg,
                                  uint64_t M, const BlendShape &shape, unsigned long long *evals,
                                  cudaStream_t s);
// ADMM proximal + dual step (kind 0: opacity, 1: sharpness) and the penalty
// gradient term; workspace bytes for n items.
size_t admm_workspace_bytes(int64_t n);
cudaError_t launch_admm_step(int kind, int64_t n, const float *x, const float *score, const float *amp,
                             int64_t kappa, float *lam, float *x_tilde, void *ws, cudaStream_t s);
cudaError_t launch_penalty_grad(int64_t n, const float *x, const float *x_tilde, const float *lam, float delta,
                                float *grad, cudaStream_t s);

// Post-processing (Sec. 3.3.3): plan (flags, scans, totals read back) and apply.
size_t post_workspace_bytes(int64_t n);
cudaError_t launch_post_plan(const sg_scene &sc, float tau_o, float tau_s, void *ws, uint64_t *totals_host,
                             cudaStream_t s);
cudaError_t launch_post_apply(const sg_scene &sc, float tau_o, float tau_s, const void *ws, const sg_scene &out,
                              int64_t n_out, int64_t l_out, cudaStream_t s);

// Resident blocks per SM x SMs for the persistent blend of this shape.
int blend_persistent_grid(bool backward, int pixels_per_thread, int batch);

}  // namespace sgk
