// Tile blend (forward) and its adjoint.
//
// Front-to-back alpha blending of Sec. 3.1, C = sum_i c_i alpha_i T_i with
// T_i = prod_{j<i} (1 - alpha_j), under the compositing rules the paper keeps
// from 3DGS: power > 0 skips a pair, alpha = min(0.99, o' exp(power)),
// alpha < 1/255 skips, and the walk stops (without blending) at the first
// pair that would take T below 1e-4.
//
// One block per 16x16 tile, P pixels per thread (P in {1, 2, 4, 8}, picked at
// run time). Batches of 256 projected Gaussians are staged in shared memory; a
// block leaves its list as soon as every pixel is done (a block-wide vote), and
// threads whose pixels are all done skip the batch.
//
// The per-pair arithmetic that decides skips is written with explicitly
// rounded operations so the backward recomputes exactly the forward's
// decisions.
#include "sg_internal.cuh"

namespace sgk {

constexpr float ALPHA_MAX = 0.99f;
constexpr float T_STOP = 1e-4f;

__device__ __forceinline__ int find_tile_view(const Batch &b, uint32_t t) {
    int lo = 0, hi = b.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.view[mid].tile_off <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Shared-memory image of one projected Gaussian, prepared once per tile batch:
//   q = (x, y, qa, qb), r = (qc, o', red, green), s = blue
// with (qa, qb, qc) = -log2(e) * (A/2, B, C/2), so that
//   power * log2(e) = qa dx^2 + qb dx dy + qc dy^2   and   exp(power) = 2^(that).
constexpr float LOG2E = 1.4426950408889634f;
// Gaussians staged per shared-memory batch: a run-time choice (sg_tuning
// fwd_batch / bwd_batch) up to these sizes, which fix the shared memory.
constexpr int FWD_BATCH_MAX = 128;
constexpr int BWD_BATCH_MAX = 64;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2 of the opacity o' (a normal number wherever a pair is kept; a
// subnormal flushes to -inf, which skips every pair)
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

static_assert(BWD_BATCH_MAX % 32 == 0 && FWD_BATCH_MAX % 32 == 0, "batch sizes");
// Minimum resident blocks requested for the 8-pixels-per-thread backward.
#ifndef SG_BWD8_MIN_BLOCKS
#define SG_BWD8_MIN_BLOCKS 24
#endif

template <int NB>
struct StagedN {
    float4 q[NB];
    float4 r[NB];
    uint2 cm[NB];        // (bits of the third colour channel, sub-blocks of the tile the Gaussian can reach)
    uint32_t id[NB];
};
using StagedB = StagedN<BWD_BATCH_MAX>;

// A 16x16 tile is 8 sub-blocks of 8x4 pixels: sub-block s covers columns
// 8 (s & 1) .. +7 and rows 4 (s >> 1) .. +3 of the tile. Warp w's pixel slot j
// is sub-block w * P + j, lane l its pixel (l & 7, l >> 3).
constexpr int SUB_W = 8, SUB_H = 4;

// Bit s set unless no pixel centre of sub-block s lies in the enlarged ellipse
// q = d^T conic d <= t, t being the record's tile-binning bound (2 ln(255 o')
// grown by 1 % + 0.01, so every pixel where alpha can reach 1/255 lies inside;
// pixels left out are ones the alpha test would skip anyway: skipping them
// changes no result). Per band of 4 pixel rows, the ellipse's x-extent over the
// band is taken where its edges are extreme (the right edge at dy = -m, the
// left at dy = +m, m = B xmax / C, both clamped into the band) and compared
// with the tile's two 8-column halves. Padded by 0.05 px. The square roots and
// reciprocals are the approximate ones (relative error ~1e-6): the mask only
// has to cover the pixels where alpha reaches 1/255, and the 1 % growth of the
// bound already moves the ellipse's edge out by ~0.5 % of its radius.
__device__ __forceinline__ uint32_t reach_mask(const Rec &rc, float x0, float y0) {
    const float x = rc.a.x, y = rc.a.y, A = rc.a.z, B = rc.a.w, C = rc.b.x, t = rc.b.y;
    if (!(t >= 0.f)) return 0u;                      // o' < 1/255: alpha < 1/255 everywhere
    const float det = A * C - B * B;
    if (!(A > 0.f) || !(C > 0.f) || !(det > 0.f)) return 0xFFu;
    const float At = A * t, invdet = rcp_approx(det), invA = rcp_approx(A);
    const float ymax = sqrt_approx(At * invdet);
    const float m = B * sqrt_approx(C * t * invdet) * rcp_approx(C);
    if (!isfinite(ymax) || !isfinite(m) || !isfinite(invA)) return 0xFFu;
    constexpr float pad = 0.05f;
    uint32_t mask = 0u;
#pragma unroll
    for (int sy = 0; sy < TILE / SUB_H; ++sy) {
        const float lo = fmaxf(y0 + (float)(SUB_H * sy) - y - pad, -ymax);
        const float hi = fminf(y0 + (float)(SUB_H * sy + SUB_H - 1) - y + pad, ymax);
        if (!(lo <= hi)) continue;
        const float dr = fminf(fmaxf(-m, lo), hi), dl = fminf(fmaxf(m, lo), hi);
        const float sr = sqrt_approx(fmaxf(0.f, At - det * dr * dr));
        const float sl = sqrt_approx(fmaxf(0.f, At - det * dl * dl));
        const float xr = x + (sr - B * dr) * invA + pad - x0, xl = x - (sl + B * dl) * invA - pad - x0;
#pragma unroll
        for (int sx = 0; sx < TILE / SUB_W; ++sx)
            if (xr >= (float)(sx * SUB_W) && xl <= (float)(sx * SUB_W + SUB_W - 1))
                mask |= 1u << (sy * (TILE / SUB_W) + sx);
    }
    return mask;
}

// Staged per entry: q = (x, y, qa, qb), r = (qc, log2 o', c0, c1) with the
// conic scaled by -log2(e)/2 (qb by -log2(e)), so that at d = pixel - centre
//   power' = qa dx^2 + qb dx dy + qc dy^2 + log2 o' = log2(o' G),  alpha = min(0.99, 2^power').
// o' < 1/255 gives the entry no pair (its record's bound t is negative), so
// log2 o' is finite wherever a pair is evaluated with culling.
template <bool CULL, int NB>
__device__ __forceinline__ void stage(StagedN<NB> &sm, int slot, const Rec &rc, uint32_t e, float x0, float y0) {
    sm.q[slot] = make_float4(rc.a.x, rc.a.y, -0.5f * LOG2E * rc.a.z, -LOG2E * rc.a.w);
    sm.r[slot] = make_float4(-0.5f * LOG2E * rc.b.x, lg2_approx(rc.b.z), rc.b.w, rc.c.x);
    sm.cm[slot] = make_uint2(__float_as_uint(rc.c.y), CULL ? reach_mask(rc, x0, y0) : 0xFFu);
    sm.id[slot] = e;
}

// Pixel (column, row inside the tile) of slot j of this thread. For P >= 2 the
// slots 2i and 2i + 1 lie in the same pixel row (sub-blocks 2s and 2s + 1).
template <int P>
__device__ __forceinline__ void slot_pixel(int j, int &cx, int &cy) {
    const int sub = (int)(threadIdx.x >> 5) * P + j;
    const int lane = threadIdx.x & 31;
    cx = SUB_W * (sub & 1) + (lane & (SUB_W - 1));
    cy = SUB_H * (sub >> 1) + (lane / SUB_W);
}

// Slots that share one pixel row: 2 for P >= 2, else 1.
template <int P>
constexpr int row_slots() { return P >= 2 ? 2 : 1; }

// The terms of the quadratic form that depend on the pixel row only:
//   dy = y_pix - y, u = qc dy, b = qb dy, c = u dy + log2 o'
struct RowEval {
    float dy, u, b, c;
};

// ag = o' G = 2^power' (before the 0.99 clamp)
struct PairEval {
    float dx, p2, ag, alpha;
};

// log2(1/255): alpha >= 1/255 is decided on the exponent, power' >= this bound.
// The 3DGS rasterizer's power > 0 skip is left out: the dilated conic is
// positive definite, so power > 0 can only come from rounding at a pixel
// within ~1e-3 px of the centre, where the pair is kept.
constexpr float LOG2_ALPHA_MIN = -7.99435343685885793f;

// Every kernel that decides a skip evaluates a pair with this exact sequence of
// explicitly rounded operations, so the forward and the backward agree:
//   t = qa dx + qb dy,  power' = t dx + (qc dy^2 + log2 o').
__device__ __forceinline__ void eval_row(float fpy, const float4 &q, const float4 &r, RowEval &w) {
    w.dy = __fsub_rn(fpy, q.y);
    w.u = __fmul_rn(r.x, w.dy);
    w.b = __fmul_rn(q.w, w.dy);
    w.c = __fmaf_rn(w.u, w.dy, r.y);
}

__device__ __forceinline__ void eval_pixel(float fpx, const float4 &q, const RowEval &w, PairEval &p) {
    p.dx = __fsub_rn(fpx, q.x);
    const float t = __fmaf_rn(q.z, p.dx, w.b);
    p.p2 = __fmaf_rn(t, p.dx, w.c);
    p.ag = ex2_approx(p.p2);
    p.alpha = fminf(ALPHA_MAX, p.ag);
}

// The pair's skip rule (alpha < 1/255), on the exponent; NaN is skipped.
__device__ __forceinline__ bool pair_kept(const PairEval &p) { return p.p2 >= LOG2_ALPHA_MIN; }

__device__ __forceinline__ bool tile_of_block(const Batch &b, uint32_t tile, int &tx, int &ty,
                                              const ViewDesc *&vw) {
    vw = &b.view[find_tile_view(b, tile)];
    const uint32_t lt = tile - vw->tile_off;
    tx = (int)(lt % (uint32_t)vw->tiles_x);
    ty = (int)(lt / (uint32_t)vw->tiles_x);
    return true;
}

// Sums a per-thread count over the warp into *evals (counting variants only).
__device__ __forceinline__ void add_evals(uint32_t ne, unsigned long long *evals) {
    const uint32_t w = __reduce_add_sync(0xffffffffu, ne);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(evals, (unsigned long long)w);
}

// ---------------------------------------------------------------------------
// K6 blend forward: one block per tile, P pixels per thread
// ---------------------------------------------------------------------------
// Warp w owns sub-blocks w P .. w P + P - 1 of the tile, one 8x4 sub-block per
// pixel slot, so that a Gaussian whose reach misses a sub-block is skipped by
// the whole warp at once (NT = 256 / P threads per tile).
// Forward modes: plain, counting (pair evaluations, no culling), importance
// (also sums alpha T per Gaussian into its scene's importance array).
enum : int { FWD_PLAIN = 0, FWD_COUNT = 1, FWD_IMPORTANCE = 2 };

// lists_ok false: a sort's bounded wait gave up in this forward (its lists may
// hold stale words): every tile renders as an empty list. (On a capacity
// overflow the tile sort does not run and every range stays empty.)
template <int P, int MODE, int NB>
__device__ __forceinline__ void blend_fwd_tile(const Batch &b, uint32_t tile, StagedN<NB> &sm,
                                               const uint2 *__restrict__ ranges,
                                               const uint32_t *__restrict__ pval,
                                               const Rec *__restrict__ rec, float *__restrict__ img,
                                               float *__restrict__ T_final, int32_t *__restrict__ last,
                                               uint32_t &ne, bool lists_ok, float *__restrict__ part) {
    constexpr int NT = BLEND_THREADS / P;
    constexpr bool COUNT = MODE == FWD_COUNT;
    constexpr bool IMP = MODE == FWD_IMPORTANCE;
    constexpr int PS = NB + 1;   // importance partials: part[thread * PS + entry], zero between batches
    int tx, ty;
    const ViewDesc *vw;
    tile_of_block(b, tile, tx, ty, vw);
    const uint2 rg = ranges[tile];
    const int n = lists_ok ? (int)(rg.y - rg.x) : 0;
    float *imp = IMP ? b.scene[vw->scene].importance : nullptr;

    float fpx[P], fpy[P], T[P], c0[P], c1[P], c2[P];
    int lastc[P];
    bool done[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        int cx, cy;
        slot_pixel<P>(j, cx, cy);
        const int px = tx * TILE + cx, py = ty * TILE + cy;
        fpx[j] = (float)px;
        fpy[j] = (float)py;
        T[j] = 1.f;
        c0[j] = c1[j] = c2[j] = 0.f;
        lastc[j] = 0;
        done[j] = !(px < vw->W && py < vw->H);
    }
    const int sub0 = (int)(threadIdx.x >> 5) * P;
    const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
    // Importance: each thread leaves its share of Sum alpha T (over its pixels) for
    // entry k of the batch in part[thread][k]; after the block's next barrier,
    // thread k sums column k, zeroes it and adds the total to the Gaussian's
    // score with one atomic (no warp collective per list entry).
    int pending = 0;   // entries of the last batch whose partials are not yet summed
    auto flush = [&]() {
        for (int k = threadIdx.x; k < pending; k += NT) {
            float sum = 0.f;
            for (int t = 0; t < NT; ++t) {
                sum += part[t * PS + k];
                part[t * PS + k] = 0.f;
            }
            // only an entry of this view's scene (a stale id from another view is left out)
            const uint32_t li = sm.id[k] - (uint32_t)vw->ent_off;
            if (sum != 0.f && li < (uint32_t)vw->n) atomicAdd(imp + li, sum);
        }
        pending = 0;
    };
    for (int base = 0; base < n; base += NB) {
        bool all = true;
#pragma unroll
        for (int j = 0; j < P; ++j) all = all && done[j];
        const bool stop = __syncthreads_count(all) == NT;
        if (IMP && pending) {   // uniform
            flush();
            __syncthreads();   // before the staging below overwrites the batch's ids
        }
        if (stop) break;
        const int cnt = min(NB, n - base);
        for (int k = threadIdx.x; k < cnt; k += NT) {
            const uint32_t e = pval[rg.x + base + k];
            stage<!COUNT>(sm, k, rec[e], e, x0, y0);
        }
        __syncthreads();
        if (IMP) pending = cnt;
        if (all) continue;
        // unrolled by 8 (measured: 3 % fewer cycles than no unrolling)
#pragma unroll 8
        for (int k = 0; k < cnt; ++k) {
            const uint2 cm = sm.cm[k];
            const uint32_t msk = cm.y >> sub0;
            if ((msk & ((1u << P) - 1u)) == 0u) continue;   // warp-uniform
            const float4 q = sm.q[k], r = sm.r[k];
            const float bl = __uint_as_float(cm.x);
            float wsum = 0.f;
            constexpr int RS = row_slots<P>();
#pragma unroll
            for (int j0 = 0; j0 < P; j0 += RS) {
                const uint32_t bits = (msk >> j0) & ((1u << RS) - 1u);
                if (!bits) continue;                           // warp-uniform
                RowEval row;
                eval_row(fpy[j0], q, r, row);
                // both pixels of the row first, with no branch between them
                PairEval pe[RS];
                bool ok[RS];
#pragma unroll
                for (int h = 0; h < RS; ++h) {
                    const int j = j0 + h;
                    eval_pixel(fpx[j], q, row, pe[h]);
                    const bool live = ((bits >> h) & 1u) && !done[j];
                    if (COUNT) ne += live ? 1u : 0u;
                    ok[h] = live && pair_kept(pe[h]);
                }
#pragma unroll
                for (int h = 0; h < RS; ++h) {
                    const int j = j0 + h;
                    if (!ok[h]) continue;
                    const PairEval &p = pe[h];
                    // T (1 - alpha) as T - alpha T
                    const float w = __fmul_rn(p.alpha, T[j]);
                    const float tt = __fsub_rn(T[j], w);
                    if (tt < T_STOP) { done[j] = true; continue; }
                    c0[j] = fmaf(r.z, w, c0[j]);
                    c1[j] = fmaf(r.w, w, c1[j]);
                    c2[j] = fmaf(bl, w, c2[j]);
                    T[j] = tt;
                    lastc[j] = base + k + 1;
                    if (IMP) wsum += w;
                }
            }
            if (IMP && wsum != 0.f) part[threadIdx.x * PS + k] = wsum;
        }
    }
    if (IMP) {
        __syncthreads();   // every thread's partials of the last batch are in
        flush();
        __syncthreads();   // the next tile's staging (persistent form) overwrites the ids
    }
    const uint64_t HW = (uint64_t)vw->W * (uint64_t)vw->H;
    float *im = img + 3 * vw->pix_off;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int px = (int)fpx[j], py = (int)fpy[j];
        if (px < vw->W && py < vw->H) {
            const uint64_t pix = (uint64_t)py * (uint64_t)vw->W + (uint64_t)px;
            im[pix] = c0[j] + T[j] * vw->bg[0];
            im[HW + pix] = c1[j] + T[j] * vw->bg[1];
            im[2 * HW + pix] = c2[j] + T[j] * vw->bg[2];
            T_final[vw->pix_off + pix] = T[j];
            last[vw->pix_off + pix] = lastc[j];
        }
    }
}

// Persistent form: resident blocks pull tiles from a work counter in the
// given order (longest lists first); otherwise one block per tile.
template <int P, int MODE, bool PERSIST, int NB>
__global__ void __launch_bounds__(BLEND_THREADS / P)
k_blend_fwd(const Batch *__restrict__ bp, const uint2 *__restrict__ ranges,
            const uint32_t *__restrict__ pval, const Rec *__restrict__ rec,
            float *__restrict__ img, float *__restrict__ T_final, int32_t *__restrict__ last,
            const uint32_t *__restrict__ tile_order, uint32_t *__restrict__ queue, uint32_t n_tiles,
            unsigned long long *__restrict__ evals, const uint64_t *__restrict__ status) {
    chain_enter();
    __shared__ StagedN<NB> sm;
    __shared__ float part[MODE == FWD_IMPORTANCE ? (BLEND_THREADS / P) * (NB + 1) : 1];
    __shared__ uint32_t s_item;
    const Batch &b = *bp;
    uint32_t ne = 0;
    const bool lists_ok = *status != (uint64_t)SG_ERR_TIMEOUT;
    if (MODE == FWD_IMPORTANCE) {
        for (int i = threadIdx.x; i < (BLEND_THREADS / P) * (NB + 1); i += BLEND_THREADS / P) part[i] = 0.f;
        __syncthreads();
    }
    if (!PERSIST) {
        blend_fwd_tile<P, MODE, NB>(b, blockIdx.x, sm, ranges, pval, rec, img, T_final, last, ne, lists_ok, part);
    } else {
        for (;;) {
            if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
            __syncthreads();
            const uint32_t item = s_item;
            __syncthreads();
            if (item >= n_tiles) break;
            blend_fwd_tile<P, MODE, NB>(b, tile_order ? tile_order[item] : item, sm, ranges, pval, rec, img,
                                        T_final, last, ne, lists_ok, part);
        }
    }
    if (MODE == FWD_COUNT) add_evals(ne, evals);
}

template <int P, int MODE, bool PERSIST, int NB>
static void fwd_launch(const Batch *db, uint32_t n_tiles, const uint2 *ranges, const uint32_t *pval,
                       const Rec *rec, float *img, float *T_final, int32_t *last, const BlendShape &sh,
                       unsigned long long *evals, cudaStream_t s) {
    const unsigned grid = PERSIST ? (unsigned)sh.grid : n_tiles;
    (void)launch_chain(k_blend_fwd<P, MODE, PERSIST, NB>, dim3(grid), dim3(BLEND_THREADS / P), s,
        db, ranges, pval, rec, img, T_final, last, sh.tile_order, sh.queue, n_tiles, evals, sh.status);
}

// The plain forward takes the batch size of the tuning; the counting form
// takes 64 and the importance form 32 (its per-thread partials of a batch sit in
// shared memory); the batch changes no result.
template <int P, bool PERSIST>
static void fwd_p(const Batch *db, uint32_t n_tiles, const uint2 *ranges, const uint32_t *pval,
                  const Rec *rec, float *img, float *T_final, int32_t *last, const BlendShape &sh,
                  unsigned long long *evals, cudaStream_t s) {
    if (evals)
        fwd_launch<P, FWD_COUNT, PERSIST, 64>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, evals, s);
    else if (sh.importance)
        fwd_launch<P, FWD_IMPORTANCE, PERSIST, 32>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh,
                                                   nullptr, s);
    else if (sh.batch == 32)
        fwd_launch<P, FWD_PLAIN, PERSIST, 32>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, nullptr, s);
    else if (sh.batch == 128)
        fwd_launch<P, FWD_PLAIN, PERSIST, 128>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, nullptr, s);
    else
        fwd_launch<P, FWD_PLAIN, PERSIST, 64>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, nullptr, s);
}

template <bool PERSIST>
static cudaError_t fwd_dispatch(const Batch *db, uint32_t n_tiles, const uint2 *ranges, const uint32_t *pval,
                                const Rec *rec, float *img, float *T_final, int32_t *last,
                                const BlendShape &sh, unsigned long long *evals, cudaStream_t s) {
    switch (sh.pixels_per_thread) {
        case 1: fwd_p<1, PERSIST>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, evals, s); break;
        case 2: fwd_p<2, PERSIST>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, evals, s); break;
        case 4: fwd_p<4, PERSIST>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, evals, s); break;
        case 8: fwd_p<8, PERSIST>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, evals, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_blend_forward(const Batch *db, uint32_t n_tiles, const uint2 *ranges,
                                 const uint32_t *pval, const Rec *rec, float *img, float *T_final,
                                 int32_t *last, const BlendShape &sh, unsigned long long *evals,
                                 cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    const bool persist = sh.persistent;
    if (persist && (sh.grid <= 0 || sh.queue == nullptr)) return cudaErrorInvalidValue;
    if (sh.status == nullptr || sh.batch < 32 || sh.batch > FWD_BATCH_MAX || sh.batch % 32 != 0)
        return cudaErrorInvalidValue;
    cudaError_t e = persist ? fwd_dispatch<true>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, evals, s)
                            : fwd_dispatch<false>(db, n_tiles, ranges, pval, rec, img, T_final, last, sh, evals, s);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K7 blend backward
// ---------------------------------------------------------------------------
// Sums 9 per-lane values over the warp and adds them to dg[k*M + e] (value k
// scaled by sc[k]). Recursive halving: 4 + 2 + 1 shuffles leave each group of
// four lanes with one of the first eight sums, two more finish it; the ninth
// value takes a plain butterfly. Eight lanes issue their atomics together.
__device__ __forceinline__ void warp_sum9_atomic(const float v[9], float *dg, uint64_t M, uint32_t e) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool h1 = lane & 16, h2 = lane & 8, h3 = lane & 4;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float keep = h1 ? v[i + 4] : v[i];
        const float send = h1 ? v[i] : v[i + 4];
        a[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
    float b2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = h2 ? a[i + 2] : a[i];
        const float send = h2 ? a[i] : a[i + 2];
        b2[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    float c = (h3 ? b2[1] : b2[0]) + __shfl_xor_sync(FULL, h3 ? b2[0] : b2[1], 4);
    c += __shfl_xor_sync(FULL, c, 2);
    c += __shfl_xor_sync(FULL, c, 1);
    float d = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(FULL, d, o);
    if ((lane & 3) == 0) {
        const int idx = (h1 ? 4 : 0) + (h2 ? 2 : 0) + (h3 ? 1 : 0);
        atomicAdd(dg + (uint64_t)idx * M + e, c);
    }
    if (lane == 1) atomicAdd(dg + 8 * M + e, d);
}

// Adds one pixel's share of one blended pair to v (in dg order) and steps the
// pixel's T and Sg back over the pair.
__device__ __forceinline__ void bwd_adjoint(const PairEval &p, float dy, const float4 &r, float bl,
                                            float &T, float &Sg, float g0, float g1, float g2, float v[9]) {
    const float oma = __fsub_rn(1.f, p.alpha);
    const float ro = rcp_approx(oma);
    const float Ti = T * ro;
    const float w = p.alpha * Ti;
    const float cg = fmaf(r.z, g0, fmaf(r.w, g1, bl * g2));
    const float dal = Ti * cg - Sg * ro;
    Sg = fmaf(cg, w, Sg);
    T = Ti;
    v[6] = fmaf(w, g0, v[6]);
    v[7] = fmaf(w, g1, v[7]);
    v[8] = fmaf(w, g2, v[8]);
    // dP = dL/dpower = dL/dalpha o' G, none where the 0.99 clamp is active
    // (dL/do' = dP / o': the division is applied once per Gaussian)
    const float dP = p.ag > ALPHA_MAX ? 0.f : dal * p.ag;
    v[5] += dP;
    const float hx = dP * p.dx, hy = dP * dy;
    v[0] += hx;                          // sum dP dx
    v[1] += hy;                          // sum dP dy
    v[2] = fmaf(hx, p.dx, v[2]);         // sum dP dx^2
    v[3] = fmaf(hx, dy, v[3]);           // sum dP dx dy
    v[4] = fmaf(hy, dy, v[4]);           // sum dP dy^2
}

// Per pixel the walk runs back from the pixel's last blended pair, recovering
// the transmittance before each pair as T_i = T_{i+1} / (1 - alpha_i) and
// keeping Sg = sum over later pairs of (c . g) alpha T, so that
//   dL/dalpha_i = T_i (c_i . g) - (Sg + T_final (bg . g)) / (1 - alpha_i).
// Per-thread sums over its P pixels are reduced over the warp before the
// atomics. Accumulated per pair (in dg order), with dP = dL/dpower =
// dL/dalpha o' G (alpha = o' G below the clamp) and (dx, dy) = pixel - centre:
//   0,1: sum dP dx, sum dP dy   2..4: sum dP dx^2, sum dP dx dy, sum dP dy^2
//   5: sum dP (= o' dL/do')   6..8: dL/drgb
// lists_ok false: a sort of the forward gave up a bounded wait (its lists may
// hold stale words): no pair contributes.
template <int P, bool COUNT>
__device__ __forceinline__ void blend_bwd_tile(const Batch &b, uint32_t tile, StagedB &sm, int *smax,
                                               float4 *__restrict__ spx, int *__restrict__ slot_last,
                                               const uint2 *__restrict__ ranges,
                                               const uint32_t *__restrict__ pval,
                                               const Rec *__restrict__ rec,
                                               const float *__restrict__ T_final,
                                               const int32_t *__restrict__ last,
                                               const float *__restrict__ d_img, float *__restrict__ dg,
                                               uint64_t M, uint32_t &ne, bool lists_ok, int nb) {
    constexpr int NT = BLEND_THREADS / P;
    int tx, ty;
    const ViewDesc *vw;
    tile_of_block(b, tile, tx, ty, vw);
    const uint2 rg = ranges[tile];
    const uint64_t HW = (uint64_t)vw->W * (uint64_t)vw->H;
    const float *gi = d_img + 3 * vw->pix_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub0 = warp * P;

    // Per pixel slot: T and Sg in registers (they change along the walk); the
    // upstream gradient and the last blended position, read-only here, in
    // this thread's own shared-memory slots (one 16-byte word per pixel:
    // g0, g1, g2, last), which keeps registers for more resident warps.
    // Sg starts at T_final (bg . g), the background's share of every dL/dalpha.
    // slot_last[s]: the largest last position over the pixels of sub-block s.
    float T[P], Sg[P];
    int tmax = 0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        int cx, cy;
        slot_pixel<P>(j, cx, cy);
        const int px = tx * TILE + cx, py = ty * TILE + cy;
        float4 pg = make_float4(0.f, 0.f, 0.f, __int_as_float(0));
        T[j] = 1.f;
        Sg[j] = 0.f;
        int lst = 0;
        if (px < vw->W && py < vw->H) {
            const uint64_t pix = (uint64_t)py * (uint64_t)vw->W + (uint64_t)px;
            lst = last[vw->pix_off + pix];
            const float tf = T_final[vw->pix_off + pix];
            pg = make_float4(gi[pix], gi[HW + pix], gi[2 * HW + pix], __int_as_float(lst));
            T[j] = tf;
            Sg[j] = tf * (pg.x * vw->bg[0] + pg.y * vw->bg[1] + pg.z * vw->bg[2]);
        }
        spx[(sub0 + j) * 32 + lane] = pg;
        const int sl = __reduce_max_sync(0xffffffffu, lst);
        if (lane == 0) slot_last[sub0 + j] = sl;
        tmax = max(tmax, lst);
    }
    const int wmax = __reduce_max_sync(0xffffffffu, tmax);
    if (lane == 0) smax[warp] = wmax;
    __syncthreads();
    int maxlast = 0;
#pragma unroll
    for (int i = 0; i < (NT + 31) / 32; ++i) maxlast = max(maxlast, smax[i]);
    if (!lists_ok) maxlast = 0;
    const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);

    // Slots with a pixel whose walk reaches position pos (slot_last > pos):
    // walking back, a slot turns live once and stays live, so the mask is
    // rebuilt only when pos drops below the next slot's last (at most P times).
    uint32_t live_slots = 0u;
    int next_on = 0x7fffffff;   // rebuild when pos < next_on
    for (int end = maxlast; end > 0; end -= nb) {
        const int start = max(0, end - nb);
        const int cnt = end - start;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += NT) {
            const uint32_t e = pval[rg.x + start + k];
            stage<!COUNT>(sm, k, rec[e], e, x0, y0);
        }
        __syncthreads();
        // warps whose pixels all end before this batch have nothing to add
        if (__all_sync(0xffffffffu, tmax <= start)) continue;
        for (int k = cnt - 1; k >= 0; --k) {
            const int pos = start + k;
            if (pos < next_on) {   // warp-uniform
                live_slots = 0u;
                int nx = -1;
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const int sl = slot_last[sub0 + j];
                    if (sl > pos) live_slots |= 1u << j;
                    else nx = max(nx, sl);
                }
                next_on = nx;   // the next slot turns live once pos drops below its last
            }
            const uint2 cm = sm.cm[k];
            const uint32_t msk = (cm.y >> sub0) & live_slots;
            if ((msk & ((1u << P) - 1u)) == 0u) continue;   // warp-uniform
            const float4 q = sm.q[k], r = sm.r[k];
            const float bl = __uint_as_float(cm.x);
            float v[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = 0.f;
            bool any = false;
            constexpr int RS = row_slots<P>();
#pragma unroll
            for (int j0 = 0; j0 < P; j0 += RS) {
                const uint32_t bits = (msk >> j0) & ((1u << RS) - 1u);
                if (!bits) continue;                           // warp-uniform
                float4 pg[RS];
#pragma unroll
                for (int hh = 0; hh < RS; ++hh) pg[hh] = spx[(sub0 + j0 + hh) * 32 + lane];
                int cx, cy;
                slot_pixel<P>(j0, cx, cy);
                RowEval row;
                eval_row((float)(ty * TILE + cy), q, r, row);
                // both pixels of the row first, with no branch between them
                PairEval pe[RS];
                bool ok[RS];
#pragma unroll
                for (int hh = 0; hh < RS; ++hh) {
                    slot_pixel<P>(j0 + hh, cx, cy);
                    eval_pixel((float)(tx * TILE + cx), q, row, pe[hh]);
                    const bool live = ((bits >> hh) & 1u) && pos < __float_as_int(pg[hh].w);
                    if (COUNT) ne += live ? 1u : 0u;
                    ok[hh] = live && pair_kept(pe[hh]);
                }
#pragma unroll
                for (int hh = 0; hh < RS; ++hh) {
                    const int j = j0 + hh;
                    if (!ok[hh]) continue;
                    any = true;
                    bwd_adjoint(pe[hh], row.dy, r, bl, T[j], Sg[j], pg[hh].x, pg[hh].y, pg[hh].z, v);
                }
            }
            // the moments are linear in dP: the conic factors and 1/o' are applied
            // once per entry by the preprocess adjoint, after the sum over tiles
            if (__any_sync(0xffffffffu, any)) warp_sum9_atomic(v, dg, M, sm.id[k]);
        }
    }
}

template <int P, bool COUNT, bool PERSIST>
__global__ void __launch_bounds__(BLEND_THREADS / P, P == 8 ? SG_BWD8_MIN_BLOCKS : 1)
k_blend_bwd(const Batch *__restrict__ bp, const uint2 *__restrict__ ranges,
            const uint32_t *__restrict__ pval, const Rec *__restrict__ rec,
            const float *__restrict__ T_final, const int32_t *__restrict__ last,
            const float *__restrict__ d_img, float *__restrict__ dg, uint64_t M,
            const uint32_t *__restrict__ tile_order, uint32_t *__restrict__ queue, uint32_t n_tiles,
            unsigned long long *__restrict__ evals, const uint64_t *__restrict__ status, int nb) {
    chain_enter();
    constexpr int NT = BLEND_THREADS / P;
    __shared__ StagedB sm;
    __shared__ float4 spx[BLEND_THREADS];   // per pixel slot: upstream gradient and last position
    __shared__ int slot_last[BLEND_THREADS / 32];
    __shared__ int smax[(NT + 31) / 32];
    __shared__ uint32_t s_item;
    const Batch &b = *bp;
    uint32_t ne = 0;
    const bool lists_ok = *status != (uint64_t)SG_ERR_TIMEOUT;
    if (!PERSIST) {
        blend_bwd_tile<P, COUNT>(b, blockIdx.x, sm, smax, spx, slot_last, ranges, pval, rec, T_final, last,
                                 d_img, dg, M, ne, lists_ok, nb);
    } else {
        for (;;) {
            if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
            __syncthreads();
            const uint32_t item = s_item;
            __syncthreads();
            if (item >= n_tiles) break;
            blend_bwd_tile<P, COUNT>(b, tile_order ? tile_order[item] : item, sm, smax, spx, slot_last, ranges,
                                     pval, rec, T_final, last, d_img, dg, M, ne, lists_ok, nb);
        }
    }
    if (COUNT) add_evals(ne, evals);
}

template <int P, bool PERSIST>
static void bwd_p(const Batch *db, uint32_t n_tiles, const uint2 *ranges, const uint32_t *pval,
                  const Rec *rec, const float *T_final, const int32_t *last, const float *d_img, float *dg,
                  uint64_t M, const BlendShape &sh, unsigned long long *evals, cudaStream_t s) {
    const unsigned grid = PERSIST ? (unsigned)sh.grid : n_tiles;
    if (evals)
        (void)launch_chain(k_blend_bwd<P, true, PERSIST>, dim3(grid), dim3(BLEND_THREADS / P), s,
            db, ranges, pval, rec, T_final, last, d_img, dg, M, sh.tile_order, sh.queue, n_tiles, evals, sh.status, sh.batch);
    else
        (void)launch_chain(k_blend_bwd<P, false, PERSIST>, dim3(grid), dim3(BLEND_THREADS / P), s,
            db, ranges, pval, rec, T_final, last, d_img, dg, M, sh.tile_order, sh.queue, n_tiles, nullptr, sh.status, sh.batch);
}

template <bool PERSIST>
static cudaError_t bwd_dispatch(const Batch *db, uint32_t n_tiles, const uint2 *ranges, const uint32_t *pval,
                                const Rec *rec, const float *T_final, const int32_t *last, const float *d_img,
                                float *dg, uint64_t M, const BlendShape &sh, unsigned long long *evals,
                                cudaStream_t s) {
    switch (sh.pixels_per_thread) {
        case 1: bwd_p<1, PERSIST>(db, n_tiles, ranges, pval, rec, T_final, last, d_img, dg, M, sh, evals, s); break;
        case 2: bwd_p<2, PERSIST>(db, n_tiles, ranges, pval, rec, T_final, last, d_img, dg, M, sh, evals, s); break;
        case 4: bwd_p<4, PERSIST>(db, n_tiles, ranges, pval, rec, T_final, last, d_img, dg, M, sh, evals, s); break;
        case 8: bwd_p<8, PERSIST>(db, n_tiles, ranges, pval, rec, T_final, last, d_img, dg, M, sh, evals, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_blend_backward(const Batch *db, uint32_t n_tiles, const uint2 *ranges,
                                  const uint32_t *pval, const Rec *rec, const float *T_final,
                                  const int32_t *last, const float *d_img, float *dg, uint64_t M,
                                  const BlendShape &sh, unsigned long long *evals, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    const bool persist = sh.persistent;
    if (persist && (sh.grid <= 0 || sh.queue == nullptr)) return cudaErrorInvalidValue;
    if (sh.status == nullptr || sh.batch < 32 || sh.batch > BWD_BATCH_MAX || sh.batch % 32 != 0)
        return cudaErrorInvalidValue;
    cudaError_t e = persist
        ? bwd_dispatch<true>(db, n_tiles, ranges, pval, rec, T_final, last, d_img, dg, M, sh, evals, s)
        : bwd_dispatch<false>(db, n_tiles, ranges, pval, rec, T_final, last, d_img, dg, M, sh, evals, s);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// persistent grid: resident blocks per SM (occupancy) x SMs, per device
// ---------------------------------------------------------------------------
template <typename K>
static int occupancy_grid(K kernel, int threads) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess) return 0;
    return sms * (per > 0 ? per : 1);
}

template <int NB>
static int fwd_grid(int p) {
    switch (p) {
        case 1: return occupancy_grid(k_blend_fwd<1, FWD_PLAIN, true, NB>, 256);
        case 2: return occupancy_grid(k_blend_fwd<2, FWD_PLAIN, true, NB>, 128);
        case 4: return occupancy_grid(k_blend_fwd<4, FWD_PLAIN, true, NB>, 64);
        case 8: return occupancy_grid(k_blend_fwd<8, FWD_PLAIN, true, NB>, 32);
    }
    return 0;
}

int blend_persistent_grid(bool backward, int p, int batch) {
    // cached per (device, direction, shape, forward batch); devices beyond 16 are computed each time
    static int cache[16][2][9][3] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int bi = backward ? 0 : (batch == 32 ? 0 : batch == 128 ? 2 : 1);
    const bool cacheable = dev >= 0 && dev < 16 && p >= 1 && p <= 8;
    if (cacheable && cache[dev][backward][p][bi]) return cache[dev][backward][p][bi];
    int g = 0;
    if (!backward) {
        g = bi == 0 ? fwd_grid<32>(p) : bi == 2 ? fwd_grid<128>(p) : fwd_grid<64>(p);
    } else {
        switch (p) {
            case 1: g = occupancy_grid(k_blend_bwd<1, false, true>, 256); break;
            case 2: g = occupancy_grid(k_blend_bwd<2, false, true>, 128); break;
            case 4: g = occupancy_grid(k_blend_bwd<4, false, true>, 64); break;
            case 8: g = occupancy_grid(k_blend_bwd<8, false, true>, 32); break;
        }
    }
    if (cacheable && g > 0) cache[dev][backward][p][bi] = g;
    return g;
}

}  // namespace sgk
