// Tile blend (forward) and its adjoint.
//
// Front-to-back alpha blending of Sec. 3.1, C = sum_i c_i alpha_i T_i with
// T_i = prod_{j<i} (1 - alpha_j), under the compositing rules the paper keeps
// from 3DGS: power > 0 skips a pair, alpha = min(0.99, o' exp(power)),
// alpha < 1/255 skips, and the walk stops (without blending) at the first
// pair that would take T below 1e-4.
//
// One 256-thread block per 16x16 tile, one pixel per thread. Batches of 256
// projected Gaussians are staged in shared memory; a block leaves its list
// as soon as every pixel is done (a block-wide vote), and a warp whose
// pixels are all done skips the batch.
//
// The per-pair arithmetic that decides skips is written with explicitly
// rounded operations so the backward recomputes exactly the forward's
// decisions.
#include "sg_internal.cuh"

namespace sgk {

constexpr float ALPHA_MIN = 1.0f / 255.0f;
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

struct PairEval {
    float dx, dy, power, G, ag, alpha;
};

// power = -1/2 (A dx^2 + C dy^2) - B dx dy with d = pixel - centre
__device__ __forceinline__ void eval_pair(float fpx, float fpy, const float4 &a, const float4 &b,
                                          PairEval &p) {
    p.dx = __fsub_rn(fpx, a.x);
    p.dy = __fsub_rn(fpy, a.y);
    const float cdy = __fmul_rn(__fmul_rn(b.x, p.dy), p.dy);
    const float q = __fmaf_rn(__fmul_rn(a.z, p.dx), p.dx, cdy);
    const float bxy = __fmul_rn(__fmul_rn(a.w, p.dx), p.dy);
    p.power = __fmaf_rn(-0.5f, q, -bxy);
    p.G = __expf(p.power);
    p.ag = __fmul_rn(b.y, p.G);
    p.alpha = fminf(ALPHA_MAX, p.ag);
}

// ---------------------------------------------------------------------------
// K6 blend forward
// ---------------------------------------------------------------------------
// Sums a per-thread count over the block into *evals (counting builds only).
__device__ __forceinline__ void add_evals(uint32_t ne, unsigned long long *evals) {
    const uint32_t w = __reduce_add_sync(0xffffffffu, ne);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(evals, (unsigned long long)w);
}

template <bool COUNT>
__global__ void __launch_bounds__(BLEND_THREADS)
k_blend_fwd(const Batch *__restrict__ bp, const uint2 *__restrict__ ranges,
            const uint32_t *__restrict__ pval, const Rec *__restrict__ rec,
            float *__restrict__ img, float *__restrict__ T_final, int32_t *__restrict__ last,
            unsigned long long *__restrict__ evals) {
    __shared__ float4 sa[BLEND_THREADS];
    __shared__ float4 sb[BLEND_THREADS];
    __shared__ float sc[BLEND_THREADS];
    const Batch &b = *bp;
    const uint32_t tile = blockIdx.x;
    const ViewDesc &vw = b.view[find_tile_view(b, tile)];
    const uint32_t lt = tile - vw.tile_off;
    const int tx = (int)(lt % (uint32_t)vw.tiles_x), ty = (int)(lt / (uint32_t)vw.tiles_x);
    const int px = tx * TILE + (threadIdx.x & (TILE - 1));
    const int py = ty * TILE + (threadIdx.x / TILE);
    const bool inside = px < vw.W && py < vw.H;
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);
    const float fpx = (float)px, fpy = (float)py;

    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    int lastc = 0;
    uint32_t ne = 0;
    bool done = !inside;
    for (int base = 0; base < n; base += BLEND_THREADS) {
        if (__syncthreads_count(done) == BLEND_THREADS) break;
        const int j = base + (int)threadIdx.x;
        if (j < n) {
            const Rec r = rec[pval[rg.x + j]];
            sa[threadIdx.x] = r.a;
            sb[threadIdx.x] = r.b;
            sc[threadIdx.x] = r.c.x;
        }
        __syncthreads();
        const int cnt = min(BLEND_THREADS, n - base);
        if (!done) {
            for (int k = 0; k < cnt; ++k) {
                const float4 a = sa[k], bb = sb[k];
                PairEval p;
                eval_pair(fpx, fpy, a, bb, p);
                if (COUNT) ++ne;
                if (p.power > 0.f) continue;
                if (p.alpha < ALPHA_MIN) continue;
                const float tt = __fmul_rn(T, __fsub_rn(1.f, p.alpha));
                if (tt < T_STOP) { done = true; break; }
                const float w = p.alpha * T;
                c0 += bb.z * w;
                c1 += bb.w * w;
                c2 += sc[k] * w;
                T = tt;
                lastc = base + k + 1;
            }
        }
    }
    if (COUNT) add_evals(ne, evals);
    if (inside) {
        const uint64_t HW = (uint64_t)vw.W * (uint64_t)vw.H;
        const uint64_t pix = (uint64_t)py * (uint64_t)vw.W + (uint64_t)px;
        float *im = img + 3 * vw.pix_off;
        im[pix] = c0 + T * vw.bg[0];
        im[HW + pix] = c1 + T * vw.bg[1];
        im[2 * HW + pix] = c2 + T * vw.bg[2];
        T_final[vw.pix_off + pix] = T;
        last[vw.pix_off + pix] = lastc;
    }
}

cudaError_t launch_blend_forward(const Batch *db, uint32_t n_tiles, const uint2 *ranges,
                                 const uint32_t *pval, const Rec *rec, float *img, float *T_final,
                                 int32_t *last, int n_views, unsigned long long *evals, cudaStream_t s) {
    (void)n_views;
    if (n_tiles == 0) return cudaSuccess;
    if (evals)
        k_blend_fwd<true><<<n_tiles, BLEND_THREADS, 0, s>>>(db, ranges, pval, rec, img, T_final, last, evals);
    else
        k_blend_fwd<false><<<n_tiles, BLEND_THREADS, 0, s>>>(db, ranges, pval, rec, img, T_final, last, nullptr);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K7 blend backward
// ---------------------------------------------------------------------------
// Sums 9 per-lane values over the warp and adds them to dg[k*M + e].
// Recursive halving: 4 + 2 + 1 shuffles leave each group of four lanes with
// one of the first eight sums, two more finish it; the ninth value takes a
// plain butterfly. 14 shuffles instead of 45, and eight lanes issue their
// atomics together.
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

template <bool COUNT>
__global__ void __launch_bounds__(BLEND_THREADS)
k_blend_bwd(const Batch *__restrict__ bp, const uint2 *__restrict__ ranges,
            const uint32_t *__restrict__ pval, const Rec *__restrict__ rec,
            const float *__restrict__ T_final, const int32_t *__restrict__ last,
            const float *__restrict__ d_img, float *__restrict__ dg, uint64_t M,
            unsigned long long *__restrict__ evals) {
    __shared__ float4 sa[BLEND_THREADS];
    __shared__ float4 sb[BLEND_THREADS];
    __shared__ float sc[BLEND_THREADS];
    __shared__ uint32_t sid[BLEND_THREADS];
    __shared__ int smax[BLEND_THREADS / 32];
    const Batch &b = *bp;
    const uint32_t tile = blockIdx.x;
    const ViewDesc &vw = b.view[find_tile_view(b, tile)];
    const uint32_t lt = tile - vw.tile_off;
    const int tx = (int)(lt % (uint32_t)vw.tiles_x), ty = (int)(lt / (uint32_t)vw.tiles_x);
    const int px = tx * TILE + (threadIdx.x & (TILE - 1));
    const int py = ty * TILE + (threadIdx.x / TILE);
    const bool inside = px < vw.W && py < vw.H;
    const uint2 rg = ranges[tile];
    const float fpx = (float)px, fpy = (float)py;

    const uint64_t HW = (uint64_t)vw.W * (uint64_t)vw.H;
    const uint64_t pix = (uint64_t)py * (uint64_t)vw.W + (uint64_t)px;
    int my_last = 0;
    float T = 1.f, Tf = 1.f, gp[3] = {0.f, 0.f, 0.f};
    if (inside) {
        my_last = last[vw.pix_off + pix];
        Tf = T_final[vw.pix_off + pix];
        T = Tf;
        const float *gi = d_img + 3 * vw.pix_off;
        gp[0] = gi[pix];
        gp[1] = gi[HW + pix];
        gp[2] = gi[2 * HW + pix];
    }
    const float bgdot = Tf * (gp[0] * vw.bg[0] + gp[1] * vw.bg[1] + gp[2] * vw.bg[2]);
    float S0 = 0.f, S1 = 0.f, S2 = 0.f;   // sum over later pairs of c alpha T
    uint32_t ne = 0;

    const int wmax = __reduce_max_sync(0xffffffffu, my_last);
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = wmax;
    __syncthreads();
    int maxlast = 0;
#pragma unroll
    for (int i = 0; i < BLEND_THREADS / 32; ++i) maxlast = max(maxlast, smax[i]);

    for (int end = maxlast; end > 0; end -= BLEND_THREADS) {
        const int start = max(0, end - BLEND_THREADS);
        const int cnt = end - start;
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const uint32_t e = pval[rg.x + start + threadIdx.x];
            const Rec r = rec[e];
            sa[threadIdx.x] = r.a;
            sb[threadIdx.x] = r.b;
            sc[threadIdx.x] = r.c.x;
            sid[threadIdx.x] = e;
        }
        __syncthreads();
        // warps whose pixels all end before this batch have nothing to add
        if (__all_sync(0xffffffffu, my_last <= start)) continue;
        for (int k = cnt - 1; k >= 0; --k) {
            const int pos = start + k;
            float v[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = 0.f;
            bool contrib = false;
            if (pos < my_last) {
                const float4 a = sa[k], bb = sb[k];
                PairEval p;
                eval_pair(fpx, fpy, a, bb, p);
                if (COUNT) ++ne;
                if (!(p.power > 0.f) && !(p.alpha < ALPHA_MIN)) {
                    contrib = true;
                    const float oma = __fsub_rn(1.f, p.alpha);
                    const float Ti = T / oma;
                    const float w = p.alpha * Ti;
                    const float cr = bb.z, cg = bb.w, cb = sc[k];
                    v[6] = w * gp[0];
                    v[7] = w * gp[1];
                    v[8] = w * gp[2];
                    const float dalpha = Ti * (cr * gp[0] + cg * gp[1] + cb * gp[2]) -
                                         (S0 * gp[0] + S1 * gp[1] + S2 * gp[2] + bgdot) / oma;
                    S0 += cr * w;
                    S1 += cg * w;
                    S2 += cb * w;
                    T = Ti;
                    if (!(p.ag > ALPHA_MAX)) {
                        const float dpower = dalpha * bb.y * p.G;
                        v[5] = dalpha * p.G;
                        v[2] = -0.5f * p.dx * p.dx * dpower;
                        v[3] = -p.dx * p.dy * dpower;
                        v[4] = -0.5f * p.dy * p.dy * dpower;
                        v[0] = dpower * (a.z * p.dx + a.w * p.dy);
                        v[1] = dpower * (bb.x * p.dy + a.w * p.dx);
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) warp_sum9_atomic(v, dg, M, sid[k]);
        }
    }
    if (COUNT) add_evals(ne, evals);
}

cudaError_t launch_blend_backward(const Batch *db, uint32_t n_tiles, const uint2 *ranges,
                                  const uint32_t *pval, const Rec *rec, const float *T_final,
                                  const int32_t *last, const float *d_img, float *dg, uint64_t M,
                                  int n_views, unsigned long long *evals, cudaStream_t s) {
    (void)n_views;
    if (n_tiles == 0) return cudaSuccess;
    if (evals)
        k_blend_bwd<true><<<n_tiles, BLEND_THREADS, 0, s>>>(db, ranges, pval, rec, T_final, last, d_img,
                                                             dg, M, evals);
    else
        k_blend_bwd<false><<<n_tiles, BLEND_THREADS, 0, s>>>(db, ranges, pval, rec, T_final, last, d_img,
                                                              dg, M, nullptr);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sgk
