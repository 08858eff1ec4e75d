// ADMM steps of the memory-constrained optimisation (Alg. 1, Sec. 3.3.2).
//
//  * penalty gradient of the gradient step: grad += delta (x - x~ + lambda)
//  * proximal step (Eq. 7-9): z = x + lambda; keep the kappa entries of z with
//    the largest score, x~ = z there and 0 elsewhere. Scores: the importance
//    I_i (App. A.2) or |z_i| for opacities, the dynamic range
//    D_i = |a_i| |1 - exp(-2 z_i)| (Eq. 10) for lobe sharpness.
//  * dual update: lambda += x - x~
//
// Selection is a radix select over order-preserving keys of the scores (the
// kappa largest, equal scores by lower index): four passes over the keys, most
// significant byte first, each histogramming the keys that match the threshold
// digits found so far and picking the next digit where the running count
// reaches kappa; then one pass that keeps every key below the threshold and the
// first of its ties in index order (a decoupled look-back over the blocks' tie
// counts), and writes x~ and the new lambda.
#include "sg_internal.cuh"

#include <algorithm>

namespace sgk {

// Order-preserving key for a DESCENDING order through ascending keys (smaller
// key = larger score). NaN scores come last.
__device__ __forceinline__ uint32_t desc_key(float f) {
    if (isnan(f)) return 0xFFFFFFFFu;
    const uint32_t u = __float_as_uint(f);
    const uint32_t asc = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ~asc;
}

// State of one selection (in the workspace).
struct SelState {
    int64_t kappa;
    int32_t mode;            // 0: select, 1: keep none (kappa <= 0), 2: keep all (kappa >= n)
    int32_t pad;
    uint64_t status;         // SG_ERR_TIMEOUT when the final pass gave up a bounded wait
    uint64_t block_ctr;      // logical blocks of the final pass
};

constexpr int SEL_ITEMS = 8;                     // consecutive entries per thread in the final pass
constexpr int SEL_TILE = 256 * SEL_ITEMS;

// Writes every key; the grid also zeroes the histograms and the look-back
// words and thread 0 sets up the selection state.
__device__ __forceinline__ void sel_setup(int64_t n, int64_t kappa, SelState *st, uint32_t *hist,
                                          uint64_t *flags, uint64_t nflags) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = t; j < 4 * RS_RADIX; j += nth) hist[j] = 0u;
    for (uint64_t j = t; j < nflags; j += nth) flags[j] = 0ull;
    if (t == 0) {
        st->kappa = kappa;
        st->mode = kappa <= 0 ? 1 : (kappa >= n ? 2 : 0);
        st->status = 0ull;
        st->block_ctr = 0ull;
    }
}

__global__ void __launch_bounds__(256) k_score_opacity(int64_t n, const float *__restrict__ x,
                                                       const float *__restrict__ lam,
                                                       const float *__restrict__ score,
                                                       uint32_t *__restrict__ keys, int64_t kappa, SelState *st,
                                                       uint32_t *hist, uint64_t *flags, uint64_t nflags) {
    chain_enter();
    sel_setup(n, kappa, st, hist, flags, nflags);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float z = __fadd_rn(x[i], lam[i]);
    keys[i] = desc_key(score ? score[i] : fabsf(z));
}

__global__ void __launch_bounds__(256) k_score_sharpness(int64_t L, const float *__restrict__ s,
                                                         const float *__restrict__ lam,
                                                         const float *__restrict__ amp,
                                                         uint32_t *__restrict__ keys, int64_t kappa, SelState *st,
                                                         uint32_t *hist, uint64_t *flags, uint64_t nflags) {
    chain_enter();
    sel_setup(L, kappa, st, hist, flags, nflags);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const float z = __fadd_rn(s[i], lam[i]);
    const float a0 = amp[i], a1 = amp[L + i], a2 = amp[2 * L + i];
    const float na = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
    const float D = na * fabsf(1.0f - expf(-2.0f * z));
    keys[i] = desc_key(D);
}

// The threshold digits of the passes done so far, from their histograms (every
// block of the later kernels redoes these picks; 256 threads, thread d: digit
// d). Pass q's digit is the one where the running count of the keys matching
// the earlier digits reaches the entries still to keep.
struct SelPrefix {
    uint32_t prefix, mask;
    int64_t remaining;
    int32_t mode;
};

__device__ __forceinline__ SelPrefix sel_resolve(const SelState *st, const uint32_t *__restrict__ hist,
                                                 int passes) {
    __shared__ uint64_t shs[33];
    __shared__ uint32_t s_digit;
    __shared__ uint64_t s_below;
    SelPrefix r{0u, 0u, st->kappa, st->mode};
    for (int q = 0; q < passes && r.mode == 0; ++q) {   // uniform
        const uint64_t c = hist[q * RS_RADIX + threadIdx.x];
        uint64_t tot;
        const uint64_t excl = block_exclusive<uint64_t>(c, tot, shs);
        if ((int64_t)excl < r.remaining && r.remaining <= (int64_t)(excl + c)) {
            s_digit = threadIdx.x;
            s_below = excl;
        }
        __syncthreads();
        if ((int64_t)tot < r.remaining) {   // fewer keys than asked (not expected): keep them all
            r.mode = 2;
        } else {
            const int shift = 24 - 8 * q;
            r.prefix |= s_digit << shift;
            r.mask |= 0xFFu << shift;
            r.remaining -= (int64_t)s_below;
        }
        __syncthreads();   // s_digit / s_below are rewritten by the next pass
    }
    return r;
}

// Histogram of pass p's digit over the keys that match the digits of passes
// 0 .. p - 1.
__global__ void __launch_bounds__(256) k_sel_hist(int64_t n, const uint32_t *__restrict__ keys,
                                                  const SelState *st, uint32_t *__restrict__ hist, int p) {
    chain_enter();
    __shared__ uint32_t h[RS_RADIX];
    const SelPrefix r = sel_resolve(st, hist, p);
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int shift = 24 - 8 * p;
    if (r.mode == 0) {   // uniform
        const uint32_t pre = r.prefix, msk = r.mask;
        const int64_t n4 = n / 4;
        const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
        const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
        for (int64_t j = t; j < n4; j += nth) {
            const uint4 k = k4[j];
            if ((k.x & msk) == pre) atomicAdd(&h[(k.x >> shift) & 255u], 1u);
            if ((k.y & msk) == pre) atomicAdd(&h[(k.y >> shift) & 255u], 1u);
            if ((k.z & msk) == pre) atomicAdd(&h[(k.z >> shift) & 255u], 1u);
            if ((k.w & msk) == pre) atomicAdd(&h[(k.w >> shift) & 255u], 1u);
        }
        for (int64_t j = 4 * n4 + t; j < n; j += nth) {
            const uint32_t k = keys[j];
            if ((k & msk) == pre) atomicAdd(&h[(k >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[p * RS_RADIX + threadIdx.x], h[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_penalty_grad(int64_t n, const float *__restrict__ x,
                                                      const float *__restrict__ x_tilde,
                                                      const float *__restrict__ lam, float delta,
                                                      float *__restrict__ grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float y = __fadd_rn(__fsub_rn(x[i], x_tilde[i]), lam[i]);
    grad[i] = __fadd_rn(grad[i], __fmul_rn(delta, y));
}

// Final pass: thread t of logical block b owns entries b * SEL_TILE + t * SEL_ITEMS
// + 0 .. SEL_ITEMS - 1 (consecutive, so block and thread prefixes of the tie
// counts follow the index order). Keeps the keys below the threshold and the
// first `remaining` keys equal to it; writes x~ = z (kept) or 0 and
// lambda += x - x~.
__global__ void __launch_bounds__(256) k_sel_final(int64_t n, const uint32_t *__restrict__ keys,
                                                   const float *__restrict__ x, float *__restrict__ lam,
                                                   float *__restrict__ x_tilde, SelState *st,
                                                   const uint32_t *__restrict__ hist,
                                                   uint64_t *__restrict__ flags, uint32_t spin_limit) {
    chain_enter();
    __shared__ uint32_t shs[33];
    __shared__ uint64_t s_blk, s_excl;
    if (threadIdx.x == 0) s_blk = atomicAdd(reinterpret_cast<unsigned long long *>(&st->block_ctr), 1ull);
    __syncthreads();
    const uint64_t blk = s_blk;
    const SelPrefix r = sel_resolve(st, hist, 4);
    const int32_t mode = r.mode;
    const uint32_t T = r.prefix;          // the threshold key (all four digits)
    const int64_t rem = r.remaining;      // its ties to keep
    const int64_t i0 = (int64_t)blk * SEL_TILE + (int64_t)threadIdx.x * SEL_ITEMS;
    uint32_t k[SEL_ITEMS];
    uint32_t ties = 0u;
#pragma unroll
    for (int it = 0; it < SEL_ITEMS; ++it) {
        k[it] = i0 + it < n ? keys[i0 + it] : 0xFFFFFFFFu;
        ties += (mode == 0 && i0 + it < n && k[it] == T) ? 1u : 0u;
    }
    uint32_t btot;
    uint32_t rank = block_exclusive<uint32_t>(ties, btot, shs);   // ties in earlier threads of the block
    if (mode == 0) {   // uniform: ties in earlier blocks
        if (threadIdx.x == 0) st_relaxed64(flags + blk, DL_AGG | ((uint64_t)btot & DL_VAL));
        if (threadIdx.x < 32) {
            const uint64_t excl = block_lookback64(flags, blk, btot, spin_limit, &st->status);
            if (threadIdx.x == 0) s_excl = excl;
        }
        __syncthreads();
    }
    const uint64_t before = mode == 0 ? s_excl : 0ull;
#pragma unroll
    for (int it = 0; it < SEL_ITEMS; ++it) {
        const int64_t i = i0 + it;
        if (i >= n) break;
        bool keep = mode == 2;
        if (mode == 0) {
            if (k[it] < T) {
                keep = true;
            } else if (k[it] == T) {
                keep = (int64_t)(before + rank) < rem;
                ++rank;
            }
        }
        const float xi = x[i], li = lam[i];
        const float z = __fadd_rn(xi, li);
        const float xt = keep ? z : 0.0f;
        x_tilde[i] = xt;
        lam[i] = __fadd_rn(li, __fsub_rn(xi, xt));
    }
}

// Workspace: the selection state, the keys, the 4 passes' histograms and the
// final pass's look-back words.
struct AdmmLayout {
    size_t state, keys, hist, flags, total;
    uint64_t nflags;
};

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

static AdmmLayout admm_layout(int64_t n) {
    AdmmLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += al256(b); return r; };
    L.state = take(sizeof(SelState));
    L.keys = take(4 * (size_t)n);
    L.hist = take((size_t)4 * RS_RADIX * 4);
    L.nflags = std::max<uint64_t>(div_up((uint64_t)n, SEL_TILE), 1);
    L.flags = take(8 * L.nflags);
    L.total = o;
    return L;
}

size_t admm_workspace_bytes(int64_t n) { return admm_layout(n < 0 ? 0 : n).total; }

// kind 0: opacity (score = importance or |z|), kind 1: sharpness (score = D)
cudaError_t launch_admm_step(int kind, int64_t n, const float *x, const float *score, const float *amp,
                             int64_t kappa, float *lam, float *x_tilde, void *ws, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if ((uint64_t)n > (uint64_t)UINT32_MAX) return cudaErrorInvalidValue;   // 32-bit histogram counts
    const AdmmLayout L = admm_layout(n);
    char *w = static_cast<char *>(ws);
    SelState *st = reinterpret_cast<SelState *>(w + L.state);
    uint32_t *keys = reinterpret_cast<uint32_t *>(w + L.keys);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + L.hist);
    uint64_t *flags = reinterpret_cast<uint64_t *>(w + L.flags);
    const dim3 grid((unsigned)div_up((uint64_t)n, 256));
    if (kind == 0)
        (void)launch_chain(k_score_opacity, grid, dim3(256), s, n, x, lam, score, keys, kappa, st, hist, flags,
                           L.nflags);
    else
        (void)launch_chain(k_score_sharpness, grid, dim3(256), s, n, x, lam, amp, keys, kappa, st, hist, flags,
                           L.nflags);
    const unsigned hgrid = (unsigned)std::min<uint64_t>(std::max<uint64_t>(div_up((uint64_t)n, 256 * 16), 1),
                                                        4 * 152);
    for (int p = 0; p < 4; ++p)
        (void)launch_chain(k_sel_hist, dim3(hgrid), dim3(256), s, n, (const uint32_t *)keys, (const SelState *)st,
                           hist, p);
    (void)launch_chain(k_sel_final, dim3((unsigned)L.nflags), dim3(256), s, n, (const uint32_t *)keys, x, lam,
                       x_tilde, st, (const uint32_t *)hist, flags, sort_wait_polls());
    count_launches(6);
    return cudaGetLastError();
}

cudaError_t launch_penalty_grad(int64_t n, const float *x, const float *x_tilde, const float *lam, float delta,
                                float *grad, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_penalty_grad<<<(unsigned)div_up((uint64_t)n, 256), 256, 0, s>>>(n, x, x_tilde, lam, delta, grad);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sgk
