// ADMM steps of the memory-constrained optimisation (Alg. 1, Sec. 3.3.2).
//
//  * penalty gradient of the gradient step: grad += delta (x - x~ + lambda)
//  * proximal step (Eq. 7-9): z = x + lambda; keep the kappa entries of z with
//    the largest score, x~ = z there and 0 elsewhere. Scores: the importance
//    I_i (App. A.2) or |z_i| for opacities, the dynamic range
//    D_i = |a_i| |1 - exp(-2 z_i)| (Eq. 10) for lobe sharpness.
//  * dual update: lambda += x - x~
//
// Selection is a stable LSD radix sort of order-preserving keys of the scores
// (largest first, equal scores by lower index), followed by one pass over the
// ranks that writes x~ and the new lambda.
#include "sg_internal.cuh"

#include <algorithm>

namespace sgk {

// Order-preserving key for a DESCENDING sort through an ascending radix sort.
// NaN scores sort last.
__device__ __forceinline__ uint32_t desc_key(float f) {
    if (isnan(f)) return 0xFFFFFFFFu;
    const uint32_t u = __float_as_uint(f);
    const uint32_t asc = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ~asc;
}

__global__ void __launch_bounds__(256) k_score_opacity(int64_t n, const float *__restrict__ x,
                                                       const float *__restrict__ lam,
                                                       const float *__restrict__ score,
                                                       uint32_t *__restrict__ keys,
                                                       uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float z = __fadd_rn(x[i], lam[i]);
    keys[i] = desc_key(score ? score[i] : fabsf(z));
    vals[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(256) k_score_sharpness(int64_t L, const float *__restrict__ s,
                                                         const float *__restrict__ lam,
                                                         const float *__restrict__ amp,
                                                         uint32_t *__restrict__ keys,
                                                         uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const float z = __fadd_rn(s[i], lam[i]);
    const float a0 = amp[i], a1 = amp[L + i], a2 = amp[2 * L + i];
    const float na = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
    const float D = na * fabsf(1.0f - expf(-2.0f * z));
    keys[i] = desc_key(D);
    vals[i] = (uint32_t)i;
}

// rank r of the sorted order: keep iff r < kappa
__global__ void __launch_bounds__(256) k_prox_dual(int64_t n, int64_t kappa, const uint32_t *__restrict__ order,
                                                   const float *__restrict__ x, float *__restrict__ lam,
                                                   float *__restrict__ x_tilde) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t i = order[r];
    if (i >= n) return;   // a stale word left by a sort whose bounded wait gave up
    const float xi = x[i], li = lam[i];
    const float z = __fadd_rn(xi, li);
    const float xt = r < kappa ? z : 0.0f;
    x_tilde[i] = xt;
    lam[i] = __fadd_rn(li, __fsub_rn(xi, xt));
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

__global__ void k_set_count(uint64_t *count, uint64_t n) { *count = n; }

// Workspace: keys/values ping-pong (4 x n), radix histograms, scan partials,
// and the item count.
struct AdmmLayout {
    size_t count, k0, v0, k1, v1, hist, sums, total;
};

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

static AdmmLayout admm_layout(int64_t n) {
    AdmmLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += al256(b); return r; };
    L.count = take(8);
    L.k0 = take(4 * (size_t)n);
    L.v0 = take(4 * (size_t)n);
    L.k1 = take(4 * (size_t)n);
    L.v1 = take(4 * (size_t)n);
    const uint64_t hb = div_up((uint64_t)n, RS_TILE);
    L.hist = take((size_t)4 * RS_RADIX * hb * 4);   // look-back flags of the 4 passes
    L.sums = take(std::max<size_t>((div_up((uint64_t)n, SCAN_TILE) + div_up((uint64_t)RS_RADIX * hb, SCAN_TILE) + 1) * 8,
                                   SORT_AUX_BYTES));
    L.total = o;
    return L;
}

size_t admm_workspace_bytes(int64_t n) { return admm_layout(n < 0 ? 0 : n).total; }

// kind 0: opacity (score = importance or |z|), kind 1: sharpness (score = D)
cudaError_t launch_admm_step(int kind, int64_t n, const float *x, const float *score, const float *amp,
                             int64_t kappa, float *lam, float *x_tilde, void *ws, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const AdmmLayout L = admm_layout(n);
    char *w = static_cast<char *>(ws);
    uint64_t *count = reinterpret_cast<uint64_t *>(w + L.count);
    uint32_t *k0 = reinterpret_cast<uint32_t *>(w + L.k0), *v0 = reinterpret_cast<uint32_t *>(w + L.v0);
    uint32_t *k1 = reinterpret_cast<uint32_t *>(w + L.k1), *v1 = reinterpret_cast<uint32_t *>(w + L.v1);
    k_set_count<<<1, 1, 0, s>>>(count, (uint64_t)n);
    count_launches(1);
    cudaError_t e = cudaSuccess;
    const unsigned grid = (unsigned)div_up((uint64_t)n, 256);
    if (kind == 0)
        k_score_opacity<<<grid, 256, 0, s>>>(n, x, lam, score, k0, v0);
    else
        k_score_sharpness<<<grid, 256, 0, s>>>(n, x, lam, amp, k0, v0);
    count_launches(1);
    e = launch_radix_sort(k0, v0, k1, v1, count, (uint64_t)n, 32, reinterpret_cast<uint32_t *>(w + L.hist),
                          reinterpret_cast<uint64_t *>(w + L.sums), s);
    if (e != cudaSuccess) return e;
    // 4 passes: the order is back in v0
    k_prox_dual<<<grid, 256, 0, s>>>(n, kappa, v0, x, lam, x_tilde);
    count_launches(1);
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
