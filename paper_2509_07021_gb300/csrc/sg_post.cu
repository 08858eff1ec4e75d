// Post-processing after the constrained optimisation (Sec. 3.3.3):
//   1. Gaussians whose opacity m_g o falls below tau_o are removed;
//   2. lobes of the remaining Gaussians whose sharpness falls below tau_s are
//      removed, and each removed lobe's mean over the sphere,
//      m_l a (1 - e^{-2s}) / (2s) (Eq. 12; limit m_l a at s = 0), is added
//      to the diffuse colour c0 (Eq. 13);
//   3. the kept Gaussians and lobes are compacted in their original order.
// The keep decisions are binary32 comparisons (m_g o is one rounded product).
#include "sg_internal.cuh"

namespace sgk {

__device__ __forceinline__ bool keep_gauss(const sg_scene &sc, int64_t g, float tau_o) {
    const float op = __fmul_rn(sc.gmask[g], static_cast<const float *>(sc.opac)[g]);
    return op >= tau_o;
}

__device__ __forceinline__ void lobe_range(const sg_scene &sc, int64_t g, int &lo, int &hi) {
    hi = min(sc.lobe_off[g + 1], (int)sc.n_lobes);
    lo = max(0, min(sc.lobe_off[g], hi));
}

__global__ void __launch_bounds__(256) k_post_count(const sg_scene sc, float tau_o, float tau_s,
                                                    uint32_t *__restrict__ gflag, uint32_t *__restrict__ lcnt) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sc.n) return;
    const bool kg = keep_gauss(sc, g, tau_o);
    uint32_t c = 0;
    if (kg) {
        int lo, hi;
        lobe_range(sc, g, lo, hi);
        const float *sh = static_cast<const float *>(sc.sharp);
        for (int k = lo; k < hi; ++k) c += sh[k] >= tau_s ? 1u : 0u;
    }
    gflag[g] = kg ? 1u : 0u;
    lcnt[g] = c;
}

// mean of a e^{s (mu.v - 1)} over the sphere divided by a: (1 - e^{-2s}) / (2s)
__device__ __forceinline__ float lobe_mean_factor(float s) {
    if (fabsf(s) < 1e-6f) return 1.0f - s;   // series 1 - s + O(s^2)
    return -expm1f(-2.0f * s) / (2.0f * s);
}

struct PostOut {
    float *means, *scales, *quats, *opac, *gmask, *c0, *axis, *sharp, *amp, *lmask;
    int32_t *lobe_off;
    int64_t n_out, l_out;
};

__global__ void __launch_bounds__(256) k_post_apply(const sg_scene sc, float tau_o, float tau_s,
                                                    const uint32_t *__restrict__ gflag,
                                                    const uint32_t *__restrict__ gidx,
                                                    const uint32_t *__restrict__ loff, PostOut o) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0) o.lobe_off[o.n_out] = (int32_t)o.l_out;
    if (g >= sc.n || !gflag[g]) return;
    const int64_t n = sc.n, L = sc.n_lobes, N2 = o.n_out, L2 = o.l_out;
    const int64_t i = gidx[g];
    const float *mean = static_cast<const float *>(sc.means), *scl = static_cast<const float *>(sc.scales);
    const float *q = static_cast<const float *>(sc.quats), *op = static_cast<const float *>(sc.opac);
    for (int d = 0; d < 3; ++d) {
        o.means[d * N2 + i] = mean[d * n + g];
        o.scales[d * N2 + i] = scl[d * n + g];
    }
    for (int d = 0; d < 4; ++d) o.quats[d * N2 + i] = q[d * n + g];
    o.opac[i] = op[g];
    o.gmask[i] = sc.gmask[g];
    float c[3] = {sc.c0[g], sc.c0[n + g], sc.c0[2 * n + g]};
    int lo, hi;
    lobe_range(sc, g, lo, hi);
    const float *ax = static_cast<const float *>(sc.axis), *sh = static_cast<const float *>(sc.sharp);
    const float *am = static_cast<const float *>(sc.amp);
    int64_t j = loff[g];
    o.lobe_off[i] = (int32_t)j;
    for (int k = lo; k < hi; ++k) {
        const float s = sh[k];
        if (s >= tau_s) {
            for (int d = 0; d < 3; ++d) {
                o.axis[d * L2 + j] = ax[d * L + k];
                o.amp[d * L2 + j] = am[d * L + k];
            }
            o.sharp[j] = s;
            o.lmask[j] = sc.lmask[k];
            ++j;
        } else {
            const float f = sc.lmask[k] * lobe_mean_factor(s);
            for (int d = 0; d < 3; ++d) c[d] = fmaf(am[d * L + k], f, c[d]);
        }
    }
    for (int d = 0; d < 3; ++d) o.c0[d * N2 + i] = c[d];
}

struct PostLayout {
    size_t gflag, lcnt, gidx, loff, sums, totals, total;
};

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

static PostLayout post_layout(int64_t n) {
    PostLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += al256(b); return r; };
    L.gflag = take(4 * (size_t)n);
    L.lcnt = take(4 * (size_t)n);
    L.gidx = take(4 * (size_t)n);
    L.loff = take(4 * (size_t)n);
    L.sums = take((div_up((uint64_t)n, SCAN_TILE) + 1) * 8);
    L.totals = take(2 * 8);
    L.total = o;
    return L;
}

size_t post_workspace_bytes(int64_t n) { return post_layout(n < 0 ? 0 : n).total; }

cudaError_t launch_post_plan(const sg_scene &sc, float tau_o, float tau_s, void *ws, uint64_t *totals_host,
                             cudaStream_t s) {
    const PostLayout L = post_layout(sc.n);
    char *w = static_cast<char *>(ws);
    uint32_t *gflag = reinterpret_cast<uint32_t *>(w + L.gflag), *lcnt = reinterpret_cast<uint32_t *>(w + L.lcnt);
    uint64_t *totals = reinterpret_cast<uint64_t *>(w + L.totals);
    uint64_t *sums = reinterpret_cast<uint64_t *>(w + L.sums);
    cudaError_t e = cudaMemsetAsync(totals, 0, 16, s);
    if (e != cudaSuccess) return e;
    if (sc.n > 0) {
        k_post_count<<<(unsigned)div_up((uint64_t)sc.n, 256), 256, 0, s>>>(sc, tau_o, tau_s, gflag, lcnt);
        count_launches(1);
        e = launch_scan(gflag, nullptr, reinterpret_cast<uint32_t *>(w + L.gidx), (uint64_t)sc.n, sums, totals, s);
        if (e != cudaSuccess) return e;
        e = launch_scan(lcnt, nullptr, reinterpret_cast<uint32_t *>(w + L.loff), (uint64_t)sc.n, sums, totals + 1, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemcpyAsync(totals_host, totals, 16, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t launch_post_apply(const sg_scene &sc, float tau_o, float tau_s, const void *ws, const sg_scene &out,
                              int64_t n_out, int64_t l_out, cudaStream_t s) {
    const PostLayout L = post_layout(sc.n);
    const char *w = static_cast<const char *>(ws);
    PostOut o;
    o.means = (float *)out.means; o.scales = (float *)out.scales; o.quats = (float *)out.quats;
    o.opac = (float *)out.opac; o.gmask = (float *)out.gmask; o.c0 = (float *)out.c0;
    o.axis = (float *)out.axis; o.sharp = (float *)out.sharp; o.amp = (float *)out.amp;
    o.lmask = (float *)out.lmask; o.lobe_off = (int32_t *)out.lobe_off;
    o.n_out = n_out; o.l_out = l_out;
    const uint64_t threads = sc.n > 0 ? (uint64_t)sc.n : 1;
    k_post_apply<<<(unsigned)div_up(threads, 256), 256, 0, s>>>(
        sc, tau_o, tau_s, reinterpret_cast<const uint32_t *>(w + L.gflag), reinterpret_cast<const uint32_t *>(w + L.gidx),
        reinterpret_cast<const uint32_t *>(w + L.loff), o);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sgk
