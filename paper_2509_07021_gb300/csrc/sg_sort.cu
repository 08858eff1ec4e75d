// Binning: exclusive scan, stable LSD radix sort of u32 (key, value) pairs,
// duplicateWithKeys and per-tile ranges.
//
// The (tile, depth) ordering of the paper's tile-depth-Gaussian key table
// (Sec. 1, rendering VRAM; the 3DGS binning it inherits) is the order of an
// LSD radix sort of 64-bit keys tile << 32 | depth_bits, equal keys by
// Gaussian id. The depth digits of every pair of one Gaussian are equal, so
// the depth passes are run once per (view, Gaussian) entry, before the
// entries are duplicated into pairs, and only the tile digits are sorted per
// pair. Duplication walks the entries in depth order and every pass is
// stable, so the result is identical to the 64-bit sort.
#include "sg_internal.cuh"

namespace sgk {

__device__ __forceinline__ uint32_t lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
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

// ---------------------------------------------------------------------------
// exclusive scan: reduce -> spine -> downsweep
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t scan_load(const uint32_t *in, const uint32_t *idx, uint64_t i) {
    return idx ? in[idx[i]] : in[i];
}

__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t *__restrict__ in,
                                                     const uint32_t *__restrict__ idx, uint64_t n,
                                                     uint64_t *__restrict__ sums) {
    __shared__ uint64_t sh[33];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint64_t acc = 0;
#pragma unroll 4
    for (int i = 0; i < SCAN_TILE / 256; ++i) {
        const uint64_t j = base + (uint64_t)i * 256 + threadIdx.x;
        if (j < n) acc += scan_load(in, idx, j);
    }
    uint64_t tot;
    block_exclusive<uint64_t>(acc, tot, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_spine(uint64_t *__restrict__ sums, uint64_t nb,
                                                     uint64_t *__restrict__ total) {
    __shared__ uint64_t sh[33];
    const uint64_t per = div_up(nb, 1024);
    const uint64_t lo = threadIdx.x * per, hi = min(nb, lo + per);
    uint64_t acc = 0;
    for (uint64_t i = lo; i < hi; ++i) acc += sums[i];
    uint64_t tot;
    uint64_t run = block_exclusive<uint64_t>(acc, tot, sh);
    for (uint64_t i = lo; i < hi; ++i) {
        const uint64_t v = sums[i];
        sums[i] = run;
        run += v;
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void __launch_bounds__(256) k_scan_down(const uint32_t *__restrict__ in,
                                                   const uint32_t *__restrict__ idx, uint64_t n,
                                                   const uint64_t *__restrict__ sums,
                                                   uint32_t *__restrict__ out) {
    // each thread owns 16 consecutive items, staged through shared memory
    __shared__ uint32_t buf[SCAN_TILE + SCAN_TILE / 32];
    __shared__ uint64_t sh[33];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
#pragma unroll 4
    for (int i = 0; i < SCAN_TILE / 256; ++i) {
        const int p = i * 256 + threadIdx.x;
        const uint64_t j = base + p;
        buf[p + (p >> 5)] = j < n ? scan_load(in, idx, j) : 0u;
    }
    __syncthreads();
    uint32_t loc[16];
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int p = threadIdx.x * 16 + k;
        loc[k] = buf[p + (p >> 5)];
        acc += loc[k];
    }
    uint64_t tot;
    uint64_t run = block_exclusive<uint64_t>(acc, tot, sh) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int p = threadIdx.x * 16 + k;
        buf[p + (p >> 5)] = (uint32_t)run;
        run += loc[k];
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < SCAN_TILE / 256; ++i) {
        const int p = i * 256 + threadIdx.x;
        const uint64_t j = base + p;
        if (j < n) out[j] = buf[p + (p >> 5)];
    }
}

cudaError_t launch_scan(const uint32_t *in, const uint32_t *gather_idx, uint32_t *out, uint64_t n,
                        uint64_t *block_sums, uint64_t *total, cudaStream_t s) {
    const uint64_t nb = div_up(n, SCAN_TILE);
    if (nb == 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
        return cudaSuccess;
    }
    k_scan_reduce<<<(unsigned)nb, 256, 0, s>>>(in, gather_idx, n, block_sums);
    count_launches(1);
    k_scan_spine<<<1, 1024, 0, s>>>(block_sums, nb, total);
    count_launches(1);
    k_scan_down<<<(unsigned)nb, 256, 0, s>>>(in, gather_idx, n, block_sums, out);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits, 4096 keys per block
// ---------------------------------------------------------------------------
// Item counts come from the device (*n_dev) and are clamped to the capacity
// the launch was sized for (max_n), so an overflowing count can never index
// past the buffers.
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint32_t *__restrict__ keys,
                                                           const uint64_t *__restrict__ n_dev,
                                                           uint64_t max_n, int shift, uint32_t mask,
                                                           uint32_t *__restrict__ hist,
                                                           uint32_t nblocks) {
    __shared__ uint32_t h[RS_RADIX];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const uint64_t n = min(*n_dev, max_n);
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    if (base < n) {
#pragma unroll 4
        for (int i = 0; i < RS_ITEMS; ++i) {
            const uint64_t j = base + (uint64_t)i * RS_THREADS + threadIdx.x;
            if (j < n) atomicAdd(&h[(keys[j] >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint64_t *__restrict__ n_dev, uint64_t max_n, int shift,
    uint32_t mask, const uint32_t *__restrict__ hist_scan, uint32_t nblocks) {
    constexpr int NW = RS_THREADS / 32;
    constexpr int PER_WARP = RS_TILE / NW;   // 512 consecutive keys per warp
    __shared__ uint32_t cnt[NW][RS_RADIX];
    __shared__ uint32_t dstart[RS_RADIX];
    __shared__ uint32_t gstart[RS_RADIX];
    __shared__ uint32_t sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    __shared__ uint32_t shs[33];

    const uint64_t n = min(*n_dev, max_n);
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    if (base >= n) return;   // uniform across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NW; ++i) cnt[i][threadIdx.x] = 0u;
    __syncthreads();

    uint32_t k[RS_ITEMS], v[RS_ITEMS], r[RS_ITEMS];
    const uint64_t wbase = base + (uint64_t)warp * PER_WARP;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t j = wbase + (uint64_t)i * 32 + lane;
        const bool ok = j < n;
        k[i] = ok ? kin[j] : 0u;
        v[i] = ok ? vin[j] : 0u;
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t j = wbase + (uint64_t)i * 32 + lane;
        const bool ok = j < n;
        const uint32_t d = ok ? ((k[i] >> shift) & mask) : 0x100u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0u;
        if (ok) before = cnt[warp][d];
        r[i] = before + __popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0u) cnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive offsets over warps, then over digits
    uint32_t run = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t c = cnt[w][threadIdx.x];
        cnt[w][threadIdx.x] = run;
        run += c;
    }
    uint32_t tot;
    const uint32_t ds = block_exclusive<uint32_t>(run, tot, shs);
    dstart[threadIdx.x] = ds;
    gstart[threadIdx.x] = hist_scan[(uint64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t j = wbase + (uint64_t)i * 32 + lane;
        if (j < n) {
            const uint32_t d = (k[i] >> shift) & mask;
            const uint32_t pos = dstart[d] + cnt[warp][d] + r[i];
            sk[pos] = k[i];
            sv[pos] = v[i];
        }
    }
    __syncthreads();
    const int items = (n - base) < (uint64_t)RS_TILE ? (int)(n - base) : RS_TILE;
    for (int p = threadIdx.x; p < items; p += RS_THREADS) {
        const uint32_t key = sk[p];
        const uint32_t d = (key >> shift) & mask;
        const uint32_t o = gstart[d] + (uint32_t)p - dstart[d];
        kout[o] = key;
        vout[o] = sv[p];
    }
}

int radix_passes(int bits) { return bits <= 0 ? 0 : (bits + 7) / 8; }

cudaError_t launch_radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                              const uint64_t *n_dev, uint64_t max_n, int bits, uint32_t *hist,
                              uint64_t *scan_sums, cudaStream_t s) {
    const uint32_t nblocks = (uint32_t)div_up(max_n, RS_TILE);
    if (nblocks == 0) return cudaSuccess;
    const int passes = radix_passes(bits);
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        const int nb = min(8, bits - shift);
        const uint32_t mask = (1u << nb) - 1u;
        k_radix_hist<<<nblocks, RS_THREADS, 0, s>>>(ki, n_dev, max_n, shift, mask, hist, nblocks);
        count_launches(1);
        cudaError_t e = launch_scan(hist, nullptr, hist, (uint64_t)RS_RADIX * nblocks, scan_sums,
                                    nullptr, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<nblocks, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n_dev, max_n, shift, mask, hist,
                                                       nblocks);
        count_launches(1);
        uint32_t *t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// duplicateWithKeys: entries in depth order -> (tile, entry) pairs
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_entry_view(const Batch &b, uint64_t e) {
    int lo = 0, hi = b.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.view[mid].ent_off <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_duplicate(const Batch *__restrict__ bp, uint64_t M,
                                                   const uint32_t *__restrict__ sorted_ent,
                                                   const uint32_t *__restrict__ tiles_touched,
                                                   const uint2 *__restrict__ rect,
                                                   const uint32_t *__restrict__ offsets,
                                                   const uint64_t *__restrict__ counters, uint64_t cap,
                                                   uint32_t *__restrict__ pkey,
                                                   uint32_t *__restrict__ pval) {
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    if (counters[CNT_PAIRS] > cap) return;   // capacity exceeded: the host reports it
    const uint32_t e = sorted_ent[j];
    const uint32_t tt = tiles_touched[e];
    if (tt == 0u) return;
    const Batch &b = *bp;
    const ViewDesc &vw = b.view[find_entry_view(b, e)];
    const uint2 rc = rect[e];
    const uint32_t x0 = rc.x & 0xFFFFu, x1 = rc.x >> 16, y0 = rc.y & 0xFFFFu, y1 = rc.y >> 16;
    uint64_t o = offsets[j];
    for (uint32_t ty = y0; ty < y1; ++ty) {
        const uint32_t row = vw.tile_off + ty * (uint32_t)vw.tiles_x;
        for (uint32_t tx = x0; tx < x1; ++tx) {
            pkey[o] = row + tx;
            pval[o] = e;
            ++o;
        }
    }
}

cudaError_t launch_duplicate(const Batch *db, uint64_t M, const uint32_t *sorted_ent,
                             const uint32_t *tiles_touched, const uint2 *rect, const uint32_t *offsets,
                             const uint64_t *counters, uint64_t cap, uint32_t *pkey, uint32_t *pval,
                             int n_views, cudaStream_t s) {
    (void)n_views;
    if (M == 0) return cudaSuccess;
    k_duplicate<<<(unsigned)div_up(M, 256), 256, 0, s>>>(db, M, sorted_ent, tiles_touched, rect, offsets,
                                                         counters, cap, pkey, pval);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// tile ranges from the sorted tile keys
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ranges(const uint32_t *__restrict__ pkey,
                                                const uint64_t *__restrict__ counters, uint64_t cap,
                                                uint2 *__restrict__ ranges) {
    const uint64_t K = counters[CNT_PAIRS];
    if (K > cap) return;
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const uint32_t t = pkey[i];
    if (i == 0 || pkey[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == K - 1 || pkey[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

cudaError_t launch_ranges(const uint32_t *pkey, const uint64_t *counters, uint64_t cap, uint2 *ranges,
                          uint64_t n_tiles, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, n_tiles * sizeof(uint2), s);
    if (e != cudaSuccess) return e;
    if (cap == 0) return cudaSuccess;
    k_ranges<<<(unsigned)div_up(cap, 256), 256, 0, s>>>(pkey, counters, cap, ranges);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// work order of the persistent blend: tiles by descending list length
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tile_keys(const uint2 *__restrict__ ranges, uint32_t n_tiles,
                                                   uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const uint2 r = ranges[t];
    const uint32_t len = r.y - r.x;
    keys[t] = 0xFFFFu - min(len >> 2, 0xFFFFu);   // 16-bit, longest first
    vals[t] = t;
}

cudaError_t launch_tile_order(const uint2 *ranges, uint32_t n_tiles, const uint64_t *n_tiles_dev,
                              uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t *hist,
                              uint64_t *scan_sums, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    k_tile_keys<<<(unsigned)div_up(n_tiles, 256), 256, 0, s>>>(ranges, n_tiles, k0, v0);
    count_launches(1);
    // two stable 8-bit passes: the order ends in (k0, v0)
    return launch_radix_sort(k0, v0, k1, v1, n_tiles_dev, n_tiles, 16, hist, scan_sums, s);
}

__global__ void k_capacity_status(uint64_t *counters, uint64_t cap) {
    if (counters[CNT_PAIRS] > cap) counters[CNT_STATUS] = (uint64_t)SG_ERR_CAPACITY;
}

cudaError_t launch_capacity_status(uint64_t *counters, uint64_t cap, cudaStream_t s) {
    k_capacity_status<<<1, 1, 0, s>>>(counters, cap);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sgk
