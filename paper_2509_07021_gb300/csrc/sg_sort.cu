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

#include <atomic>

namespace sgk {

__host__ __device__ __forceinline__ int radix_passes_dev(int bits) { return bits <= 0 ? 0 : (bits + 7) / 8; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
}


// ---------------------------------------------------------------------------
// exclusive scan: reduce -> spine -> downsweep
// ---------------------------------------------------------------------------
// With idx, in[idx[i]]; an index outside in's n_in items reads 0. (Indices
// come from a sort whose bounded wait may have given up, leaving stale words
// in its output: the gather stays inside the array whatever they hold.)
__device__ __forceinline__ uint32_t scan_load(const uint32_t *in, const uint32_t *idx, uint64_t i, uint64_t n_in) {
    if (!idx) return in[i];
    const uint32_t e = idx[i];
    return e < n_in ? in[e] : 0u;
}

__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t *__restrict__ in,
                                                     const uint32_t *__restrict__ idx, uint64_t n_in, uint64_t n,
                                                     const uint64_t *__restrict__ n_dev,
                                                     uint64_t *__restrict__ sums) {
    __shared__ uint64_t sh[33];
    if (n_dev) n = min(n, *n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint64_t acc = 0;
#pragma unroll 4
    for (int i = 0; i < SCAN_TILE / 256; ++i) {
        const uint64_t j = base + (uint64_t)i * 256 + threadIdx.x;
        if (j < n) acc += scan_load(in, idx, j, n_in);
    }
    uint64_t tot;
    block_exclusive<uint64_t>(acc, tot, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// mirror (nullable; host memory mapped into the device): receives the total
// and *status_src, so the host can read both without a copy in the stream.
__global__ void __launch_bounds__(1024) k_scan_spine(uint64_t *__restrict__ sums, uint64_t nb,
                                                     uint64_t *__restrict__ total, uint64_t *mirror,
                                                     const uint64_t *status_src) {
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
    if (threadIdx.x == 0 && mirror) {
        mirror[0] = tot;
        mirror[1] = status_src ? *status_src : 0;
    }
}

__global__ void __launch_bounds__(256) k_scan_down(const uint32_t *__restrict__ in,
                                                   const uint32_t *__restrict__ idx, uint64_t n_in, uint64_t n,
                                                   const uint64_t *__restrict__ n_dev,
                                                   const uint64_t *__restrict__ sums,
                                                   uint32_t *__restrict__ out) {
    if (n_dev) n = min(n, *n_dev);
    // each thread owns 16 consecutive items, staged through shared memory
    __shared__ uint32_t buf[SCAN_TILE + SCAN_TILE / 32];
    __shared__ uint64_t sh[33];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
#pragma unroll 4
    for (int i = 0; i < SCAN_TILE / 256; ++i) {
        const int p = i * 256 + threadIdx.x;
        const uint64_t j = base + p;
        buf[p + (p >> 5)] = j < n ? scan_load(in, idx, j, n_in) : 0u;
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
                        uint64_t *block_sums, uint64_t *total, cudaStream_t s, const uint64_t *n_dev,
                        uint64_t *mirror, const uint64_t *status_src) {
    const uint64_t nb = div_up(n, SCAN_TILE);
    if (nb == 0) {
        if (mirror) {   // the spine alone writes the zero total
            k_scan_spine<<<1, 1024, 0, s>>>(block_sums, 0, total, mirror, status_src);
            count_launches(1);
            return cudaGetLastError();
        }
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
        return cudaSuccess;
    }
    k_scan_reduce<<<(unsigned)nb, 256, 0, s>>>(in, gather_idx, n, n, n_dev, block_sums);
    count_launches(1);
    k_scan_spine<<<1, 1024, 0, s>>>(block_sums, nb, total, mirror, status_src);
    count_launches(1);
    k_scan_down<<<(unsigned)nb, 256, 0, s>>>(in, gather_idx, n, n, n_dev, block_sums, out);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits, RS_TILE keys per block, one sweep per pass
// ---------------------------------------------------------------------------
// One kernel histograms every digit position at once (and clears the look-back
// flags of every pass). Each pass is then a single kernel: blocks take key
// tiles in order from an atomic counter, rank their keys stably (warp
// match_any + per-warp digit counters), scan the pass's digit histogram for
// the digit bases, publish their digit counts, and get their offsets among
// the tiles before them by looking back (decoupled look-back). A look-back
// spin is bounded: past the bound the block records SG_ERR_TIMEOUT in the
// status word and carries on with a smaller offset (wrong order, still inside
// the array) instead of waiting forever.

// packed look-back word: 2 status bits, 30 count bits
constexpr uint32_t LB_AGG = 1u << 30, LB_INC = 2u << 30, LB_VAL = (1u << 30) - 1u;
static_assert(LB_VAL == SORT_MAX_KEYS, "look-back count width");
constexpr uint32_t LB_SPIN_LIMIT = 1u << 20;   // default bound on unanswered look-back polls
constexpr int LB_WINDOW = 16;

// Process-wide bound on the polls a block makes of an unpublished predecessor
// before it gives up (sg_tuning.sort_wait_polls; 0 = LB_SPIN_LIMIT).
static std::atomic<uint32_t> g_spin_limit{0};
void set_sort_wait_polls(uint32_t polls) { g_spin_limit.store(polls); }
uint32_t sort_wait_polls() {
    const uint32_t v = g_spin_limit.load();
    return v ? v : LB_SPIN_LIMIT;
}

struct SortAux {
    uint32_t hist[4][RS_RADIX];   // global digit counts per pass
    uint32_t tile_ctr[4];         // tile counter per pass
    uint32_t status;              // 0 or SG_ERR_TIMEOUT
    uint32_t pad;
    uint64_t kept;                // keys other than SORT_DROP_KEY (drop mode)
};
static_assert(sizeof(SortAux) <= SORT_AUX_BYTES, "sort aux region");

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

// Per-warp private shared histograms keep the shared-memory atomics of keys
// with few distinct digits (the high tile bits) from serialising.
__global__ void __launch_bounds__(RS_THREADS) k_os_hist(const uint32_t *__restrict__ keys,
                                                        const uint64_t *__restrict__ n_dev, uint64_t max_n,
                                                        int bits, bool drop, SortAux *aux,
                                                        uint32_t *__restrict__ flags, uint64_t flag_words) {
    chain_enter();
    constexpr int NW = RS_THREADS / 32;
    __shared__ uint32_t h[NW][4][RS_RADIX];
    const int passes = radix_passes_dev(bits);
    // the look-back flags of every pass start at zero (the passes run after this kernel)
    for (uint64_t i = (uint64_t)blockIdx.x * RS_THREADS + threadIdx.x; i < flag_words;
         i += (uint64_t)gridDim.x * RS_THREADS)
        flags[i] = 0u;
    const int warp = threadIdx.x >> 5;
    for (int w = 0; w < NW; ++w)
        for (int p = 0; p < 4; ++p) h[w][p][threadIdx.x] = 0u;
    __syncthreads();
    const uint64_t n = min(*n_dev, max_n);
    const uint64_t stride = (uint64_t)gridDim.x * RS_THREADS;
    uint32_t kept = 0u;
    auto count = [&](uint32_t k) {
        if (drop && k == SORT_DROP_KEY) return;
        ++kept;
        for (int p = 0; p < passes; ++p) {
            const int nb = min(8, bits - 8 * p);
            atomicAdd(&h[warp][p][(k >> (8 * p)) & ((1u << nb) - 1u)], 1u);
        }
    };
    // four keys per 16-byte load (the key arrays are 256-byte aligned), then the tail
    const uint64_t n4 = n / 4;
    const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
    for (uint64_t j = (uint64_t)blockIdx.x * RS_THREADS + threadIdx.x; j < n4; j += stride) {
        const uint4 q = k4[j];
        count(q.x);
        count(q.y);
        count(q.z);
        count(q.w);
    }
    for (uint64_t j = 4 * n4 + (uint64_t)blockIdx.x * RS_THREADS + threadIdx.x; j < n; j += stride)
        count(keys[j]);
    if (drop) {
        const uint32_t wk = __reduce_add_sync(0xffffffffu, kept);
        if ((threadIdx.x & 31) == 0 && wk)
            atomicAdd(reinterpret_cast<unsigned long long *>(&aux->kept), (unsigned long long)wk);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        uint32_t c = 0u;
        for (int w = 0; w < NW; ++w) c += h[w][p][threadIdx.x];
        if (c) atomicAdd(&aux->hist[p][threadIdx.x], c);
    }
}

// three resident blocks per SM (80 registers a thread)
__global__ void __launch_bounds__(RS_THREADS, 3) k_os_pass(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint64_t *__restrict__ n_dev, uint64_t max_n, int pass, int shift,
    uint32_t mask, bool drop, uint32_t *__restrict__ flags, SortAux *aux, uint2 *__restrict__ ranges,
    uint64_t n_ranges, uint32_t spin_limit, const uint64_t *__restrict__ skip_status) {
    chain_enter();
    constexpr int NW = RS_THREADS / 32;
    constexpr int PER_WARP = RS_TILE / NW;   // 512 consecutive keys per warp
    __shared__ uint32_t cnt[NW][RS_RADIX];
    __shared__ uint32_t dstart[RS_RADIX];
    __shared__ uint32_t gstart[RS_RADIX];
    __shared__ uint32_t sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    __shared__ uint32_t shs[33];
    __shared__ uint32_t s_tile;

    // an earlier bounded wait gave up (stale words) or the pairs overflowed (uniform)
    if (skip_status && *skip_status != 0ull) return;
    if (threadIdx.x == 0) s_tile = atomicAdd(&aux->tile_ctr[pass], 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    const uint64_t n = min(*n_dev, max_n);
    const uint64_t base = (uint64_t)t * RS_TILE;
    if (base >= n) return;   // uniform across the block; later tiles exit too
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
    // Warp-local stable ranks. Per item, the lowest lane of each group of equal
    // digits adds the group's size to the warp's counter; shared-memory atomics
    // of one warp take effect in issue order, so the returned bases follow the
    // key order. All atomics are issued before any base is broadcast.
    const uint32_t lt = lanemask_lt();
    uint32_t meta[RS_ITEMS];   // leader lane | (rank inside the group << 5)
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t j = wbase + (uint64_t)i * 32 + lane;
        const bool ok = j < n && !(drop && k[i] == SORT_DROP_KEY);
        const uint32_t d = ok ? ((k[i] >> shift) & mask) : 0x100u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t below = peers & lt;
        r[i] = (ok && below == 0u) ? atomicAdd(&cnt[warp][d], (uint32_t)__popc(peers)) : 0u;
        meta[i] = (uint32_t)(__ffs(peers) - 1) | ((uint32_t)__popc(below) << 5);
    }
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i)
        r[i] = __shfl_sync(0xffffffffu, r[i], (int)(meta[i] & 31u)) + (meta[i] >> 5);
    __syncthreads();
    // per digit: exclusive offsets over warps, block total, block-local start
    uint32_t run = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t c = cnt[w][threadIdx.x];
        cnt[w][threadIdx.x] = run;
        run += c;
    }
    const uint32_t d = threadIdx.x;
    // publish this tile's count, then look back for the exclusive prefix
    uint32_t *my = flags + (uint64_t)t * RS_RADIX + d;
    st_relaxed(my, LB_AGG | run);
    // Look back LB_WINDOW predecessors per step (independent loads in flight):
    // add counts until the nearest tile that carries its inclusive prefix;
    // a tile not yet published stops the step and is re-read.
    uint32_t excl = 0u;
    uint32_t spins = 0;
    for (int64_t p = (int64_t)t - 1; p >= 0;) {
        uint32_t fv[LB_WINDOW];
#pragma unroll
        for (int i = 0; i < LB_WINDOW; ++i)
            fv[i] = (p - i >= 0) ? ld_relaxed(flags + (uint64_t)(p - i) * RS_RADIX + d) : LB_INC;
        int used = 0;
        bool found = false, stalled = false;
#pragma unroll
        for (int i = 0; i < LB_WINDOW; ++i) {
            if (found || stalled) continue;
            if ((fv[i] & ~LB_VAL) == 0u) { stalled = true; continue; }
            excl += fv[i] & LB_VAL;
            ++used;
            if (fv[i] & LB_INC) found = true;
        }
        if (found) break;
        p -= used;
        if (stalled) {
            if (++spins >= spin_limit) {
                atomicExch(&aux->status, (uint32_t)SG_ERR_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
    }
    st_relaxed(my, LB_INC | ((excl + run) & LB_VAL));
    uint32_t tot, all;
    const uint32_t ds = block_exclusive<uint32_t>(run, tot, shs);
    // global start of digit d in this pass: keys of smaller digits (all tiles) + earlier tiles
    const uint32_t dbase = block_exclusive<uint32_t>(aux->hist[pass][d], all, shs);
    dstart[d] = ds;
    gstart[d] = dbase + excl;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t j = wbase + (uint64_t)i * 32 + lane;
        if (j < n && !(drop && k[i] == SORT_DROP_KEY)) {
            const uint32_t dd = (k[i] >> shift) & mask;
            const uint32_t pos = dstart[dd] + cnt[warp][dd] + r[i];
            sk[pos] = k[i];
            sv[pos] = v[i];
        }
    }
    __syncthreads();
    const int items = (int)tot;   // the block's kept keys
    // Last pass with ranges: the block's keys are now in full key order (its
    // input is sorted by the lower digits, its local sort by this one is
    // stable), so each run of one key is contiguous in the output; its ends
    // bound that key's range. Skipped when the count exceeded the capacity.
    const bool want_ranges = ranges != nullptr && *n_dev <= max_n;
    for (int p = threadIdx.x; p < items; p += RS_THREADS) {
        const uint32_t key = sk[p];
        const uint32_t dd = (key >> shift) & mask;
        const uint32_t o = gstart[dd] + (uint32_t)p - dstart[dd];
        kout[o] = key;
        vout[o] = sv[p];
        if (want_ranges && key < n_ranges) {
            if (p == 0 || sk[p - 1] != key) atomicMin(&ranges[key].x, o);
            if (p == items - 1 || sk[p + 1] != key) atomicMax(&ranges[key].y, o + 1u);
        }
    }
}

int radix_passes(int bits) { return bits <= 0 ? 0 : (bits + 7) / 8; }

uint64_t sort_flag_words(uint64_t max_n, int bits) {
    return div_up(max_n, RS_TILE) * RS_RADIX * (uint64_t)radix_passes(bits);
}

// Buckets by list length on a log scale with 8 buckets per octave (exponent and
// the 3 bits below the leading one), longest bucket first; inside a bucket the
// order is whatever the atomics give (it only steers scheduling).
constexpr int TB_BUCKETS = 256;
__device__ __forceinline__ uint32_t len_bucket(const uint2 r) {
    const uint32_t len = (r.y - r.x) | 1u;
    const uint32_t e = 31u - (uint32_t)__clz(len);              // 0..31
    const uint32_t m = e >= 3u ? (len >> (e - 3u)) & 7u : (len << (3u - e)) & 7u;
    return e * 8u + m;                                           // 0..255
}

// Status and kept count (one thread); ids that got no key get the range (0, 0).
// no_pass: the keys had no bits, so no pass ran and every key is id 0.
// status_mirror (nullable, host memory mapped into the device): receives the
// status word after this sort's own status is merged in.
// bucket_counts (nullable, with ranges; 256-thread blocks): adds every tile to
// its list-length bucket (len_bucket), the counts of the persistent blends'
// tile order.
__global__ void k_os_finish(const SortAux *aux, uint64_t *status, uint64_t *kept_out, uint2 *ranges,
                            uint64_t n_ranges, bool no_pass, const uint64_t *n_dev, uint64_t max_n,
                            uint64_t *status_mirror, uint32_t *bucket_counts) {
    chain_enter();
    __shared__ uint32_t h[TB_BUCKETS];
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && !no_pass) {
        if (status && aux->status) *status = aux->status;
        if (kept_out) *kept_out = aux->kept;
    }
    if (i == 0 && status_mirror) *status_mirror = status ? *status : 0u;
    if (!ranges) return;   // uniform
    uint2 rg = make_uint2(0u, 0u);
    if (i < n_ranges) {
        if (no_pass) {
            const uint64_t nd = *n_dev, n = nd <= max_n ? nd : 0;   // none when over capacity
            rg = (i == 0 && n > 0) ? make_uint2(0u, (uint32_t)n) : make_uint2(0u, 0u);
            ranges[i] = rg;
        } else {
            rg = ranges[i];
            if (rg.x == RANGE_EMPTY) {
                rg = make_uint2(0u, 0u);
                ranges[i] = rg;
            }
        }
    }
    if (!bucket_counts) return;   // uniform
    h[threadIdx.x] = 0u;
    __syncthreads();
    if (i < n_ranges) atomicAdd(&h[len_bucket(rg)], 1u);
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&bucket_counts[threadIdx.x], h[threadIdx.x]);
}

cudaError_t launch_radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                              const uint64_t *n_dev, uint64_t max_n, int bits, uint32_t *hist,
                              uint64_t *scan_sums, cudaStream_t s, uint64_t *status, uint64_t *kept_out,
                              bool aux_zeroed, uint2 *ranges, uint64_t n_ranges, bool hist_ready,
                              uint64_t *status_mirror, const uint64_t *skip_status, uint32_t *order_counts) {
    const uint32_t nblocks = (uint32_t)div_up(max_n, RS_TILE);
    const int passes = radix_passes(bits);
    const uint64_t fgrid = ranges ? std::max<uint64_t>(div_up(n_ranges, 256), 1) : 1;
    if (nblocks == 0 || passes == 0) {
        // nothing to sort; ranges still get their final values
        if (ranges) {
            (void)launch_chain(k_os_finish, dim3((unsigned)fgrid), dim3(256), s, reinterpret_cast<SortAux *>(scan_sums),
                               status, nullptr, ranges, n_ranges, passes == 0, n_dev, max_n, status_mirror,
                               order_counts);
            count_launches(1);
            return cudaGetLastError();
        }
        if (status_mirror) {
            (void)launch_chain(k_os_finish, dim3(1), dim3(1), s, reinterpret_cast<SortAux *>(scan_sums), status,
                               nullptr, nullptr, 0, true, n_dev, max_n, status_mirror, nullptr);
            count_launches(1);
            return cudaGetLastError();
        }
        return cudaSuccess;
    }
    if (max_n > (uint64_t)LB_VAL) return cudaErrorInvalidValue;   // counts must fit the look-back word
    SortAux *aux = reinterpret_cast<SortAux *>(scan_sums);
    const bool drop = kept_out != nullptr;
    const uint32_t spin_limit = sort_wait_polls();
    const uint64_t pass_words = (uint64_t)nblocks * RS_RADIX;
    if (!hist_ready) {
        if (!aux_zeroed) {
            const cudaError_t e = cudaMemsetAsync(aux, 0, sizeof(SortAux), s);
            if (e != cudaSuccess) return e;
        }
        const unsigned hgrid = nblocks < 4u * 152u ? nblocks : 4u * 152u;
        (void)launch_chain(k_os_hist, dim3(hgrid), dim3(RS_THREADS), s, k0, n_dev, max_n, bits, drop, aux, hist, pass_words * passes);
        count_launches(1);
    }
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        const int nb = min(8, bits - shift);
        const uint32_t mask = (1u << nb) - 1u;
        // with drop, pass 0 leaves SORT_DROP_KEY out and later passes see only the kept keys
        const uint64_t *np = (drop && p > 0) ? &aux->kept : n_dev;
        uint2 *rg = p == passes - 1 ? ranges : nullptr;
        (void)launch_chain(k_os_pass, dim3(nblocks), dim3(RS_THREADS), s, ki, vi, ko, vo, np, max_n, p, shift, mask, drop && p == 0,
                                                 hist + pass_words * p, aux, rg, n_ranges, spin_limit,
                                                 skip_status);
        count_launches(1);
        uint32_t *t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    if (status || kept_out || ranges || status_mirror) {
        (void)launch_chain(k_os_finish, dim3((unsigned)fgrid), dim3(ranges ? 256 : 1), s, aux, status, kept_out, ranges, n_ranges, false,
                                                                 n_dev, max_n, status_mirror, ranges ? order_counts : nullptr);
        count_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// tile sort by counting (tile counts up to TC_MAX_TILES)
// ---------------------------------------------------------------------------
// The duplicate's pairs, in depth order, are cut into C chunks of equal length.
// k_tc_count counts each chunk's pairs per tile (row c of the [C][row] count
// matrix); k_tc_scan scans the matrix in (tile, chunk) order, which turns row c
// into the first output position of chunk c's pairs of every tile and bounds
// every tile's range; k_tc_place walks each chunk's pairs in order and puts
// each at its tile's next position. Inside a tile the pairs follow the chunks
// in order and, inside a chunk, their input order: the result is the stable
// sort by tile, identical to the LSD radix sort's.
uint32_t tc_chunks(uint64_t cap) {
    const uint64_t c = div_up(cap, TC_CHUNK_TARGET);
    return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(c, 1), TC_MAX_CHUNKS);
}

uint64_t tc_row(uint64_t n_tiles) { return div_up(n_tiles, 4) * 4; }

// [lo, hi): chunk c of the pairs the duplicate wrote; none when the status
// says the pairs are incomplete (capacity overflow, or a bounded wait that
// gave up: the lists may hold stale words).
__device__ __forceinline__ void tc_chunk(const uint64_t *counters, uint64_t cap, uint32_t n_chunks, uint32_t c,
                                         uint64_t &lo, uint64_t &hi) {
    const uint64_t st = counters[CNT_STATUS];
    const uint64_t K = st == (uint64_t)SG_OK ? min(counters[CNT_WRITTEN], cap) : 0ull;
    const uint64_t len = div_up(div_up(K, n_chunks), 32) * 32;
    lo = min(K, (uint64_t)c * len);
    hi = min(K, lo + len);
}

// One block per chunk: shared-memory counters of every tile, then row c.
__global__ void __launch_bounds__(256) k_tc_count(const uint16_t *__restrict__ keys,
                                                  const uint64_t *__restrict__ counters, uint64_t cap,
                                                  uint32_t n_tiles, uint32_t row, uint32_t *__restrict__ counts) {
    chain_enter();
    extern __shared__ uint4 tc_smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(tc_smem);
    for (uint32_t q = threadIdx.x; q < row / 4; q += blockDim.x) tc_smem[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    uint64_t lo, hi;
    tc_chunk(counters, cap, gridDim.x, blockIdx.x, lo, hi);
    // 16-byte loads of 8 keys (a chunk starts at a multiple of 32 keys), then the tail
    const uint64_t n8 = (hi - lo) / 8;
    const uint4 *k8 = reinterpret_cast<const uint4 *>(keys + lo);
#pragma unroll 4
    for (uint64_t q = threadIdx.x; q < n8; q += blockDim.x) {
        const uint4 w = k8[q];
        const uint32_t h[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t a = h[k] & 0xFFFFu, b = h[k] >> 16;
            if (a < n_tiles) atomicAdd(&cnt[a], 1u);
            if (b < n_tiles) atomicAdd(&cnt[b], 1u);
        }
    }
    for (uint64_t i = lo + 8 * n8 + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t t = keys[i];
        if (t < n_tiles) atomicAdd(&cnt[t], 1u);
    }
    __syncthreads();
    uint4 *dst = reinterpret_cast<uint4 *>(counts + (uint64_t)blockIdx.x * row);
    for (uint32_t q = threadIdx.x; q < row / 4; q += blockDim.x) dst[q] = tc_smem[q];
}

// Groups of 32 tiles (lane = tile), taken in order from a ticket by resident
// blocks (two per SM); the chunks split into TC_SCAN_WARPS runs (one per warp),
// whose counts wait in shared memory for the second walk. The sum of each tile's counts and the group's total go
// through a decoupled look-back over the groups before it, which gives every
// tile's first position; the second walk replaces each count with its chunk's
// first position of the tile. Also writes every tile's range ((0, 0) when
// empty) and adds the tile to its list-length bucket.
// words: zeroed; [0] the ticket, [1 + g] group g's look-back word.
constexpr int TC_SCAN_WARPS = 32;
constexpr int TC_SCAN_RUN = (TC_MAX_CHUNKS + TC_SCAN_WARPS - 1) / TC_SCAN_WARPS;
__global__ void __launch_bounds__(TC_SCAN_WARPS * 32, 2) k_tc_scan(uint32_t *__restrict__ counts, uint32_t n_chunks,
                                                              uint32_t row, uint32_t n_tiles,
                                                              uint64_t *__restrict__ words,
                                                              uint2 *__restrict__ ranges,
                                                              uint32_t *__restrict__ bucket_counts,
                                                              uint64_t *__restrict__ status, uint32_t spin_limit) {
    chain_enter();
    __shared__ uint32_t part[TC_SCAN_WARPS][32];
    __shared__ uint32_t s_start[32];
    __shared__ uint32_t s_grp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_groups = (n_tiles + 31) / 32;
    const uint32_t per = (n_chunks + TC_SCAN_WARPS - 1) / TC_SCAN_WARPS;
    const uint32_t c0 = min(n_chunks, warp * per), c1 = min(n_chunks, c0 + per);
    constexpr int RUN = TC_SCAN_RUN;
    extern __shared__ uint32_t cvs[];   // [RUN][block threads]: the run's counts
    for (;;) {
        // every thread is past the previous group's reads of the shared words
        __syncthreads();
        if (threadIdx.x == 0) s_grp = (uint32_t)atomicAdd(reinterpret_cast<unsigned long long *>(words), 1ull);
        __syncthreads();
        const uint32_t grp = s_grp;
        if (grp >= n_groups) break;   // uniform
        const uint32_t t = grp * 32 + lane;
        const bool tv = t < n_tiles;
        uint32_t *col = counts + t;
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < RUN; ++j) {
            const uint32_t c = c0 + (uint32_t)j;
            const uint32_t x = (tv && c < c1) ? col[(uint64_t)c * row] : 0u;
            cvs[j * TC_SCAN_WARPS * 32 + threadIdx.x] = x;
            sum += x;
        }
        part[warp][lane] = sum;
        __syncthreads();
        // each warp its runs' prefix over the warps before it; warp 0 the totals
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += part[w][lane];
        uint32_t tot = 0;
        if (warp == 0) {
#pragma unroll
            for (int w = 0; w < TC_SCAN_WARPS; ++w) tot += part[w][lane];
        }
        if (warp == 0) {
            const uint32_t inc = warp_inclusive(tot);
            const uint32_t grp_total = __shfl_sync(0xffffffffu, inc, 31);
            if (lane == 0) st_relaxed64(words + 1 + grp, DL_AGG | (uint64_t)grp_total);
            const uint64_t excl = block_lookback64(words + 1, grp, grp_total, spin_limit, status);
            const uint32_t start = (uint32_t)(excl + inc - tot);
            s_start[lane] = start;
            if (tv) {
                const uint2 rg = tot ? make_uint2(start, start + tot) : make_uint2(0u, 0u);
                ranges[t] = rg;
                if (bucket_counts) atomicAdd(&bucket_counts[len_bucket(rg)], 1u);
            }
        }
        __syncthreads();
        uint32_t run = s_start[lane] + before;
#pragma unroll
        for (int j = 0; j < RUN; ++j) {
            const uint32_t c = c0 + (uint32_t)j;
            if (tv && c < c1) col[(uint64_t)c * row] = run;
            run += cvs[j * TC_SCAN_WARPS * 32 + threadIdx.x];
        }
    }
}

// One warp per chunk: its row of first positions in shared memory, then the
// chunk's pairs 32 at a time in order (the entries only: a pair's tile is the
// tile whose range holds it). Lanes holding the same tile are grouped
// (match_any); the group's first lane takes as many positions from the tile's
// cursor as the group has lanes, and each lane takes the one of its rank in the
// group. The warp barrier between rounds orders the cursor updates of
// successive rounds. Positions at or past cap are not written.
__global__ void __launch_bounds__(32) k_tc_place(const uint16_t *__restrict__ keys,
                                                 const uint32_t *__restrict__ vals,
                                                 const uint64_t *__restrict__ counters, uint64_t cap,
                                                 uint32_t n_tiles, uint32_t row,
                                                 const uint32_t *__restrict__ first,
                                                 uint32_t *__restrict__ ovals, uint64_t *status_mirror) {
    chain_enter();
    extern __shared__ uint4 tc_smem[];
    uint32_t *next = reinterpret_cast<uint32_t *>(tc_smem);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    if (blockIdx.x == 0 && lane == 0 && status_mirror) *status_mirror = counters[CNT_STATUS];
    // the row arrives by asynchronous 16-byte copies while the first batch loads
    const uint4 *src = reinterpret_cast<const uint4 *>(first + (uint64_t)blockIdx.x * row);
    for (uint32_t q = lane; q < row / 4; q += 32) {
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(tc_smem + q);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + q) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    uint64_t lo, hi;
    tc_chunk(counters, cap, gridDim.x, blockIdx.x, lo, hi);
    const uint32_t lt = (1u << lane) - 1u;
    // rounds of 32 pairs, U rounds per batch; the next batch's keys and values
    // are loaded while this one is placed
    constexpr int U = 8;
    uint32_t tn[U], vn[U];
    auto load = [&](uint64_t base) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t i = base + (uint64_t)(32 * u + lane);
            tn[u] = i < hi ? (uint32_t)keys[i] : 0xFFFFFFFFu;
            vn[u] = i < hi ? vals[i] : 0u;
        }
    };
    load(lo);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    for (uint64_t base = lo; base < hi; base += 32 * U) {
        uint32_t t[U], v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            t[u] = tn[u];
            v[u] = vn[u];
        }
        if (base + 32 * U < hi) load(base + 32 * U);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = t[u] < n_tiles;
            const uint32_t grp = __match_any_sync(FULL, ok ? t[u] : 0xFFFFFFFFu);
            const int leader = __ffs(grp) - 1;
            uint32_t at = 0;
            if (ok && lane == leader) at = atomicAdd(&next[t[u]], (uint32_t)__popc(grp));
            at = __shfl_sync(FULL, at, leader);
            const uint32_t pos = at + (uint32_t)__popc(grp & lt);
            if (ok && pos < cap) ovals[pos] = v[u];
            __syncwarp();
        }
    }
}

cudaError_t launch_tile_count_sort(const uint16_t *keys, const uint32_t *vals, uint32_t *ovals,
                                   uint64_t *counters, uint64_t cap, uint32_t n_tiles, uint32_t n_chunks,
                                   uint32_t *matrix, uint64_t *words, uint2 *ranges, uint32_t *order_counts,
                                   uint64_t *status_mirror, cudaStream_t s) {
    if (n_tiles == 0 || n_tiles > TC_MAX_TILES || n_chunks == 0 || n_chunks > TC_MAX_CHUNKS || cap > UINT32_MAX)
        return cudaErrorInvalidValue;
    const uint32_t row = (uint32_t)tc_row(n_tiles);
    const size_t smem = (size_t)row * 4;
    (void)launch_chain_smem(k_tc_count, dim3(n_chunks), dim3(256), smem, s, keys, (const uint64_t *)counters, cap,
                       n_tiles, row, matrix);
    // resident blocks only: a group's look-back may wait on any earlier group
    const size_t scan_smem = (size_t)TC_SCAN_RUN * TC_SCAN_WARPS * 32 * 4;
    static int scan_blocks = 0;
    if (scan_blocks == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaFuncSetAttribute(k_tc_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scan_smem) !=
                cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_scan, TC_SCAN_WARPS * 32, scan_smem) !=
                cudaSuccess)
            return cudaErrorUnknown;
        scan_blocks = std::max(1, sms * per_sm);
    }
    const unsigned sgrid = (unsigned)std::min<uint64_t>(div_up(n_tiles, 32), (uint64_t)scan_blocks);
    (void)launch_chain_smem(k_tc_scan, dim3(sgrid), dim3(TC_SCAN_WARPS * 32), scan_smem, s, matrix, n_chunks,
                       row, n_tiles, words, ranges, order_counts, counters + CNT_STATUS, sort_wait_polls());
    (void)launch_chain_smem(k_tc_place, dim3(n_chunks), dim3(32), smem, s, keys, vals, (const uint64_t *)counters, cap,
                       n_tiles, row, (const uint32_t *)matrix, ovals, status_mirror);
    count_launches(3);
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

// Adds the keys a, a + 1, .., b - 1 to a block's digit histograms: one count
// per key for the lowest digit, one per run of equal digit above it.
__device__ __forceinline__ void hist_key_run(uint32_t (*h)[RS_RADIX], int passes, uint32_t a, uint32_t b) {
    for (uint32_t t = a; t < b; ++t) atomicAdd(&h[0][t & (RS_RADIX - 1)], 1u);
    for (int p = 1; p < passes; ++p) {
        const int sh = 8 * p;
        for (uint32_t t = a; t < b;) {
            const uint64_t next = ((uint64_t)(t >> sh) + 1u) << sh;   // first key of the next digit
            const uint32_t seg = next < (uint64_t)b ? (uint32_t)next : b;
            atomicAdd(&h[p][(t >> sh) & (RS_RADIX - 1)], seg - t);
            t = seg;
        }
    }
}


// One block per 256 depth-sorted entries, in the order the blocks start
// (logical index from counters[CNT_DUP_BLOCK]). The block's pairs go, entry by
// entry and row by row, to [out0, out0 + the block's total), out0 from the
// look-back over the earlier blocks' totals: work items are (entry, tile row);
// each finds its reached columns once and writes that run (row-major inside an
// entry), so a large rectangle is spread over the whole block and the stores
// stay coalesced. Positions at or past cap are not written. With hist_passes > 0
// the kernel also prepares the tile sort: it clears its look-back flags and
// adds exactly the keys it writes to the digit histograms of its hist_passes
// passes. KeyT: uint32_t, or uint16_t for the counting tile sort (tile ids
// below 2^16).
template <typename KeyT>
__global__ void __launch_bounds__(256) k_duplicate(const Batch *__restrict__ bp, uint64_t M,
                                                   const uint32_t *__restrict__ sorted_ent,
                                                   const uint32_t *__restrict__ tiles_touched,
                                                   const uint2 *__restrict__ rect, const Rec *__restrict__ rec,
                                                   uint64_t *__restrict__ counters, uint64_t cap,
                                                   KeyT *__restrict__ pkey,
                                                   uint32_t *__restrict__ pval, int hist_passes,
                                                   SortAux *__restrict__ aux, uint32_t *__restrict__ flags,
                                                   uint64_t flag_words, uint64_t *__restrict__ dflags,
                                                   uint64_t *mirror, uint32_t spin_limit) {
    chain_enter();
    __shared__ uint32_t s_rinc[256], s_e[256], s_rx[256], s_ry[256], s_base[256], s_tx[256];
    __shared__ TileReach s_R[256];
    __shared__ uint32_t shs[33];
    __shared__ uint32_t h[4][RS_RADIX];
    __shared__ unsigned long long s_blk, s_out0;
    // the tile sort's look-back flags start at zero (its passes run after this kernel)
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < flag_words; i += (uint64_t)gridDim.x * 256)
        flags[i] = 0u;
    for (int i = threadIdx.x; i < 4 * RS_RADIX; i += 256) h[i / RS_RADIX][i % RS_RADIX] = 0u;
    // a sort gave up a bounded wait: its order may hold stale words (uniform)
    if (counters[CNT_STATUS] == (uint64_t)SG_ERR_TIMEOUT) return;
    if (threadIdx.x == 0)
        s_blk = atomicAdd(reinterpret_cast<unsigned long long *>(counters + CNT_DUP_BLOCK), 1ull);
    __syncthreads();
    const uint64_t blk = s_blk;
    const uint64_t j0 = blk * 256;
    const uint64_t j = j0 + threadIdx.x;
    const uint64_t V = min(M, counters[CNT_VISIBLE]);   // entries in depth order with at least one pair
    if (j0 >= V) {   // no entry: only the first block, when there is none at all, reports the zero total
        if (V == 0 && blk == 0 && threadIdx.x == 0 && mirror) mirror[0] = 0;
        return;
    }
    uint32_t e = 0, tt = 0, rows = 0, rx = 0, ry = 0, tbase = 0, tx = 1;
    if (j < V) {
        e = sorted_ent[j];
        tt = e < M ? tiles_touched[e] : 0u;   // an id left by a sort that gave up a wait reaches no tile
    }
    // the block's pair count goes out first; the row bookkeeping below hides the
    // latency of the predecessors' counts
    uint32_t total;
    block_exclusive<uint32_t>(tt, total, shs);
    if (threadIdx.x == 0) st_relaxed64(dflags + blk, DL_AGG | ((uint64_t)total & DL_VAL));
    if (j < V) {
        if (tt) {
            const Batch &b = *bp;
            const ViewDesc &vw = b.view[find_entry_view(b, e)];
            const uint2 rc = rect[e];
            rx = rc.x;
            ry = rc.y;
            rows = (ry >> 16) - (ry & 0xFFFFu);
            tbase = vw.tile_off;
            tx = (uint32_t)vw.tiles_x;
            // the binning reads the record's first 24 bytes: x, y, conic, bound (one sector)
            const float4 ra = rec[e].a;
            const float2 rb = *reinterpret_cast<const float2 *>(&rec[e].b);
            tile_reach_init(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, s_R[threadIdx.x]);
        }
    }
    uint32_t total_rows;
    const uint32_t rexcl = block_exclusive<uint32_t>(rows, total_rows, shs);
    s_rinc[threadIdx.x] = rexcl + rows;
    s_e[threadIdx.x] = e;
    s_rx[threadIdx.x] = rx;
    s_ry[threadIdx.x] = ry;
    s_base[threadIdx.x] = tbase;
    s_tx[threadIdx.x] = tx;
    if (threadIdx.x < 32) {
        const uint64_t excl = block_lookback64(dflags, blk, total, spin_limit, counters + CNT_STATUS);
        if (threadIdx.x == 0) {
            s_out0 = excl;
            if ((V - 1) / 256 == blk) {   // the last block: the totals
                const uint64_t all = excl + total;
                counters[CNT_PAIRS] = all;
                counters[CNT_WRITTEN] = min(all, cap);
                if (mirror) mirror[0] = all;
                if (all > cap)
                    atomicCAS(reinterpret_cast<unsigned long long *>(counters + CNT_STATUS), 0ull,
                              (unsigned long long)SG_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    if (total == 0u) return;
    const uint64_t out0 = s_out0;
    // pairs the block may write: positions below cap only
    const uint32_t lim = out0 >= cap ? 0u : (uint32_t)min((uint64_t)total, cap - out0);
    if (lim == 0u) return;
    uint32_t done = 0u;
    for (uint32_t base = 0; base < total_rows; base += 256) {
        const uint32_t item = base + threadIdx.x;
        int o = 0, row = 0, c0 = 0, c1 = 0;
        if (item < total_rows) {
            // first owner o with s_rinc[o] > item
            int lo = 0, hi = 255;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_rinc[mid] > item) hi = mid; else lo = mid + 1;
            }
            o = lo;
            const uint32_t r0 = o ? s_rinc[o - 1] : 0u;
            row = (int)(s_ry[o] & 0xFFFFu) + (int)(item - r0);
            tile_reach_row(s_R[o], row, (int)(s_rx[o] & 0xFFFFu), (int)(s_rx[o] >> 16), c0, c1);
        }
        uint32_t chunk;
        const uint32_t at = done + block_exclusive<uint32_t>((uint32_t)(c1 - c0), chunk, shs);
        const uint32_t key0 = s_base[o] + (uint32_t)row * s_tx[o];
        for (int c = c0; c < c1; ++c) {
            const uint32_t q = at + (uint32_t)(c - c0);
            if (q < lim) {   // rows sum to tiles_touched by construction; never write past the block or cap
                pkey[out0 + q] = (KeyT)(key0 + (uint32_t)c);
                pval[out0 + q] = s_e[o];
            }
        }
        if (hist_passes > 0 && at < lim)   // the keys written above, no more
            hist_key_run(h, hist_passes, key0 + (uint32_t)c0,
                         key0 + (uint32_t)c0 + min((uint32_t)(c1 - c0), lim - at));
        done += chunk;
    }
    // Rows add up to tiles_touched by construction. Should they ever fall short,
    // the rest of the block's range still gets valid tile ids and entries.
    for (uint32_t q = done + threadIdx.x; q < lim; q += 256) {
        pkey[out0 + q] = (KeyT)s_base[0];
        pval[out0 + q] = s_e[0];
        if (hist_passes > 0) hist_key_run(h, hist_passes, s_base[0], s_base[0] + 1u);
    }
    if (hist_passes > 0) {
        __syncthreads();
        for (int i = threadIdx.x; i < hist_passes * RS_RADIX; i += 256) {
            const uint32_t c = h[i / RS_RADIX][i % RS_RADIX];
            if (c) atomicAdd(&aux->hist[i / RS_RADIX][i % RS_RADIX], c);
        }
    }
}

cudaError_t launch_duplicate(const Batch *db, uint64_t M, const uint32_t *sorted_ent,
                             const uint32_t *tiles_touched, const uint2 *rect, const Rec *rec, uint64_t *counters,
                             uint64_t cap, void *pkey, uint32_t *pval, uint64_t *dup_flags, uint64_t *mirror,
                             cudaStream_t s, int hist_passes, uint64_t *sort_aux, uint32_t *flags,
                             uint64_t flag_words, bool key16) {
    if (key16 && hist_passes > 0) return cudaErrorInvalidValue;   // 16-bit keys feed the counting sort only
    // one block at least: it reports the zero total of a call without entries
    const uint64_t grid = std::max<uint64_t>(div_up(M, 256), 1);
    SortAux *aux = reinterpret_cast<SortAux *>(sort_aux);
    if (key16)
        (void)launch_chain(k_duplicate<uint16_t>, dim3((unsigned)grid), dim3(256), s, db, M, sorted_ent,
                           tiles_touched, rect, rec, counters, cap, static_cast<uint16_t *>(pkey), pval, hist_passes,
                           aux, flags, flag_words, dup_flags, mirror, sort_wait_polls());
    else
        (void)launch_chain(k_duplicate<uint32_t>, dim3((unsigned)grid), dim3(256), s, db, M, sorted_ent,
                           tiles_touched, rect, rec, counters, cap, static_cast<uint32_t *>(pkey), pval, hist_passes,
                           aux, flags, flag_words, dup_flags, mirror, sort_wait_polls());
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// work order of the persistent blend: tiles by descending list length
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tile_bucket_scatter(const uint2 *__restrict__ ranges, uint32_t n_tiles,
                                                             const uint32_t *__restrict__ counts,
                                                             uint32_t *__restrict__ cursor,
                                                             uint32_t *__restrict__ order) {
    chain_enter();
    __shared__ uint32_t base[TB_BUCKETS];
    __shared__ uint32_t shs[33];
    // longest lists first: exclusive scan over the buckets in reverse
    const uint32_t c = counts[TB_BUCKETS - 1 - threadIdx.x];
    uint32_t tot;
    base[TB_BUCKETS - 1 - threadIdx.x] = block_exclusive<uint32_t>(c, tot, shs);
    __syncthreads();
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
        const uint32_t b = len_bucket(ranges[t]);
        order[base[b] + atomicAdd(&cursor[b], 1u)] = t;
    }
}

cudaError_t launch_tile_order(const uint2 *ranges, uint32_t n_tiles, uint32_t *order, uint32_t *scratch,
                              cudaStream_t s) {
    static_assert(TILE_ORDER_WORDS == 2 * TB_BUCKETS, "tile order scratch");
    if (n_tiles == 0) return cudaSuccess;
    uint32_t *counts = scratch, *cursor = scratch + TB_BUCKETS;
    const uint64_t want = div_up(n_tiles, 256);
    const unsigned grid = (unsigned)(want < 608u ? want : 608u);
    (void)launch_chain(k_tile_bucket_scatter, dim3(grid), dim3(256), s, ranges, n_tiles, counts, cursor, order);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sgk
