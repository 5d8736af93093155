// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits.
//
// The sparse grid needs it only for boxes whose block bit mask would exceed
// 64 MiB, where it puts the active block keys in ascending Eq.-(key) order
// (the canonical compaction that fixes Phi; smaller boxes rank blocks by the
// mask and a popcount, and sort particles by a counting sort).  The dense
// grid uses it every step to reorder particles by (block, cell, id), and the
// allocation-free active-set entry point to sort its block keys.
// Each pass is reduce-then-scan: per-tile digit histograms, a scan of every
// digit's row of tile counts, and a stable scatter that ranks keys inside a
// tile with warp match/popc.  The live element count may sit in device
// memory (written by an earlier kernel), so a pass needs no host sync.
#include "mpm_internal.cuh"

namespace mpm {

namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RADIX = 256;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int64_t live_count(const unsigned int* n_dev, int64_t n_cap,
                                              const unsigned int* abort) {
    if (abort && *abort) return 0;   // the step was abandoned
    if (!n_dev) return n_cap;
    int64_t n = (int64_t)(*n_dev);
    return n < n_cap ? n : n_cap;
}

// Element j of lane `lane` in warp `w` of tile `t`: warps own contiguous
// segments of 32*ITEMS keys, so (warp, round, lane) order is index order.
__device__ __forceinline__ int64_t item_index(int t, int w, int j, int lane) {
    return (int64_t)t * RS_TILE + (int64_t)w * 32 * RS_ITEMS + j * 32 + lane;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n_cap,
                                                         const unsigned int* n_dev, int shift,
                                                         uint32_t* __restrict__ counts, int ntiles,
                                                         const unsigned int* abort) {
    __shared__ uint32_t hist[RS_WARPS][RADIX];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) (&hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = live_count(n_dev, n_cap, abort);
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        int64_t idx = item_index(blockIdx.x, w, j, lane);
        unsigned d = idx < n ? (keys[idx] >> shift) & (RADIX - 1) : RADIX;
        unsigned peers = __match_any_sync(FULL, d);
        if (d < RADIX && lane == __ffs(peers) - 1) hist[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) {
        uint32_t s = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) s += hist[ww][d];
        counts[(int64_t)d * ntiles + blockIdx.x] = s;
    }
}

// One CTA per digit: exclusive scan of that digit's tile counts, in place.
__global__ void __launch_bounds__(1024) k_rs_scan_rows(uint32_t* __restrict__ counts, int ntiles,
                                                        uint32_t* __restrict__ totals) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* row = counts + (int64_t)blockIdx.x * ntiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < ntiles ? row[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(FULL, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const uint32_t excl = carry + (w ? wsum[w - 1] : 0u) + x - v;
        if (i < ntiles) row[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin,
                                                            uint32_t* __restrict__ kout,
                                                            uint32_t* __restrict__ vout, int64_t n_cap,
                                                            const unsigned int* n_dev, int shift,
                                                            const uint32_t* __restrict__ counts,
                                                            const uint32_t* __restrict__ totals, int ntiles,
                                                            const unsigned int* abort) {
    __shared__ uint32_t off[RS_WARPS][RADIX];
    __shared__ uint32_t dbase[RADIX];
    __shared__ uint32_t wsum[RS_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = live_count(n_dev, n_cap, abort);

    // global start of every digit for this tile: exclusive scan of the digit
    // totals plus this tile's scanned count
    {
        const int d = threadIdx.x;   // RS_THREADS == RADIX
        const uint32_t v = totals[d];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) (&off[0][0])[i] = 0;
        __syncthreads();
        uint32_t pre = 0;
        for (int ww = 0; ww < w; ++ww) pre += wsum[ww];
        dbase[d] = pre + x - v + counts[(int64_t)d * ntiles + blockIdx.x];
    }

    uint32_t kk[RS_ITEMS], vv[RS_ITEMS];
    unsigned dd[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        int64_t idx = item_index(blockIdx.x, w, j, lane);
        if (idx < n) {
            kk[j] = kin[idx];
            vv[j] = vin[idx];
            dd[j] = (kk[j] >> shift) & (RADIX - 1);
        } else {
            kk[j] = vv[j] = 0;
            dd[j] = RADIX;
        }
        unsigned peers = __match_any_sync(FULL, dd[j]);
        if (dd[j] < RADIX && lane == __ffs(peers) - 1) off[w][dd[j]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per (digit, warp) start = digit start + counts of earlier warps
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) {
        uint32_t run = dbase[d];
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            uint32_t t = off[ww][d];
            off[ww][d] = run;
            run += t;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const unsigned d = dd[j];
        const unsigned peers = __match_any_sync(FULL, d);
        if (d < RADIX) {
            const uint32_t pos = off[w][d] + __popc(peers & lt);
            kout[pos] = kk[j];
            vout[pos] = vv[j];
        }
        __syncwarp();
        if (d < RADIX && lane == __ffs(peers) - 1) off[w][d] += __popc(peers);
        __syncwarp();
    }
}
}  // namespace

cudaError_t radix_reserve(mpm_ctx* c, int64_t n_cap) {
    int64_t tiles = (n_cap + RS_TILE - 1) / RS_TILE;
    if (tiles < 1) tiles = 1;
    if (tiles <= c->rs.tiles_cap && c->rs.counts) return cudaSuccess;
    dfree(c, c->rs.counts, sizeof(uint32_t) * RADIX * c->rs.tiles_cap);
    c->rs.counts = nullptr;
    if (!c->rs.totals) {
        cudaError_t e = dalloc(c, (void**)&c->rs.totals, sizeof(uint32_t) * RADIX);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = dalloc(c, (void**)&c->rs.counts, sizeof(uint32_t) * RADIX * tiles);
    if (e != cudaSuccess) return e;
    c->rs.tiles_cap = tiles;
    return cudaSuccess;
}

int radix_sort_pairs(mpm_ctx* c, uint32_t* k[2], uint32_t* v[2], int64_t n_cap, const unsigned int* n_dev,
                     int bits, cudaStream_t st, const unsigned int* abort) {
    if (n_cap <= 1 || bits <= 0) return 0;
    const int ntiles = (int)((n_cap + RS_TILE - 1) / RS_TILE);
    const int passes = (bits + 7) / 8;
    int sel = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<ntiles, RS_THREADS, 0, st>>>(k[sel], n_cap, n_dev, shift, c->rs.counts, ntiles, abort);
        k_rs_scan_rows<<<RADIX, 1024, 0, st>>>(c->rs.counts, ntiles, c->rs.totals);
        k_rs_scatter<<<ntiles, RS_THREADS, 0, st>>>(k[sel], v[sel], k[1 - sel], v[1 - sel], n_cap, n_dev, shift,
                                                     c->rs.counts, c->rs.totals, ntiles, abort);
        sel = 1 - sel;
        c->launches += 3;
    }
    return sel;
}

// The same passes with caller-provided scratch (counts: 256 * ceil(n_cap/2048)
// words, totals: 256 words) and no context.
int radix_sort_pairs_scratch(uint32_t* k[2], uint32_t* v[2], int64_t n_cap, const unsigned int* n_dev, int bits,
                             uint32_t* counts, uint32_t* totals, cudaStream_t st) {
    if (n_cap <= 1 || bits <= 0) return 0;
    const int ntiles = (int)((n_cap + RS_TILE - 1) / RS_TILE);
    const int passes = (bits + 7) / 8;
    int sel = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<ntiles, RS_THREADS, 0, st>>>(k[sel], n_cap, n_dev, shift, counts, ntiles, nullptr);
        k_rs_scan_rows<<<RADIX, 1024, 0, st>>>(counts, ntiles, totals);
        k_rs_scatter<<<ntiles, RS_THREADS, 0, st>>>(k[sel], v[sel], k[1 - sel], v[1 - sel], n_cap, n_dev, shift, counts,
                                                     totals, ntiles, nullptr);
        sel = 1 - sel;
    }
    return sel;
}

}  // namespace mpm
