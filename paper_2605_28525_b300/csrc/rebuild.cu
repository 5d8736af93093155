// Active-set rebuild: Sec. 4.3, Alg. 5-7, with a canonical compaction.
//
//   k_hash_clear      Alg. 5: keys <- EMPTY, values <- invalid, counter <- 0
//                     (the overflow flag is already clear: the host clears it
//                     before a retry, and a raised flag stops the step).
//   k_insert          Alg. 6: per particle, the blocks of its 27 stencil nodes
//                     (at most 8 for B = 4, 27 for B = 1), deduplicated inside
//                     the warp with match.any so one lane per distinct key
//                     probes; CAS(EMPTY -> key) claims a slot, the counter
//                     appends the key to the active list, linear probing up to
//                     n_probe, overflow flag on failure or capacity excess.
//   (host)            Alg. 7: on overflow double H (and the list capacity)
//                     and insert again.
//   k_assign_bits     Phi(b) = rank of b in ascending Eq.-(key) order: the
//                     insert also sets b's bit in a bit mask over the blocks
//                     of the box, and the rank is the bit count below it (a
//                     scan of the words' counts, then a popcount); written to
//                     the table value of its slot; block coordinates per
//                     Phi; the block's grid nodes are zeroed for P2G.
//                     (k_assign: the same from a radix sort of the keys, for
//                     boxes whose mask would be too large.)
//   k_neighbours      Phi of the blocks b + {0,1}^3 (b + {0,1,2}^3 for B = 1)
//                     of every active block, for P2G and G2P.
//   k_particle_keys   dense grid: sort key (Phi(b(base)), l(base)) per
//                     particle, a radix sort, and k_ranges: particle range of
//                     every block that holds particles and the list of such
//                     blocks.
//   k_particle_bins   sparse grid: a counting sort.  Bin (Phi, cell) and
//   k_scan_tiles      rank in the bin per particle, and a tile scan of the
//                     bins; then
//   k_block_prep      in the fast mode at B = 4: per block, its particle
//   k_scatter_kmajor  range, neighbour table and cells ordered by count, and
//                     one scatter straight to the k-major order (the k-th
//                     particle of each cell, then the next) by its closed
//                     form;
//   k_bin_scatter     otherwise (deterministic mode, B = 1): the scatter
//   k_block_ranges    into (block, cell) order, then the particle ranges and
//                     the neighbour table;
//   k_interleave      at B = 4 after those and after the dense grid's radix
//                     sort: the k-major order inside every block (each
//                     cell's particles in id order in deterministic mode)
//                     and the particle count per cell.
#include <algorithm>

#include "mpm_internal.cuh"

namespace mpm {

namespace {

// Start of a step.  Nothing here sets the abort word, so every thread reads
// the same value.  `go` tells the insert whether to run: the insert cannot
// test `abort` itself, since its own overflow would stop its later CTAs and
// the block count the host regrows from would come out short.
__global__ void k_hash_clear(unsigned long long* __restrict__ keys, int* __restrict__ vals, int64_t H,
                             uint32_t* __restrict__ bmask, int64_t bwords, DevStatus* st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ab = st->abort != 0u;
    if (i == 0) st->go = ab ? 0u : 1u;
    if (ab) return;
    for (int64_t j = i; j < H; j += (int64_t)gridDim.x * blockDim.x) {
        keys[j] = EMPTY_KEY;
        vals[j] = -1;
    }
    for (int64_t j = i; j < bwords; j += (int64_t)gridDim.x * blockDim.x) bmask[j] = 0u;
    if (i == 0) {
        st->n_active = 0;
        st->n_pblocks = 0;
        st->work = 0;
        st->gen += 1u;
    }
}

// Dense grid: the identity map has every block of the box.
__global__ void k_status_clear(DevStatus* st, unsigned int n_dom_blocks) {
    const bool ab = st->abort != 0u;
    st->go = ab ? 0u : 1u;
    if (ab) return;
    st->n_active = n_dom_blocks;
    st->n_pblocks = 0;
    st->work = 0;
    st->gen += 1u;
}

// Flags found while a thread works through its particles are collected as
// bits and raised once at the end of the kernel (raise_errors): a flag raise
// (two atomics) inside the per-particle code would constrain how its loads
// and probes are scheduled.
enum : unsigned { ERR_NUMERIC = 1u, ERR_DOMAIN = 2u, ERR_PROBE = 4u, ERR_LIST = 8u };

__device__ __forceinline__ void raise_errors(DevStatus* st, unsigned err) {
    if (!err) return;
    if (err & ERR_NUMERIC) raise_flag(st, &st->numeric, 1u);
    if (err & ERR_DOMAIN) raise_flag(st, &st->out_of_domain, 1u);
    if (err & ERR_PROBE) raise_flag(st, &st->overflow, 1u);
    if (err & ERR_LIST) raise_flag(st, &st->overflow, 2u);
}

// Alg. 6 for one key; returns the slot holding it or -1 when n_probe slots
// were all taken by other keys (overflow).
__device__ int hash_insert(const HashView& hv, uint64_t key, uint32_t rkey, int max_probe,
                           uint32_t* __restrict__ akey, uint32_t* __restrict__ aslot, int64_t cap,
                           uint32_t* __restrict__ bmask, DevStatus* st, unsigned& err) {
    uint64_t s = mix64(key) & hv.mask;
    for (int r = 0; r < max_probe; ++r) {
        // an L1-cached read: a key, once claimed, stays for the whole step, so a
        // stale copy can only read EMPTY, and the CAS below then decides
        unsigned long long cur = __ldca(&hv.keys[s]);
        if (cur == key) return (int)s;
        if (cur == EMPTY_KEY) {
            unsigned long long old = atomicCAS(&hv.keys[s], EMPTY_KEY, (unsigned long long)key);
            if (old == EMPTY_KEY) {
                if (bmask) atomicOr(&bmask[rkey >> 5], 1u << (rkey & 31u));
                // one counter add for the lanes that claimed a key in this probe step
                const unsigned grp = __activemask();
                const int lead = __ffs(grp) - 1, me = (int)(threadIdx.x & 31);
                unsigned base = 0;
                if (me == lead) base = atomicAdd(&st->n_active, (unsigned)__popc(grp));
                const unsigned idx = __shfl_sync(grp, base, lead) + __popc(grp & ((1u << me) - 1u));
                if ((int64_t)idx < cap) {
                    akey[idx] = rkey;
                    aslot[idx] = (uint32_t)s;
                } else {
                    err |= ERR_LIST;
                }
                return (int)s;
            }
            if (old == key) return (int)s;
        }
        s = (s + 1) & hv.mask;
    }
    err |= ERR_PROBE;
    return -1;
}

// Checks x and computes the stencil base node; false if the particle is
// unusable (error bits set).
__device__ __forceinline__ bool particle_base_x(const float x[3], const Params& P, int base[3], unsigned& err) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float fx = x[a] * P.inv_h;
        if (!isfinite(fx)) {
            err |= ERR_NUMERIC;
            ok = false;
            base[a] = 0;
            continue;
        }
        // the stencil base..base+2 must lie inside the node box
        if (!(fx >= (float)P.lo[a] + 0.5f && fx < (float)(P.hi[a] - 2) + 1.5f)) {
            err |= ERR_DOMAIN;
            ok = false;
            base[a] = 0;
            continue;
        }
        base[a] = base_index(fx);
    }
    return ok;
}

__device__ __forceinline__ bool particle_base(const float* __restrict__ ps, int64_t stride, int64_t p,
                                              const Params& P, int base[3], unsigned& err) {
    const float4 a0 = reinterpret_cast<const float4*>(ps)[pel4(p, 0)];
    const float x[3] = {a0.x, a0.y, a0.z};
    return particle_base_x(x, P, base, err);
}

// The stencil of one particle: its base block b0 (shifted by its scenario's
// pitch in an ensemble), the mask of the blocks b0 + {0..R-1}^3 that hold
// one of its 27 nodes, the key of b0 (EMPTY_KEY for an unusable particle or
// p >= n) and its cell in b0.
template <int B>
struct Stencil {
    int b0[3];
    unsigned need;   // bit j: block b0 + (j / R^2, (j / R) % R, j % R) holds a stencil node
    uint64_t key0;
    int cell;
    bool ok;
};

template <int B>
__device__ __forceinline__ Stencil<B> particle_stencil(const float* __restrict__ ps, int64_t stride, int64_t n,
                                                       int64_t p, const float x[3], const Params& P, unsigned& err) {
    constexpr int S = (B == 4) ? 2 : 0;
    constexpr int R = (B == 4) ? 2 : 3;   // blocks a stencil can span per axis
    constexpr int NJ = R * R * R;
    Stencil<B> t;
    int base[3] = {0, 0, 0};
    t.ok = p < n;
    if (t.ok) t.ok = particle_base_x(x, P, base, err);
    t.need = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) t.b0[a] = base[a] >> S;
    if (t.ok) {
        int nbk[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) nbk[a] = ((base[a] + 2) >> S) - t.b0[a] + 1;
        if (B == 4) {
            // bit j = 4 ex + 2 ey + ez: the offsets allowed along each axis as
            // masks (ex = 0 only: bits 0-3; ey = 0 only: 0, 1, 4, 5; ez = 0
            // only: the even bits), and their intersection
            t.need = (nbk[0] > 1 ? 0xffu : 0x0fu) & (nbk[1] > 1 ? 0xffu : 0x33u) & (nbk[2] > 1 ? 0xffu : 0x55u);
        } else {
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j / (R * R) < nbk[0] && (j / R) % R < nbk[1] && j % R < nbk[2]) t.need |= 1u << j;
        }
    }
    // An ensemble's scenario s has its blocks ens_pitch * s further along x.
    if (P.n_scen > 1 && t.ok) t.b0[0] += scenario_of(P, __float_as_uint(ps[pel(p, PID)])) * P.ens_pitch;
    t.key0 = t.ok ? pack_key(t.b0[0], t.b0[1], t.b0[2]) : EMPTY_KEY;
    t.cell = (base[0] & (B - 1)) + B * ((base[1] & (B - 1)) + B * (base[2] & (B - 1)));
    return t;
}

// SCAN: the scan realisation (Sec. 4.2, Alg. 2): the block's bit is set in
// the mask and its "slot" is its relative key; no table.  Otherwise Alg. 6
// (hash_insert) and the table slot.  Block b0 + offset j.
template <int B, bool SCAN>
__device__ __forceinline__ int insert_block(const Params& P, const HashView& hv, const int b0[3], int j,
                                            uint32_t* __restrict__ akey, uint32_t* __restrict__ aslot, int64_t cap,
                                            uint32_t* __restrict__ bmask, DevStatus* st, unsigned& err) {
    constexpr int R = (B == 4) ? 2 : 3;
    const int bi = b0[0] + j / (R * R), bj = b0[1] + (j / R) % R, bk = b0[2] + j % R;
    if (SCAN) {
        const uint32_t rk = rel_key(P, bi, bj, bk), bit = 1u << (rk & 31u);
        if (!(*((volatile uint32_t*)&bmask[rk >> 5]) & bit)) atomicOr(&bmask[rk >> 5], bit);
        return (int)rk;
    }
    return hash_insert(hv, pack_key(bi, bj, bk), rel_key(P, bi, bj, bk), P.max_probe, akey, aslot, cap, bmask, st,
                       err);
}

__device__ __forceinline__ void write_code(uint32_t* __restrict__ pcode, int64_t p, bool ok, int slot0, int cell,
                                           int B3) {
    if (ok) pcode[p] = slot0 < 0 ? 0xffffffffu : (uint32_t)slot0 * (uint32_t)B3 + (uint32_t)cell;
}

// One particle per lane (every lane of the warp calls it).  Lanes with the
// same base block form one group (particles are sorted, so a warp usually
// holds one group).  The group's union of needed blocks is one OR reduction
// (one ballot per block offset when the warp holds several groups), and
// member r inserts offsets r, r + group size, ..., so the probes of one warp
// run in parallel.
template <int B, bool SCAN>
__device__ __forceinline__ void insert_group(const Stencil<B>& t, int64_t p, const Params& P, const HashView& hv,
                                             uint32_t* __restrict__ akey, uint32_t* __restrict__ aslot, int64_t cap,
                                             uint32_t* __restrict__ bmask, uint32_t* __restrict__ pcode,
                                             DevStatus* st, unsigned& err) {
    constexpr int R = (B == 4) ? 2 : 3;
    constexpr int NJ = R * R * R;
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const unsigned peers = __match_any_sync(FULL, t.key0);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int gsize = __popc(peers);
    unsigned gneed = 0;
    if (peers == FULL) {
        gneed = __reduce_or_sync(FULL, t.need);   // the usual case: one group per warp
    } else {
#pragma unroll
        for (int j = 0; j < NJ; ++j)
            if (__ballot_sync(FULL, (t.need >> j) & 1u) & peers) gneed |= 1u << j;
    }
    int myslot = -1;
    if (t.ok) {
        // member `rank` takes block offsets rank, rank + gsize, ...
        for (int j = rank; j < NJ; j += gsize) {
            if (!((gneed >> j) & 1u)) continue;
            const int slot = insert_block<B, SCAN>(P, hv, t.b0, j, akey, aslot, cap, bmask, st, err);
            if (j == 0) myslot = slot;   // offset 0 (the base block) is taken by rank 0 = the leader
        }
    }
    write_code(pcode, p, t.ok, __shfl_sync(FULL, myslot, leader), t.cell, B * B * B);
}

#ifndef MPM_INSERT_PER_LANE
#define MPM_INSERT_PER_LANE 2
#endif
constexpr int INS_PL = MPM_INSERT_PER_LANE;   // particles per lane in the insert

// Each warp takes 32 x INS_PL consecutive particles, p, p + 32, ... per
// lane; all their coordinates are loaded before the first one's probes, so
// the later loads overlap them.  With B = 4 and two particles per lane, when
// each half of the warp is one group (the usual case, particles being
// sorted) both halves probe in one phase: one OR reduction over all 64
// particles when they share their base block, else lanes 0-7 take the first
// half's offsets and lanes 16-23 the second's.  Otherwise each half is
// inserted as one group after the other.
// Registers capped for MPM_INSERT_MINB CTAs per SM (8: 64 warps): the
// insert waits on its coordinate loads and probes, and more warps in flight
// hide more of that (the 8M landslide's step 2% faster than at 39 registers
// and 6 CTAs).
#ifndef MPM_INSERT_MINB
#define MPM_INSERT_MINB 8
#endif
template <int B, bool SCAN>
__global__ void __launch_bounds__(256, MPM_INSERT_MINB) k_insert(const float* __restrict__ ps, int64_t stride, int64_t n,
                                                Params P, HashView hv, uint32_t* __restrict__ akey,
                                                uint32_t* __restrict__ aslot, int64_t cap,
                                                uint32_t* __restrict__ bmask, uint32_t* __restrict__ pcode,
                                                DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * INS_PL + lane;
    float xs[INS_PL][3];
#pragma unroll
    for (int h = 0; h < INS_PL; ++h) {
        // plane 0 of the particle: x and alpha (read before the go test: in
        // bounds, and its latency overlaps the test's)
        const float4 a0 = (p0 + 32 * h < n) ? reinterpret_cast<const float4*>(ps)[pel4(p0 + 32 * h, 0)]
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
        xs[h][0] = a0.x;
        xs[h][1] = a0.y;
        xs[h][2] = a0.z;
    }
    if (st->go == 0u) return;   // written by the clear before this kernel: uniform
    unsigned err = 0u;
    Stencil<B> t[INS_PL];
#pragma unroll
    for (int h = 0; h < INS_PL; ++h) t[h] = particle_stencil<B>(ps, stride, n, p0 + 32 * h, xs[h], P, err);
    bool done = false;
    if (B == 4 && INS_PL == 2) {
        const unsigned pa = __match_any_sync(FULL, t[0].key0), pb = __match_any_sync(FULL, t[INS_PL - 1].key0);
        if (pa == FULL && pb == FULL) {   // warp-uniform: each half is one group
            const Stencil<B>& ta = t[0];
            const Stencil<B>& tb = t[INS_PL - 1];
            const bool same = ta.key0 == tb.key0;
            const unsigned na = __reduce_or_sync(FULL, ta.need), nb = __reduce_or_sync(FULL, tb.need);
            const bool second = lane >= 16;
            const int j = lane & 15;
            const unsigned gneed = same ? (na | nb) : (second ? nb : na);
            int slot = -1;
            if (j < 8 && !(same && second) && ((gneed >> j) & 1u))
                slot = insert_block<B, SCAN>(P, hv, second ? tb.b0 : ta.b0, j, akey, aslot, cap, bmask, st, err);
            const int sa = __shfl_sync(FULL, slot, 0), sb = __shfl_sync(FULL, slot, same ? 0 : 16);
            write_code(pcode, p0, ta.ok, sa, ta.cell, B * B * B);
            write_code(pcode, p0 + 32 * (INS_PL - 1), tb.ok, sb, tb.cell, B * B * B);
            done = true;
        }
    }
    if (!done) {
#pragma unroll
        for (int h = 0; h < INS_PL; ++h)
            insert_group<B, SCAN>(t[h], p0 + 32 * h, P, hv, akey, aslot, cap, bmask, pcode, st, err);
    }
    raise_errors(st, err);
}

// Dense comparator: the identity map.  The particle's sort key is the block's
// linear index in the box times B^3 plus the cell.
template <int B>
__global__ void __launch_bounds__(256) k_dense_codes(const float* __restrict__ ps, int64_t stride, int64_t n,
                                                     Params P, uint32_t* __restrict__ pcode, DevStatus* st) {
    constexpr int S = (B == 4) ? 2 : 0;
    if (st->go == 0u) return;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int base[3];
    unsigned err = 0u;
    if (!particle_base(ps, stride, p, P, base, err)) {
        raise_errors(st, err);
        return;
    }
    const int cell = (base[0] & (B - 1)) + B * ((base[1] & (B - 1)) + B * (base[2] & (B - 1)));
    pcode[p] = rel_key(P, base[0] >> S, base[1] >> S, base[2] >> S) * (uint32_t)(B * B * B) + (uint32_t)cell;
}

// Phi in key order: the sorted list position is the compact block index.
// Tile scans (k_scan_tiles, k_bits_scan_tiles): each tile of SC_TILE items
// is scanned locally, and the last CTA turns the tile totals into exclusive
// tile offsets (tsum[ntiles] = the total).  Readers add the offset of the
// item's tile themselves; there is no separate pass that adds it.
constexpr int SC_THREADS = 256, SC_ITEMS = 8, SC_TILE = SC_THREADS * SC_ITEMS;

// Exclusive prefix at item i (0 <= i <= n) of a tile scan over n items.
__device__ __forceinline__ int scan_at(const int* __restrict__ local, const int* __restrict__ tsum, int64_t i,
                                       int64_t n, int ntiles) {
    return i < n ? local[i] + tsum[i / SC_TILE] : tsum[ntiles];
}

__global__ void k_assign(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sslot, int64_t cap,
                         const DevStatus* st, Params P, int* __restrict__ hvals, int4* __restrict__ bcoord,
                         float4* __restrict__ gmv, float4* __restrict__ gf, int* __restrict__ bins, int B3,
                         int zero_grid) {
    if (cta_aborted(st)) return;
    const int64_t nact = live_blocks(st, cap);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nact * B3) return;
    const int64_t r = i / B3;
    if (i % B3 == 0) {
        hvals[sslot[r]] = (int)r;
        int bi, bj, bk;
        rel_decode(P, skey[r], bi, bj, bk);
        bcoord[r] = make_int4(bi, bj, bk, 0);
    }
    if (zero_grid) {
        gmv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        gf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (bins) bins[i] = 0;   // counting-sort bins: one per (block, cell) = one per node
}

// Phi from the block bit mask: the rank of a key is the number of set bits
// below it (the word's local prefix plus its tile's offset, then the bits
// below it in the word).  Thread i handles node i % B3 of the i / B3-th
// inserted block.
__global__ void k_assign_bits(const uint32_t* __restrict__ akey, const uint32_t* __restrict__ aslot, int64_t cap,
                              const DevStatus* st, Params P, const uint32_t* __restrict__ bmask,
                              const int* __restrict__ bpre, const int* __restrict__ btsum,
                              int* __restrict__ hvals, int4* __restrict__ bcoord,
                              float4* __restrict__ gmv, float4* __restrict__ gf, int* __restrict__ bins, int B3,
                              int zero_grid) {
    if (cta_aborted(st)) return;
    const int64_t nact = live_blocks(st, cap);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nact * B3) return;
    const int64_t q = i / B3;
    const int l = (int)(i % B3);
    const uint32_t key = akey[q];
    const uint32_t w = key >> 5;
    const int64_t r = (int64_t)bpre[w] + btsum[w / SC_TILE] + __popc(bmask[w] & ((1u << (key & 31u)) - 1u));
    if (l == 0) {
        hvals[aslot[q]] = (int)r;
        int bi, bj, bk;
        rel_decode(P, key, bi, bj, bk);
        bcoord[r] = make_int4(bi, bj, bk, 0);
    }
    const int64_t node = r * B3 + l;
    if (zero_grid) {
        gmv[node] = make_float4(0.f, 0.f, 0.f, 0.f);
        gf[node] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (bins) bins[node] = 0;
}

// Scan mode: block coordinates per Phi from the marked bits (thread per mask
// word), and the live grid nodes and counting-sort bins zeroed.
__global__ void k_assign_scan(const uint32_t* __restrict__ bmask, const int* __restrict__ bpre, int64_t words,
                              int64_t cap, const DevStatus* st, Params P, int4* __restrict__ bcoord,
                              float4* __restrict__ gmv, float4* __restrict__ gf, int* __restrict__ bins, int B3,
                              int zero_grid) {
    if (cta_aborted(st)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t w = t0; w < words; w += stride) {
        uint32_t m = bmask[w];
        int64_t r = bpre[w];
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            int bi, bj, bk;
            rel_decode(P, (uint32_t)(w * 32 + b), bi, bj, bk);
            if (r < cap) bcoord[r] = make_int4(bi, bj, bk, 0);
            ++r;
        }
    }
    const int64_t nn = live_blocks(st, cap) * B3;
    for (int64_t i = t0; i < nn; i += stride) {
        if (zero_grid) {
            gmv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            gf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (bins) bins[i] = 0;
    }
}

// Scan mode: the block count is the scan's total; beyond the capacity the
// step stops (overflow bit 1, as for the table's list).
__global__ void k_scan_count(const int* __restrict__ bpre, int64_t words, int64_t cap, DevStatus* st) {
    if (st->go == 0u) return;
    const unsigned tot = (unsigned)bpre[words];
    st->n_active = tot;
    if ((int64_t)tot > cap) raise_flag(st, &st->overflow, 2u);
}

// Phi of the blocks b + {0..R-1}^3 of every active block (runs after
// k_assign, once every table value holds its rank).
template <int B>
__global__ void k_neighbours(const int4* __restrict__ bcoord, int64_t cap, const DevStatus* st, Params P,
                             HashView hv, int* __restrict__ nbr) {
    constexpr int R = (B == 4) ? 2 : 3;
    constexpr int NNB = R * R * R;
    if (cta_aborted(st)) return;
    const int64_t nact = live_blocks(st, cap);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nact * NNB) return;
    const int64_t r = t / NNB;
    const int e = (int)(t % NNB);
    const int4 b = bcoord[r];
    nbr[t] = lookup_block(P, hv, b.x + e / (R * R), b.y + (e / R) % R, b.z + e % R);
}

__global__ void k_zero_grid(float4* __restrict__ gmv, float4* __restrict__ gf, int64_t nn, const DevStatus* st) {
    if (cta_aborted(st)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        gmv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        gf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Sort key (Phi, cell) and value (storage index).  With by_id the pair is
// written at the particle's id so that the stable sort breaks ties by id.
template <bool DENSE>
__global__ void k_particle_keys(const float* __restrict__ ps, int64_t stride, int64_t n,
                                const uint32_t* __restrict__ pcode, HashView hv, int B3,
                                int by_id, uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                                DevStatus* st) {
    if (cta_aborted(st)) return;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t code = pcode[p];
    uint32_t k;
    if (DENSE) {
        k = code;
    } else {
        const uint32_t q = code / (uint32_t)B3;   // table slot, or the block's relative key in scan mode
        const int r = code == 0xffffffffu ? -1 : (hv.bits ? mask_rank(hv, q) : hv.vals[q]);
        if (r < 0) {
            raise_flag(st, &st->map_miss, 1u);
            k = 0xffffffffu;   // sorts last; k_ranges ignores it
        } else {
            k = (uint32_t)r * (uint32_t)B3 + code % (uint32_t)B3;
        }
    }
    const int64_t q = by_id ? (int64_t)__float_as_uint(ps[pel(p, PID)]) : p;
    key[q] = k;
    val[q] = (uint32_t)p;
}

__global__ void k_ranges(const uint32_t* __restrict__ skey, int64_t n, int shift, int64_t cap,
                         int* __restrict__ bstart, int* __restrict__ bend, int* __restrict__ pblocks,
                         int* __restrict__ hasp, DevStatus* st) {
    if (cta_aborted(st)) return;
    const int64_t nblocks = live_blocks(st, cap);
    const int gen = (int)st->gen;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t r = skey[i] >> shift;
    if ((int64_t)r >= nblocks) {
        raise_flag(st, &st->map_miss, 1u);
        return;
    }
    const bool first = (i == 0) || ((skey[i - 1] >> shift) != r);
    const bool last = (i == n - 1) || ((skey[i + 1] >> shift) != r);
    if (first) {
        bstart[r] = (int)i;
        hasp[r] = gen;
        pblocks[atomicAdd(&st->n_pblocks, 1u)] = (int)r;
    }
    if (last) bend[r] = (int)(i + 1);
}

__device__ __forceinline__ int first_geq(const uint32_t* __restrict__ skey, int lo, int hi, uint32_t q) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (skey[mid] < q) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Slots of a block's 64 cells ordered by particle count, largest first (ties
// by cell index): slot of cell c = the cells with more particles, or as many
// and a smaller index, a permutation of 0..63.  Counts are compared clamped
// to 63, which only reorders cells fuller than that.  Lane l holds the counts
// of cells l and l + 32 and gets their slots q0, q1, and in more0, more1 the
// number of cells holding more than l and l + 32 particles (exact below 63);
// hall and hlow are 64-int scratch arrays of the calling warp.  Every lane of
// the warp calls it.
__device__ __forceinline__ void count_order_slots(int cnt0, int cnt1, int lane, int* hall, int* hlow, int& q0,
                                                  int& q1, int& more0, int& more1) {
    const unsigned FULL = 0xffffffffu;
    const int v0 = min(cnt0, 63), v1 = min(cnt1, 63);
    hall[lane] = hall[lane + 32] = 0;
    hlow[lane] = hlow[lane + 32] = 0;
    __syncwarp();
    atomicAdd(&hall[v0], 1);
    atomicAdd(&hall[v1], 1);
    atomicAdd(&hlow[v0], 1);   // cells 0-31 only
    __syncwarp();
    // more[v] = cells with a clamped count above v (a suffix sum)
    const int h0 = hall[lane], h1 = hall[lane + 32];
    int s1 = h1, s0 = h0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {   // inclusive suffix sums inside each half
        const int t1 = __shfl_down_sync(FULL, s1, o), t0 = __shfl_down_sync(FULL, s0, o);
        if (lane + o < 32) {
            s1 += t1;
            s0 += t0;
        }
    }
    s0 += __shfl_sync(FULL, s1, 0);   // the upper half lies above every lower value
    more0 = s0 - h0;   // for values lane and lane + 32
    more1 = s1 - h1;
    const int m0a = __shfl_sync(FULL, more0, v0 & 31), m0b = __shfl_sync(FULL, more1, v0 & 31);
    const int m1a = __shfl_sync(FULL, more0, v1 & 31), m1b = __shfl_sync(FULL, more1, v1 & 31);
    const unsigned below = (1u << lane) - 1u;
    q0 = (v0 < 32 ? m0a : m0b) + __popc(__match_any_sync(FULL, v0) & below);
    q1 = (v1 < 32 ? m1a : m1b) + hlow[v1] + __popc(__match_any_sync(FULL, v1) & below);
}

// Reorders every block's particles from (cell, k) to k-major order: the
// k-th particle of each cell (cells in slot order) before any (k+1)-th one,
// and records the particle count per slot.  One warp per block; lane l
// handles slots l and l + 32.  Without `cperm` slot j is cell j.  With it
// (the fast mode) the slots hold the block's cells by particle count,
// largest first (ties by cell index), and cperm records the cell of every
// slot: P2G's two work units of a block are slots 0-31 and 32-63, and a unit
// takes as many rounds as its fullest cell, so the heavy cells share a unit.
// Output goes to the spare sort buffers.
__global__ void __launch_bounds__(128) k_interleave(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ perm,
                                                    const int* __restrict__ bstart, const int* __restrict__ bend,
                                                    const int* __restrict__ pblocks, const DevStatus* stc,
                                                    const int* __restrict__ cs, const int* __restrict__ tsum,
                                                    int ntiles, int64_t cap, const float* __restrict__ ps,
                                                    int64_t pstride, uint32_t* __restrict__ byid,
                                                    uint32_t* __restrict__ skey2, uint32_t* __restrict__ perm2,
                                                    int* __restrict__ ccount, uint8_t* __restrict__ cperm) {
    __shared__ unsigned char slot_cell[4][64];
    __shared__ int hist_all[4][64], hist_low[4][64];
    if (cta_aborted(stc)) return;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * 4 + (threadIdx.x >> 5), nw = gridDim.x * 4;
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    const int nblk = (int)stc->n_pblocks;
    for (int kb = gw; kb < nblk; kb += nw) {
        const int r = pblocks[kb];
        const int s = bstart[r], e = bend[r];
        const uint32_t base = (uint32_t)r * 64u;
        int lo0, hi0, lo1, hi1;
        if (cs) {   // cell starts known from the counting sort
            const int64_t n = live_blocks(stc, cap) * 64;
            lo0 = scan_at(cs, tsum, base + lane, n, ntiles);
            hi0 = scan_at(cs, tsum, base + lane + 1, n, ntiles);
            lo1 = scan_at(cs, tsum, base + 32 + lane, n, ntiles);
            hi1 = scan_at(cs, tsum, base + 33 + lane, n, ntiles);
        } else {
            lo0 = first_geq(skey, s, e, base + lane);
            hi0 = first_geq(skey, lo0, e, base + lane + 1);
            lo1 = first_geq(skey, s, e, base + 32 + lane);
            hi1 = first_geq(skey, lo1, e, base + 33 + lane);
        }
        int cnt0 = hi0 - lo0, cnt1 = hi1 - lo1;
        int cell0 = lane, cell1 = lane + 32;
        if (cperm) {
            const int w = threadIdx.x >> 5;
            int q0, q1, more0, more1;
            count_order_slots(cnt0, cnt1, lane, hist_all[w], hist_low[w], q0, q1, more0, more1);
            unsigned char* sc = slot_cell[w];
            sc[q0] = (unsigned char)lane;
            sc[q1] = (unsigned char)(lane + 32);
            __syncwarp();
            cell0 = sc[lane];
            cell1 = sc[lane + 32];
            __syncwarp();   // the slots are read before the next block rewrites them
            // range of the cells now in slots lane and lane + 32 (cell c's range
            // sits in lane c & 31, in its first pair for c < 32)
            const int l0a = __shfl_sync(FULL, lo0, cell0 & 31), l0b = __shfl_sync(FULL, lo1, cell0 & 31);
            const int c0a = __shfl_sync(FULL, cnt0, cell0 & 31), c0b = __shfl_sync(FULL, cnt1, cell0 & 31);
            const int l1a = __shfl_sync(FULL, lo0, cell1 & 31), l1b = __shfl_sync(FULL, lo1, cell1 & 31);
            const int c1a = __shfl_sync(FULL, cnt0, cell1 & 31), c1b = __shfl_sync(FULL, cnt1, cell1 & 31);
            lo0 = cell0 < 32 ? l0a : l0b;
            lo1 = cell1 < 32 ? l1a : l1b;
            cnt0 = cell0 < 32 ? c0a : c0b;
            cnt1 = cell1 < 32 ? c1a : c1b;
            cperm[(int64_t)r * 64 + lane] = (uint8_t)cell0;
            cperm[(int64_t)r * 64 + 32 + lane] = (uint8_t)cell1;
        }
        ccount[(int64_t)r * 64 + lane] = cnt0;
        ccount[(int64_t)r * 64 + 32 + lane] = cnt1;
        // Deterministic mode on the counting sort (ps given): the counting
        // sort leaves a cell's particles in arrival order, so each lane puts
        // its two cells' particles in id order first: particle j goes to slot
        // lo + (number of the cell's particles with a smaller id) of byid.
        const uint32_t* src = perm;
        if (ps) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int lo = h ? lo1 : lo0, cnt = h ? cnt1 : cnt0;
                for (int j = 0; j < cnt; ++j) {
                    const uint32_t pj = perm[lo + j];
                    const uint32_t idj = __float_as_uint(ps[pel(pj, PID)]);
                    int rank = 0;
                    for (int i = 0; i < cnt; ++i)
                        rank += __float_as_uint(ps[pel(perm[lo + i], PID)]) < idj ? 1 : 0;
                    byid[lo + rank] = pj;
                }
            }
            src = byid;   // each lane reads back only its own cells' slots
        }
        int off = 0;
        for (int k = 0; k <= e - s; ++k) {   // no cell holds more than the block's particles
            const unsigned M0 = __ballot_sync(FULL, cnt0 > k), M1 = __ballot_sync(FULL, cnt1 > k);
            if ((M0 | M1) == 0u) break;
            if (cnt0 > k) {
                const int pos = s + off + __popc(M0 & lt);
                perm2[pos] = src[lo0 + k];
                skey2[pos] = base + cell0;
            }
            if (cnt1 > k) {
                const int pos = s + off + __popc(M0) + __popc(M1 & lt);
                perm2[pos] = src[lo1 + k];
                skey2[pos] = base + cell1;
            }
            off += __popc(M0) + __popc(M1);
        }
    }
}

// ------------------------------------------------ counting sort (fast mode)

// Sort key per particle and its rank among the particles of its (block, cell)
// bin: lanes of a warp with the same key take consecutive ranks from one
// atomic add by their leader.  Each warp takes 32 x BIN_PL consecutive
// particles, BIN_PL per lane, so that as many chains of dependent loads are in
// flight per lane.
__device__ __forceinline__ uint32_t bin_key(int64_t p, int64_t n, uint32_t code, const HashView& hv, int B3,
                                            DevStatus* st, bool& miss) {
    if (p >= n) return 0xffffffffu;
    const uint32_t q = code / (uint32_t)B3;
    if (code != 0xffffffffu && !hv.bits && !index_ok(q, (int64_t)hv.mask + 1, st)) return 0xffffffffu;
    const int r = code == 0xffffffffu ? -1 : (hv.bits ? mask_rank(hv, q) : hv.vals[q]);
    if (r < 0) {
        miss = true;   // raised by the caller once both keys are known
        return 0xffffffffu;
    }
    return (uint32_t)r * (uint32_t)B3 + code % (uint32_t)B3;
}

__device__ __forceinline__ void bin_rank(int64_t p, int64_t n, uint32_t k, int lane, int* __restrict__ bins,
                                         uint32_t* __restrict__ key, uint32_t* __restrict__ prank) {
    const unsigned FULL = 0xffffffffu;
    const unsigned peers = __match_any_sync(FULL, k);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (k != 0xffffffffu && lane == leader) base = atomicAdd(&bins[k], __popc(peers));
    base = __shfl_sync(FULL, base, leader);
    if (p < n) {
        key[p] = k;
        prank[p] = (uint32_t)(base + __popc(peers & ((1u << lane) - 1u)));
    }
}

// The 256 x BIN_PL particles of a CTA are consecutive in the previous step's
// sorted order, so their keys usually span a few blocks' bins: when the span
// fits BIN_SPAN, the CTA counts them in shared memory and adds one total per
// distinct bin to the global counts (a particle's rank = the bin's global
// base + its shared-memory rank); otherwise every particle takes the
// warp-aggregated global path.  Four particles per lane: 0.4% off the 8M
// landslide's step against two (eight: 2% slower).
constexpr int BIN_SPAN = 2048;

#ifndef MPM_BINS_PER_LANE
#define MPM_BINS_PER_LANE 4
#endif
constexpr int BIN_PL = MPM_BINS_PER_LANE;   // particles per lane in the binning

__global__ void __launch_bounds__(256) k_particle_bins(int64_t n, const uint32_t* __restrict__ pcode,
                                                       HashView hv, int B3, int* __restrict__ bins,
                                                       uint32_t* __restrict__ key, uint32_t* __restrict__ prank,
                                                       DevStatus* st) {
    __shared__ int hist[BIN_SPAN];
    __shared__ uint32_t wmin[8], wmax[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * BIN_PL + lane;
    uint32_t code[BIN_PL];
#pragma unroll
    for (int h = 0; h < BIN_PL; ++h) {   // read before the abort test: in bounds, and it overlaps them
        const int64_t p = p0 + 32 * h;
        code[h] = p < n ? pcode[p] : 0xffffffffu;
    }
    if (cta_aborted(st)) return;
    bool miss = false;
    uint32_t k[BIN_PL];
#pragma unroll
    for (int h = 0; h < BIN_PL; ++h) k[h] = bin_key(p0 + 32 * h, n, code[h], hv, B3, st, miss);
    if (miss) raise_flag(st, &st->map_miss, 1u);
    // key range of the CTA's valid keys (invalid keys are all ones)
    uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
    for (int h = 0; h < BIN_PL; ++h) {
        lo = min(lo, k[h]);
        hi = max(hi, k[h] == 0xffffffffu ? 0u : k[h]);
    }
    const uint32_t wl = __reduce_min_sync(0xffffffffu, lo), wh = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
        wmin[w] = wl;
        wmax[w] = wh;
    }
    for (int i = threadIdx.x; i < BIN_SPAN; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        kmin = min(kmin, wmin[i]);
        kmax = max(kmax, wmax[i]);
    }
    if (kmin == 0xffffffffu) {       // no valid key in this CTA
#pragma unroll
        for (int h = 0; h < BIN_PL; ++h)
            if (p0 + 32 * h < n) key[p0 + 32 * h] = 0xffffffffu;
        return;
    }
    if (kmax - kmin >= (uint32_t)BIN_SPAN) {   // CTA-uniform: the global path
#pragma unroll
        for (int h = 0; h < BIN_PL; ++h) bin_rank(p0 + 32 * h, n, k[h], lane, bins, key, prank);
        return;
    }
    int rl[BIN_PL];
#pragma unroll
    for (int h = 0; h < BIN_PL; ++h) rl[h] = k[h] != 0xffffffffu ? atomicAdd(&hist[k[h] - kmin], 1) : 0;
    __syncthreads();
    const int span = (int)(kmax - kmin) + 1;
    for (int i = threadIdx.x; i < span; i += blockDim.x) {
        const int c = hist[i];
        if (c > 0) hist[i] = atomicAdd(&bins[kmin + i], c);   // the bin's global base for this CTA
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < BIN_PL; ++h) {
        const int64_t p = p0 + 32 * h;
        if (p >= n) continue;
        key[p] = k[h];
        if (k[h] != 0xffffffffu) prank[p] = (uint32_t)(hist[k[h] - kmin] + rl[h]);
    }
}


// The end of a tile scan: every CTA has written its tile total to tsum; the
// last CTA to arrive (counted on `counter`, which it resets) turns the
// totals into exclusive tile offsets and writes the grand total to
// tsum[ntiles].  Every thread of every CTA calls it.
__device__ __forceinline__ void finish_tile_sums(int* __restrict__ tsum, int ntiles, unsigned int* counter) {
    __shared__ int wsum[SC_THREADS / 32];
    __shared__ int carry;
    __shared__ bool last;
    __threadfence();   // this CTA's total is visible device-wide before the CTA counts in
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < ntiles; b += SC_THREADS) {
        const int i = b + threadIdx.x;
        const int v = i < ntiles ? __ldcg(&tsum[i]) : 0;   // other CTAs' totals: from L2
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        int pre = 0;
        for (int k = 0; k < w; ++k) pre += wsum[k];
        const int excl = carry + pre + x - v;
        __syncthreads();
        if (i < ntiles) tsum[i] = excl;
        if (threadIdx.x == SC_THREADS - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tsum[ntiles] = carry;
        *counter = 0u;
    }
}

// Exclusive scan of the live bins (live blocks x B3; the grid covers the
// capacity): each tile of 2048 bins scanned locally, tile totals (zero for
// tiles past the live bins) turned into tile offsets by the last CTA.  A
// bin's start is scan_at(cs, tsum, ...).
__global__ void __launch_bounds__(SC_THREADS) k_scan_tiles(const int* __restrict__ in, int64_t cap, int B3,
                                                           DevStatus* st, int* __restrict__ out,
                                                           int* __restrict__ tsum) {
    __shared__ int wsum[SC_THREADS / 32];
    if (cta_aborted(st)) return;
    const int64_t n = live_blocks(st, cap) * B3;
    if ((int64_t)blockIdx.x * SC_TILE >= n) {
        if (threadIdx.x == 0) tsum[blockIdx.x] = 0;
        finish_tile_sums(tsum, (int)gridDim.x, &st->scan_done[1]);
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS];
    int tot = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        v[j] = base + j < n ? in[base + j] : 0;
        tot += v[j];
    }
    int x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int pre = 0;
    for (int k = 0; k < w; ++k) pre += wsum[k];
    int run = pre + x - tot;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == SC_THREADS - 1) tsum[blockIdx.x] = pre + x;
    finish_tile_sums(tsum, (int)gridDim.x, &st->scan_done[1]);
}

// Exclusive scan of the bit counts of the block mask's words, steps 1 and 2
// (step 3, k_scan_add_n, only where lookups read the scan: scan mode).
__global__ void __launch_bounds__(SC_THREADS) k_bits_scan_tiles(const uint32_t* __restrict__ bmask, int64_t n,
                                                                DevStatus* st, int* __restrict__ out,
                                                                int* __restrict__ tsum) {
    __shared__ int wsum[SC_THREADS / 32];
    if (cta_aborted(st)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS];
    int tot = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        v[j] = base + j < n ? __popc(bmask[base + j]) : 0;
        tot += v[j];
    }
    int x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int pre = 0;
    for (int k = 0; k < w; ++k) pre += wsum[k];
    int run = pre + x - tot;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == SC_THREADS - 1) tsum[blockIdx.x] = pre + x;
    finish_tile_sums(tsum, (int)gridDim.x, &st->scan_done[0]);
}

// Step 3 for a fixed count n: add the tile offsets; cs[n] = total.
__global__ void k_scan_add_n(int* __restrict__ cs, int64_t n, const DevStatus* st, const int* __restrict__ tsum,
                             int ntiles) {
    if (cta_aborted(st)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cs[i] += tsum[i / SC_TILE];
    if (i == n) cs[n] = tsum[ntiles];
}

#ifndef MPM_SCATTER_PER_LANE
#define MPM_SCATTER_PER_LANE 2
#endif
constexpr int SCT_PL = MPM_SCATTER_PER_LANE;   // particles per lane in the scatter

// Scatter into (block, cell) order, SCT_PL particles per lane (p, p + 32,
// ... within the warp's 32 x SCT_PL) for as many load chains in flight.
__global__ void __launch_bounds__(256) k_bin_scatter(int64_t n, const uint32_t* __restrict__ key,
                                                     const uint32_t* __restrict__ prank, const int* __restrict__ cs,
                                                     const int* __restrict__ tsum, uint32_t* __restrict__ skey,
                                                     uint32_t* __restrict__ perm, DevStatus* st) {
    if (cta_aborted(st)) return;
    const int lane = threadIdx.x & 31;
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * SCT_PL + lane;
    uint32_t k[SCT_PL], r[SCT_PL];
#pragma unroll
    for (int h = 0; h < SCT_PL; ++h) {
        const int64_t p = p0 + 32 * h;
        k[h] = 0xffffffffu;
        r[h] = 0u;
        if (p < n) {
            k[h] = key[p];
            r[h] = prank[p];
        }
    }
#pragma unroll
    for (int h = 0; h < SCT_PL; ++h) {
        if (k[h] == 0xffffffffu) continue;
        const int pos = cs[k[h]] + tsum[k[h] / SC_TILE] + (int)r[h];   // a particle's bin is live
        if (!index_ok(pos, n, st)) continue;
        skey[pos] = k[h];
        perm[pos] = (uint32_t)(p0 + 32 * h);
    }
}

// Counting-sort mode: the neighbour table of every active block (as
// k_neighbours: thread t looks up neighbour t % NNB of block t / NNB), and,
// in the thread of neighbour 0, the block's particle range and flag from its
// cell starts.
template <int B>
__global__ void k_block_ranges(int64_t cap, int B3, const int* __restrict__ cs, const int* __restrict__ tsum,
                               int ntiles, int* __restrict__ bstart, int* __restrict__ bend,
                               int* __restrict__ pblocks, int* __restrict__ hasp, DevStatus* st,
                               const int4* __restrict__ bcoord, Params P, HashView hv, int* __restrict__ nbr) {
    constexpr int R = (B == 4) ? 2 : 3;
    constexpr int NNB = R * R * R;
    if (cta_aborted(st)) return;
    const int64_t nact = live_blocks(st, cap);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nact * NNB) return;
    const int64_t r = t / NNB;
    const int e = (int)(t % NNB);
    const int4 b = bcoord[r];
    nbr[t] = lookup_block(P, hv, b.x + e / (R * R), b.y + (e / R) % R, b.z + e % R);
    if (e != 0) return;
    const int64_t n = nact * B3;
    const int s = scan_at(cs, tsum, r * B3, n, ntiles), en = scan_at(cs, tsum, r * B3 + B3, n, ntiles);
    if (en > s) {
        bstart[r] = s;
        bend[r] = en;
        hasp[r] = (int)st->gen;
        pblocks[atomicAdd(&st->n_pblocks, 1u)] = (int)r;
    }
}

// ------------------------------- k-major scatter (fast sparse mode, B = 4)
//
// With a block's slots ordered by count, largest first, the cells that still
// hold a particle in round k are exactly slots 0 .. n_k - 1 (n_k = cells with
// more than k particles).  So the k-major position of the particle of rank k
// in the cell of slot s is fixed by the counts alone:
//     block start + sum_c min(count_c, k) + s,
// and the counting sort can scatter particles straight to it, with no
// cell-major pass in between.

// One warp per active block (one warp per block of the capacity, grid-stride
// beyond it): the block's particle range and
// the "holds particles" mark, its neighbour table, the count order of its
// cells (cperm: slot -> cell, cslot: cell -> slot, ccount per slot) and the
// round prefixes kpre[k] = sum_c min(count_c, k) for k < 64.
__global__ void __launch_bounds__(128) k_block_prep(int64_t cap, const int* __restrict__ cs,
                                                    const int* __restrict__ tsum, int ntiles, int* __restrict__ bstart,
                                                    int* __restrict__ bend, int* __restrict__ pblocks,
                                                    int* __restrict__ hasp, DevStatus* st,
                                                    const int4* __restrict__ bcoord, Params P, HashView hv,
                                                    int* __restrict__ nbr, int* __restrict__ ccount,
                                                    uint8_t* __restrict__ cperm, uint8_t* __restrict__ cslot,
                                                    int* __restrict__ kpre) {
    __shared__ int hist_all[4][64], hist_low[4][64];
    if (cta_aborted(st)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = blockIdx.x * 4 + w, nw = gridDim.x * 4;
    const unsigned FULL = 0xffffffffu;
    const int64_t nact = live_blocks(st, cap);
    const int64_t n = nact * 64;
    const int gen = (int)st->gen;
    for (int64_t r = gw; r < nact; r += nw) {
        if (lane < 8) {
            const int4 b = bcoord[r];
            nbr[r * 8 + lane] = lookup_block(P, hv, b.x + (lane >> 2), b.y + ((lane >> 1) & 1), b.z + (lane & 1));
        }
        const int64_t base = r * 64;
        const int lo0 = scan_at(cs, tsum, base + lane, n, ntiles), hi0 = scan_at(cs, tsum, base + lane + 1, n, ntiles);
        const int lo1 = scan_at(cs, tsum, base + 32 + lane, n, ntiles);
        const int hi1 = scan_at(cs, tsum, base + 33 + lane, n, ntiles);
        const int cnt0 = hi0 - lo0, cnt1 = hi1 - lo1;
        const int s = __shfl_sync(FULL, lo0, 0), e = __shfl_sync(FULL, hi1, 31);
        if (e <= s) continue;   // warp-uniform: no particle in this block
        if (lane == 0) {
            bstart[r] = s;
            bend[r] = e;
            hasp[r] = gen;
            pblocks[atomicAdd(&st->n_pblocks, 1u)] = (int)r;
        }
        int q0, q1, n0, n1;
        count_order_slots(cnt0, cnt1, lane, hist_all[w], hist_low[w], q0, q1, n0, n1);
        cslot[base + lane] = (uint8_t)q0;
        cslot[base + 32 + lane] = (uint8_t)q1;
        cperm[base + q0] = (uint8_t)lane;
        cperm[base + q1] = (uint8_t)(lane + 32);
        ccount[base + q0] = cnt0;
        ccount[base + q1] = cnt1;
        // kpre[k] = sum_c min(count_c, k) = sum over k' < k of the cells
        // holding more than k' particles (n0, n1 for k' = lane, lane + 32):
        // an exclusive scan over k = 0..63
        int i0 = n0, i1 = n1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {   // inclusive scans inside each half
            const int t0 = __shfl_up_sync(FULL, i0, o), t1 = __shfl_up_sync(FULL, i1, o);
            if (lane >= o) {
                i0 += t0;
                i1 += t1;
            }
        }
        i1 += __shfl_sync(FULL, i0, 31);
        kpre[base + lane] = i0 - n0;
        kpre[base + 32 + lane] = i1 - n1;
    }
}

// Per particle (two per lane): its k-major position from its (block, cell)
// key and its rank in the cell, then the sort key and permutation there.  A
// rank of 64 or more (a cell that full) sums the block's 64 slot counts.
__global__ void __launch_bounds__(256) k_scatter_kmajor(int64_t n, const uint32_t* __restrict__ key,
                                                        const uint32_t* __restrict__ prank,
                                                        const int* __restrict__ bstart,
                                                        const uint8_t* __restrict__ cslot,
                                                        const int* __restrict__ kpre, const int* __restrict__ ccount,
                                                        uint32_t* __restrict__ skey, uint32_t* __restrict__ perm,
                                                        DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * SCT_PL + lane;
    uint32_t k[SCT_PL], rk[SCT_PL];
#pragma unroll
    for (int h = 0; h < SCT_PL; ++h) {   // read before the abort test: in bounds, and it overlaps them
        const int64_t p = p0 + 32 * h;
        k[h] = 0xffffffffu;
        rk[h] = 0u;
        if (p < n) {
            k[h] = key[p];
            rk[h] = prank[p];
        }
    }
    if (cta_aborted(st)) return;
#pragma unroll
    for (int h = 0; h < SCT_PL; ++h) {
        if (k[h] == 0xffffffffu) continue;
        const int64_t r = k[h] >> 6;
        int pre;
        if (rk[h] < 64u) {
            pre = kpre[r * 64 + rk[h]];
        } else {
            pre = 0;
            for (int j = 0; j < 64; ++j) pre += min(ccount[r * 64 + j], (int)rk[h]);
        }
        const int pos = bstart[r] + pre + (int)cslot[k[h]];
        if (!index_ok(pos, n, st)) continue;
        skey[pos] = k[h];
        perm[pos] = (uint32_t)(p0 + 32 * h);
    }
}


inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
}  // namespace

// Every launch below goes to c->ls and takes its sizes from capacities
// (c->n, c->H, c->live_cap); live counts come from the status words, so the
// same launch sequence serves any step and can be captured in a graph.

HashView hash_view(const mpm_ctx* c) {
    HashView hv{c->hkeys, c->hvals, (uint64_t)(c->H ? c->H - 1 : 0)};
    if (c->scan) {
        hv.bits = c->bmask;
        hv.pre = c->bpre;
    }
    return hv;
}

cudaError_t launch_insert(mpm_ctx* c, int64_t ins_cap) {
    const HashView hv = hash_view(c);
    const unsigned gc = (unsigned)std::min<int64_t>(blocks_for(std::max<int64_t>(c->H, c->bwords), 256), 148 * 16);
    k_hash_clear<<<gc, 256, 0, c->ls>>>(c->hkeys, c->hvals, c->H, c->bmask, c->bwords, c->dstat);
    c->launches += 2;
    const float* ps = c->ps[c->cur];
#define MPM_INS(B_, S_)                                                                                           \
    k_insert<B_, S_><<<blocks_for(c->n, 256 * INS_PL), 256, 0, c->ls>>>(ps, c->pstride, c->n, c->P, hv, c->akey[0],       \
                                                               c->aslot[0], ins_cap, c->bmask, c->pcode, c->dstat)
    if (c->B == 4) {
        if (c->scan) MPM_INS(4, true);
        else MPM_INS(4, false);
    } else {
        if (c->scan) MPM_INS(1, true);
        else MPM_INS(1, false);
    }
#undef MPM_INS
    if (c->scan) {   // Alg. 3: the scan of the marks gives the block count before the host reads it
        const int ntiles = (int)((c->bwords + SC_TILE - 1) / SC_TILE);
        k_bits_scan_tiles<<<ntiles, SC_THREADS, 0, c->ls>>>(c->bmask, c->bwords, c->dstat, c->bpre, c->btsum);
        k_scan_add_n<<<blocks_for(c->bwords + 1, 256), 256, 0, c->ls>>>(c->bpre, c->bwords, c->dstat, c->btsum, ntiles);
        k_scan_count<<<1, 1, 0, c->ls>>>(c->bpre, c->bwords, ins_cap, c->dstat);
        c->launches += 3;
    }
    return cudaGetLastError();
}

cudaError_t launch_dense_codes(mpm_ctx* c) {
    k_status_clear<<<1, 1, 0, c->ls>>>(c->dstat, (unsigned)c->n_dom_blocks);
    c->launches += 2;
    const float* ps = c->ps[c->cur];
    if (c->B == 4)
        k_dense_codes<4><<<blocks_for(c->n, 256), 256, 0, c->ls>>>(ps, c->pstride, c->n, c->P, c->pcode, c->dstat);
    else
        k_dense_codes<1><<<blocks_for(c->n, 256), 256, 0, c->ls>>>(ps, c->pstride, c->n, c->P, c->pcode, c->dstat);
    return cudaGetLastError();
}

cudaError_t launch_assign(mpm_ctx* c) {
    const int zero = c->det ? 0 : 1;
    const int64_t cap = c->live_cap;
    if (c->dense) {
        if (zero) {
            k_zero_grid<<<148 * 8, 256, 0, c->ls>>>(c->gmv, c->gf, c->n_dom_blocks * c->B3, c->dstat);
            ++c->launches;
        }
        return cudaGetLastError();
    }
    int* bins = counting_sort(c) ? c->bins : nullptr;
    if (c->scan) {   // Alg. 4: block coordinates per Phi from the scanned marks
        const unsigned g = (unsigned)std::min<int64_t>(blocks_for(std::max<int64_t>(c->bwords, cap * c->B3), 256),
                                                       148 * 16);
        k_assign_scan<<<g, 256, 0, c->ls>>>(c->bmask, c->bpre, c->bwords, cap, c->dstat, c->P, c->bcoord, c->gmv, c->gf,
                                            bins, c->B3, zero);
        ++c->launches;
    } else if (c->bmask) {
        const int ntiles = (int)((c->bwords + SC_TILE - 1) / SC_TILE);
        k_bits_scan_tiles<<<ntiles, SC_THREADS, 0, c->ls>>>(c->bmask, c->bwords, c->dstat, c->bpre, c->btsum);
        k_assign_bits<<<blocks_for(cap * c->B3, 256), 256, 0, c->ls>>>(c->akey[0], c->aslot[0], cap, c->dstat, c->P,
                                                                       c->bmask, c->bpre, c->btsum, c->hvals,
                                                                       c->bcoord, c->gmv, c->gf, bins, c->B3, zero);
        c->launches += 2;
    } else {
        const int bits = 64 - __builtin_clzll((unsigned long long)(c->n_dom_blocks > 1 ? c->n_dom_blocks - 1 : 1));
        int sel = radix_sort_pairs(c, c->akey, c->aslot, cap, &c->dstat->n_active, bits, c->ls, &c->dstat->abort);
        k_assign<<<blocks_for(cap * c->B3, 256), 256, 0, c->ls>>>(c->akey[sel], c->aslot[sel], cap, c->dstat, c->P,
                                                                  c->hvals, c->bcoord, c->gmv, c->gf, bins, c->B3,
                                                                  zero);
        ++c->launches;
    }
    if (counting_sort(c)) return cudaGetLastError();   // the neighbour table comes with the block ranges
    const HashView hv = hash_view(c);
    const int nnb = c->B == 4 ? 8 : 27;
    if (c->B == 4)
        k_neighbours<4><<<blocks_for(cap * nnb, 256), 256, 0, c->ls>>>(c->bcoord, cap, c->dstat, c->P, hv, c->nbr);
    else
        k_neighbours<1><<<blocks_for(cap * nnb, 256), 256, 0, c->ls>>>(c->bcoord, cap, c->dstat, c->P, hv, c->nbr);
    ++c->launches;
    return cudaGetLastError();
}

// The sparse grid sorts particles by counting sort, in deterministic mode too:
// the interleave then puts each cell's particles in id order, so the order
// is (block, cell, id) as the dense grid's radix sort by (key, id) gives.
bool counting_sort(const mpm_ctx* c) { return !c->dense; }

// The fast sparse mode at B = 4 scatters particles straight to their k-major
// positions (k_block_prep, k_scatter_kmajor); the deterministic mode keeps
// the cell-major scatter and the interleave, which puts each cell's
// particles in id order.
static bool kmajor_scatter(const mpm_ctx* c) { return counting_sort(c) && !c->det && c->B == 4; }

cudaError_t launch_particle_keys(mpm_ctx* c) {
    const float* ps = c->ps[c->cur];
    const int64_t cap = c->live_cap;
    const int64_t nkeys = cap * c->B3;
    if (counting_sort(c)) {
        // one pass: key + rank in bin; scan of the bins; scatter
        k_particle_bins<<<blocks_for(c->n, 256 * BIN_PL), 256, 0, c->ls>>>(c->n, c->pcode, hash_view(c), c->B3, c->bins, c->pkey[0],
                                                                  c->prank, c->dstat);
        const int ntiles = (int)((nkeys + SC_TILE - 1) / SC_TILE);
        k_scan_tiles<<<ntiles, SC_THREADS, 0, c->ls>>>(c->bins, cap, c->B3, c->dstat, c->cs, c->tsum);
        c->launches += 2;
        if (kmajor_scatter(c)) return cudaGetLastError();   // launch_ranges scatters
        k_bin_scatter<<<blocks_for(c->n, 256 * SCT_PL), 256, 0, c->ls>>>(c->n, c->pkey[0], c->prank, c->cs, c->tsum,
                                                                         c->pkey[1], c->pval[1], c->dstat);
        ++c->launches;
        c->sorted_sel = 1;
        return cudaGetLastError();
    }
    const int by_id = c->det ? 1 : 0;
    if (c->dense)
        k_particle_keys<true><<<blocks_for(c->n, 256), 256, 0, c->ls>>>(ps, c->pstride, c->n, c->pcode, hash_view(c), c->B3,
                                                                       by_id, c->pkey[0], c->pval[0], c->dstat);
    else
        k_particle_keys<false><<<blocks_for(c->n, 256), 256, 0, c->ls>>>(ps, c->pstride, c->n, c->pcode, hash_view(c), c->B3,
                                                                        by_id, c->pkey[0], c->pval[0], c->dstat);
    ++c->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int bits = 64 - __builtin_clzll((unsigned long long)(nkeys > 1 ? nkeys - 1 : 1));
    c->sorted_sel = radix_sort_pairs(c, c->pkey, c->pval, c->n, nullptr, bits, c->ls, &c->dstat->abort);
    return cudaGetLastError();
}

cudaError_t launch_ranges(mpm_ctx* c, const uint32_t* skey) {
    const bool cnt = counting_sort(c);
    const int64_t cap = c->live_cap;
    const int ntiles = (int)((cap * c->B3 + SC_TILE - 1) / SC_TILE);   // the bin scan's tiles
    if (kmajor_scatter(c)) {
        k_block_prep<<<blocks_for(cap, 4), 128, 0, c->ls>>>(cap, c->cs, c->tsum, ntiles, c->bstart, c->bend, c->pblocks, c->hasp,
                                                 c->dstat, c->bcoord, c->P, hash_view(c), c->nbr, c->ccount, c->cperm,
                                                 c->cslot, c->kpre);
        k_scatter_kmajor<<<blocks_for(c->n, 256 * SCT_PL), 256, 0, c->ls>>>(c->n, c->pkey[0], c->prank, c->bstart,
                                                                            c->cslot, c->kpre, c->ccount, c->pkey[1],
                                                                            c->pval[1], c->dstat);
        c->launches += 2;
        c->sorted_sel = 1;
        return cudaGetLastError();
    }
    if (cnt) {
        const HashView hv = hash_view(c);
        if (c->B == 4)
            k_block_ranges<4><<<blocks_for(cap * 8, 256), 256, 0, c->ls>>>(
                cap, c->B3, c->cs, c->tsum, ntiles, c->bstart, c->bend, c->pblocks, c->hasp, c->dstat, c->bcoord, c->P,
                hv, c->nbr);
        else
            k_block_ranges<1><<<blocks_for(cap * 27, 256), 256, 0, c->ls>>>(
                cap, c->B3, c->cs, c->tsum, ntiles, c->bstart, c->bend, c->pblocks, c->hasp, c->dstat, c->bcoord, c->P,
                hv, c->nbr);
    } else {
        const int shift = (c->B == 4) ? 6 : 0;
        k_ranges<<<blocks_for(c->n, 256), 256, 0, c->ls>>>(skey, c->n, shift, cap, c->bstart, c->bend, c->pblocks,
                                                           c->hasp, c->dstat);
    }
    ++c->launches;
    if (c->B == 4) {
        const int o = 1 - c->sorted_sel;
        const bool by_id = cnt && c->det;   // deterministic mode: id order inside every cell
        k_interleave<<<148 * 8, 128, 0, c->ls>>>(skey, c->pval[c->sorted_sel], c->bstart, c->bend, c->pblocks, c->dstat,
                                                cnt ? c->cs : nullptr, c->tsum, ntiles, cap,
                                                by_id ? c->ps[c->cur] : nullptr, c->pstride, c->prank, c->pkey[o],
                                                c->pval[o], c->ccount, (cnt && !c->det) ? c->cperm : nullptr);
        c->sorted_sel = o;
        ++c->launches;
    }
    return cudaGetLastError();
}

}  // namespace mpm
