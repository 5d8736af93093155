// Active-set rebuild: Sec. 4.3, Alg. 5-7, with a canonical compaction.
//
//   k_hash_clear      Alg. 5: keys <- EMPTY, values <- invalid, counter <- 0,
//                     overflow flag <- false.
//   k_insert          Alg. 6: per particle, the blocks of its 27 stencil nodes
//                     (at most 8 for B = 4, 27 for B = 1), deduplicated inside
//                     the warp with match.any so one lane per distinct key
//                     probes; CAS(EMPTY -> key) claims a slot, the counter
//                     appends the key to the active list, linear probing up to
//                     n_probe, overflow flag on failure or capacity excess.
//   (host)            Alg. 7: on overflow double H (and the list capacity)
//                     and insert again.
//   k_assign          Phi(b) = rank of b in ascending Eq.-(key) order, written
//                     to the table value of its slot; block coordinates per
//                     Phi; the block's grid nodes are zeroed for P2G.
//   k_particle_keys   sort key (Phi(b(base)), l(base)) per particle.
//   k_ranges          particle range of every block that holds particles and
//                     the list of such blocks.
//   k_interleave      k-major particle order inside every block (the k-th
//                     particle of each cell, then the next), and the particle
//                     count per cell, for the cell-lane P2G.
#include "mpm_internal.cuh"

namespace mpm {

namespace {
constexpr unsigned FULL = 0xffffffffu;

__global__ void k_hash_clear(unsigned long long* __restrict__ keys, int* __restrict__ vals, int64_t H,
                             DevStatus* st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < H) {
        keys[i] = EMPTY_KEY;
        vals[i] = -1;
    }
    if (i == 0) {
        st->n_active = 0;
        st->overflow = 0;
        st->out_of_domain = 0;
        st->n_pblocks = 0;
    }
}

__global__ void k_status_clear(DevStatus* st) {
    st->n_active = 0;
    st->overflow = 0;
    st->out_of_domain = 0;
    st->n_pblocks = 0;
}

// Alg. 6 for one key; returns the slot holding it or -1 when n_probe slots
// were all taken by other keys (overflow).
__device__ int hash_insert(const HashView& hv, uint64_t key, uint32_t rkey, int max_probe,
                           uint32_t* __restrict__ akey, uint32_t* __restrict__ aslot, int64_t cap,
                           DevStatus* st) {
    uint64_t s = mix64(key) & hv.mask;
    for (int r = 0; r < max_probe; ++r) {
        unsigned long long cur = *((volatile unsigned long long*)&hv.keys[s]);
        if (cur == key) return (int)s;
        if (cur == EMPTY_KEY) {
            unsigned long long old = atomicCAS(&hv.keys[s], EMPTY_KEY, (unsigned long long)key);
            if (old == EMPTY_KEY) {
                unsigned idx = atomicAdd(&st->n_active, 1u);
                if ((int64_t)idx < cap) {
                    akey[idx] = rkey;
                    aslot[idx] = (uint32_t)s;
                } else {
                    atomicOr(&st->overflow, 2u);
                }
                return (int)s;
            }
            if (old == key) return (int)s;
        }
        s = (s + 1) & hv.mask;
    }
    atomicOr(&st->overflow, 1u);
    return -1;
}

// Reads x, checks it and computes the stencil base node; false if the
// particle is unusable (flags set).
__device__ __forceinline__ bool particle_base(const float* __restrict__ ps, int64_t stride, int64_t p,
                                              const Params& P, int base[3], DevStatus* st) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float fx = ps[(PX + a) * stride + p] * P.inv_h;
        if (!isfinite(fx)) {
            atomicOr(&st->numeric, 1u);
            ok = false;
            base[a] = 0;
            continue;
        }
        // the stencil base..base+2 must lie inside the node box
        if (!(fx >= (float)P.lo[a] + 0.5f && fx < (float)(P.hi[a] - 2) + 1.5f)) {
            atomicOr(&st->out_of_domain, 1u);
            ok = false;
            base[a] = 0;
            continue;
        }
        base[a] = base_index(fx);
    }
    return ok;
}

template <int B>
__global__ void __launch_bounds__(256) k_insert(const float* __restrict__ ps, int64_t stride, int64_t n,
                                                Params P, HashView hv, uint32_t* __restrict__ akey,
                                                uint32_t* __restrict__ aslot, int64_t cap,
                                                uint32_t* __restrict__ pcode, DevStatus* st) {
    constexpr int S = (B == 4) ? 2 : 0;
    constexpr int R = (B == 4) ? 2 : 3;   // blocks a stencil can span per axis
    constexpr int NJ = R * R * R;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int base[3] = {0, 0, 0};
    bool ok = p < n;
    if (ok) ok = particle_base(ps, stride, p, P, base, st);
    int b0[3], nbk[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b0[a] = base[a] >> S;
        nbk[a] = ((base[a] + 2) >> S) - b0[a] + 1;
    }
    int myslot = -1;
#pragma unroll 1
    for (int j = 0; j < NJ; ++j) {
        const int jx = j / (R * R), jy = (j / R) % R, jz = j % R;
        const bool has = ok && jx < nbk[0] && jy < nbk[1] && jz < nbk[2];
        const int bi = b0[0] + jx, bj = b0[1] + jy, bk = b0[2] + jz;
        const uint64_t key = has ? pack_key(bi, bj, bk) : EMPTY_KEY;
        const unsigned peers = __match_any_sync(FULL, key);
        const int leader = __ffs(peers) - 1;
        int slot = -1;
        if (has && lane == leader) slot = hash_insert(hv, key, rel_key(P, bi, bj, bk), P.max_probe, akey, aslot, cap, st);
        slot = __shfl_sync(FULL, slot, leader);
        if (j == 0) myslot = slot;
    }
    if (ok) {
        const int cell = (base[0] & (B - 1)) + B * ((base[1] & (B - 1)) + B * (base[2] & (B - 1)));
        pcode[p] = myslot < 0 ? 0xffffffffu : (uint32_t)myslot * (uint32_t)(B * B * B) + (uint32_t)cell;
    }
}

// Dense comparator: the identity map.  The particle's sort key is the block's
// linear index in the box times B^3 plus the cell.
template <int B>
__global__ void __launch_bounds__(256) k_dense_codes(const float* __restrict__ ps, int64_t stride, int64_t n,
                                                     Params P, uint32_t* __restrict__ pcode, DevStatus* st) {
    constexpr int S = (B == 4) ? 2 : 0;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int base[3];
    if (!particle_base(ps, stride, p, P, base, st)) return;
    const int cell = (base[0] & (B - 1)) + B * ((base[1] & (B - 1)) + B * (base[2] & (B - 1)));
    pcode[p] = rel_key(P, base[0] >> S, base[1] >> S, base[2] >> S) * (uint32_t)(B * B * B) + (uint32_t)cell;
}

// Phi in key order: the sorted list position is the compact block index.
__global__ void k_assign(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sslot, int64_t nact,
                         Params P, int* __restrict__ hvals, int4* __restrict__ bcoord, float4* __restrict__ gmv,
                         float4* __restrict__ gf, int B3, int zero_grid) {
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
}

// Phi of the blocks b + {0..R-1}^3 of every active block (runs after
// k_assign, once every table value holds its rank).
template <int B>
__global__ void k_neighbours(const int4* __restrict__ bcoord, int64_t nact, Params P, HashView hv,
                             int* __restrict__ nbr) {
    constexpr int R = (B == 4) ? 2 : 3;
    constexpr int NNB = R * R * R;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nact * NNB) return;
    const int64_t r = t / NNB;
    const int e = (int)(t % NNB);
    const int4 b = bcoord[r];
    nbr[t] = hash_find(hv, pack_key(b.x + e / (R * R), b.y + (e / R) % R, b.z + e % R), P.max_probe);
}

__global__ void k_zero_grid(float4* __restrict__ gmv, float4* __restrict__ gf, int64_t nn) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        gmv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        gf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Sort key (Phi, cell) and value (storage index).  With by_id the pair is
// written at the particle's id so that the stable sort breaks ties by id.
template <bool DENSE>
__global__ void k_particle_keys(const float* __restrict__ ps, int64_t stride, int64_t n,
                                const uint32_t* __restrict__ pcode, const int* __restrict__ hvals, int B3,
                                int by_id, uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                                DevStatus* st) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t code = pcode[p];
    uint32_t k;
    if (DENSE) {
        k = code;
    } else {
        const int r = code == 0xffffffffu ? -1 : hvals[code / (uint32_t)B3];
        if (r < 0) {
            atomicOr(&st->map_miss, 1u);
            k = 0xffffffffu;   // sorts last; k_ranges ignores it
        } else {
            k = (uint32_t)r * (uint32_t)B3 + code % (uint32_t)B3;
        }
    }
    const int64_t q = by_id ? (int64_t)__float_as_uint(ps[PID * stride + p]) : p;
    key[q] = k;
    val[q] = (uint32_t)p;
}

__global__ void k_ranges(const uint32_t* __restrict__ skey, int64_t n, int shift, int64_t nblocks,
                         int* __restrict__ bstart, int* __restrict__ bend, int* __restrict__ pblocks,
                         int* __restrict__ hasp, int gen, DevStatus* st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t r = skey[i] >> shift;
    if ((int64_t)r >= nblocks) {
        atomicOr(&st->map_miss, 1u);
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

// Reorders every block's particles from (cell, k) to k-major order: the
// k-th particle of each cell (cells in l order) before any (k+1)-th one, and
// records the particle count per cell.  One warp per block; lane l handles
// cells l and l + 32.  Output goes to the spare sort buffers.
__global__ void __launch_bounds__(128) k_interleave(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ perm,
                                                    const int* __restrict__ bstart, const int* __restrict__ bend,
                                                    const int* __restrict__ pblocks, const DevStatus* __restrict__ stc,
                                                    uint32_t* __restrict__ skey2, uint32_t* __restrict__ perm2,
                                                    int* __restrict__ ccount) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * 4 + (threadIdx.x >> 5), nw = gridDim.x * 4;
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    const int nblk = (int)stc->n_pblocks;
    for (int kb = gw; kb < nblk; kb += nw) {
        const int r = pblocks[kb];
        const int s = bstart[r], e = bend[r];
        const uint32_t base = (uint32_t)r * 64u;
        const int lo0 = first_geq(skey, s, e, base + lane), hi0 = first_geq(skey, lo0, e, base + lane + 1);
        const int lo1 = first_geq(skey, s, e, base + 32 + lane), hi1 = first_geq(skey, lo1, e, base + 33 + lane);
        const int cnt0 = hi0 - lo0, cnt1 = hi1 - lo1;
        ccount[(int64_t)r * 64 + lane] = cnt0;
        ccount[(int64_t)r * 64 + 32 + lane] = cnt1;
        int off = 0;
        for (int k = 0; k <= e - s; ++k) {   // no cell holds more than the block's particles
            const unsigned M0 = __ballot_sync(FULL, cnt0 > k), M1 = __ballot_sync(FULL, cnt1 > k);
            if ((M0 | M1) == 0u) break;
            if (cnt0 > k) {
                const int pos = s + off + __popc(M0 & lt);
                perm2[pos] = perm[lo0 + k];
                skey2[pos] = base + lane;
            }
            if (cnt1 > k) {
                const int pos = s + off + __popc(M0) + __popc(M1 & lt);
                perm2[pos] = perm[lo1 + k];
                skey2[pos] = base + 32 + lane;
            }
            off += __popc(M0) + __popc(M1);
        }
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
}  // namespace

cudaError_t launch_insert(mpm_ctx* c) {
    HashView hv{c->hkeys, c->hvals, (uint64_t)(c->H - 1)};
    k_hash_clear<<<blocks_for(c->H, 256), 256, 0, c->st>>>(c->hkeys, c->hvals, c->H, c->dstat);
    c->launches += 2;
    const float* ps = c->ps[c->cur];
    if (c->B == 4)
        k_insert<4><<<blocks_for(c->n, 256), 256, 0, c->st>>>(ps, c->pstride, c->n, c->P, hv, c->akey[0], c->aslot[0],
                                                              c->block_cap, c->pcode, c->dstat);
    else
        k_insert<1><<<blocks_for(c->n, 256), 256, 0, c->st>>>(ps, c->pstride, c->n, c->P, hv, c->akey[0], c->aslot[0],
                                                              c->block_cap, c->pcode, c->dstat);
    return cudaGetLastError();
}

cudaError_t launch_dense_codes(mpm_ctx* c) {
    k_status_clear<<<1, 1, 0, c->st>>>(c->dstat);
    c->launches += 2;
    const float* ps = c->ps[c->cur];
    if (c->B == 4)
        k_dense_codes<4><<<blocks_for(c->n, 256), 256, 0, c->st>>>(ps, c->pstride, c->n, c->P, c->pcode, c->dstat);
    else
        k_dense_codes<1><<<blocks_for(c->n, 256), 256, 0, c->st>>>(ps, c->pstride, c->n, c->P, c->pcode, c->dstat);
    return cudaGetLastError();
}

cudaError_t launch_assign(mpm_ctx* c) {
    const int zero = c->det ? 0 : 1;
    if (c->dense) {
        if (zero) {
            k_zero_grid<<<148 * 8, 256, 0, c->st>>>(c->gmv, c->gf, c->n_active * c->B3);
            ++c->launches;
        }
        return cudaGetLastError();
    }
    if (c->n_active == 0) return cudaSuccess;
    const int bits = 64 - __builtin_clzll((unsigned long long)(c->n_dom_blocks > 1 ? c->n_dom_blocks - 1 : 1));
    int sel = radix_sort_pairs(c, c->akey, c->aslot, c->n_active, nullptr, bits, c->st);
    k_assign<<<blocks_for(c->n_active * c->B3, 256), 256, 0, c->st>>>(c->akey[sel], c->aslot[sel], c->n_active, c->P,
                                                                      c->hvals, c->bcoord, c->gmv, c->gf, c->B3, zero);
    HashView hv{c->hkeys, c->hvals, (uint64_t)(c->H - 1)};
    const int nnb = c->B == 4 ? 8 : 27;
    if (c->B == 4)
        k_neighbours<4><<<blocks_for(c->n_active * nnb, 256), 256, 0, c->st>>>(c->bcoord, c->n_active, c->P, hv, c->nbr);
    else
        k_neighbours<1><<<blocks_for(c->n_active * nnb, 256), 256, 0, c->st>>>(c->bcoord, c->n_active, c->P, hv, c->nbr);
    c->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_particle_keys(mpm_ctx* c) {
    const float* ps = c->ps[c->cur];
    const int by_id = c->det ? 1 : 0;
    if (c->dense)
        k_particle_keys<true><<<blocks_for(c->n, 256), 256, 0, c->st>>>(ps, c->pstride, c->n, c->pcode, nullptr, c->B3,
                                                                       by_id, c->pkey[0], c->pval[0], c->dstat);
    else
        k_particle_keys<false><<<blocks_for(c->n, 256), 256, 0, c->st>>>(ps, c->pstride, c->n, c->pcode, c->hvals, c->B3,
                                                                        by_id, c->pkey[0], c->pval[0], c->dstat);
    ++c->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nkeys = c->n_active * c->B3;
    const int bits = 64 - __builtin_clzll((unsigned long long)(nkeys > 1 ? nkeys - 1 : 1));
    c->sorted_sel = radix_sort_pairs(c, c->pkey, c->pval, c->n, nullptr, bits, c->st);
    return cudaGetLastError();
}

cudaError_t launch_ranges(mpm_ctx* c, const uint32_t* skey) {
    const int shift = (c->B == 4) ? 6 : 0;
    k_ranges<<<blocks_for(c->n, 256), 256, 0, c->st>>>(skey, c->n, shift, c->n_active, c->bstart, c->bend, c->pblocks,
                                                        c->hasp, c->gen, c->dstat);
    ++c->launches;
    if (c->B == 4) {
        const int o = 1 - c->sorted_sel;
        k_interleave<<<148 * 8, 128, 0, c->st>>>(skey, c->pval[c->sorted_sel], c->bstart, c->bend, c->pblocks, c->dstat,
                                                c->pkey[o], c->pval[o], c->ccount);
        c->sorted_sel = o;
        ++c->launches;
    }
    return cudaGetLastError();
}

}  // namespace mpm
