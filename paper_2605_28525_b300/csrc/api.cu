// C-ABI of the sparse-grid MPM library (include/mpm.h).
//
// Host-side orchestration on one stream.  One step:
//   rebuild  = insert (Alg. 6) -> regrowth (Alg. 7) if needed -> canonical
//              compaction -> particle sort -> block ranges
//   p2g      = cell-lane tile scatter (or fixed-order tile reduction)
//   grid     = explicit Euler + boundary conditions
//   g2p      = gather + constitutive update into the other particle buffer
// The phase calls (and a context's first step) read the status after the
// insert, so the host knows the block count before the compaction.  mpm_step
// instead queues whole steps with no host synchronisation: every kernel
// takes its launch size from capacities and its live counts from the status
// words, a raised error flag makes the rest of the queue return at entry,
// and one status read at the end tells how many steps completed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <vector>
#include <chrono>
#include <thread>

#include <nvtx3/nvToolsExt.h>

#include "mpm_internal.cuh"

using namespace mpm;

namespace {

thread_local std::string g_create_error;

struct AllocRegistry {
    std::unordered_map<void*, size_t> sizes;
};

std::unordered_map<const mpm_ctx*, AllocRegistry>& registries() {
    static std::unordered_map<const mpm_ctx*, AllocRegistry> r;
    return r;
}

mpm_status fail(mpm_ctx* c, mpm_status s, const std::string& why) {
    if (c) c->last_error = why;
    else g_create_error = why;
    return s;
}

mpm_status cuda_fail(mpm_ctx* c, cudaError_t e, const char* where) {
    std::string why = std::string(where) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA, why);
}

#define CK(expr)                                                   \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return cuda_fail(c, _e, #expr);     \
    } while (0)

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

template <class T>
cudaError_t grow(mpm_ctx* c, T*& p, int64_t& cap, int64_t need, double factor) {
    if (need <= cap && p) return cudaSuccess;
    int64_t nc = std::max<int64_t>(need, (int64_t)((double)cap * factor));
    nc = std::max<int64_t>(nc, 1);
    dfree(c, p, sizeof(T) * cap);
    p = nullptr;
    cap = 0;
    cudaError_t e = dalloc(c, (void**)&p, sizeof(T) * nc);
    if (e != cudaSuccess) return e;
    cap = nc;
    return cudaSuccess;
}

__global__ void k_load_comp(const float* __restrict__ src, int ncomp, int64_t n, float* __restrict__ ps,
                            int64_t stride, int comp0, int identity_fill) {
    // src is id-ordered AoS (n x ncomp); the storage is in id order here.
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    for (int k = 0; k < ncomp; ++k) {
        float v;
        if (src) v = src[p * ncomp + k];
        else v = (identity_fill && (k % 4) == 0) ? 1.f : 0.f;
        ps[pel(p, comp0 + k)] = v;
    }
}

__global__ void k_load_alpha(const float* __restrict__ phi, float phi_const, int64_t n, float* __restrict__ ps,
                             int64_t stride) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    // Drucker-Prager cone constant alpha = sqrt(2/3) 2 sin(phi) / (3 - sin(phi)),
    // kept per particle so the step needs no trigonometry.
    const float ph = phi ? phi[p] : phi_const;
    const float sp = sinf(ph * 0.017453292519943295f);
    ps[pel(p, PPHI)] = 0.816496580927726f * 2.f * sp / (3.f - sp);
    ps[pel(p, PID)] = __uint_as_float((uint32_t)p);
}

__global__ void k_store_comp(const float* __restrict__ ps, int64_t stride, int64_t n, int comp0, int ncomp,
                             float* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t id = (int64_t)__float_as_uint(ps[pel(i, PID)]);
    for (int k = 0; k < ncomp; ++k) dst[id * ncomp + k] = ps[pel(i, comp0 + k)];
}

// Permute the whole state into id order (restart path).
__global__ void k_to_id_order(const float* __restrict__ ps, float* __restrict__ po, int64_t stride, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t id = (int64_t)__float_as_uint(ps[pel(i, PID)]);
    for (int k = 0; k < NF; ++k) po[pel(id, k)] = ps[pel(i, k)];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

mpm_status validate(const mpm_config* cfg, int64_t n) {
    if (!cfg) return fail(nullptr, MPM_ERR_INVALID_ARG, "cfg is NULL");
    if (n < 1 || n > (int64_t)INT32_MAX) return fail(nullptr, MPM_ERR_INVALID_ARG, "particle count out of range");
    if (cfg->block_size != 1 && cfg->block_size != 4) return fail(nullptr, MPM_ERR_INVALID_ARG, "block_size must be 1 or 4");
    if ((cfg->flags & MPM_DETERMINISTIC) && cfg->block_size != 4)
        return fail(nullptr, MPM_ERR_INVALID_ARG, "MPM_DETERMINISTIC needs block_size 4");
    if (!(cfg->dx > 0.0) || !std::isfinite(cfg->dx)) return fail(nullptr, MPM_ERR_INVALID_ARG, "dx must be positive");
    int ex;
    if (std::frexp(cfg->dx, &ex) != 0.5) return fail(nullptr, MPM_ERR_INVALID_ARG, "dx must be a power of two");
    if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt)) return fail(nullptr, MPM_ERR_INVALID_ARG, "dt must be positive");
    for (int a = 0; a < 3; ++a) {
        if (cfg->domain_lo[a] > cfg->domain_hi[a] - 3)
            return fail(nullptr, MPM_ERR_INVALID_ARG, "domain box needs at least 3 cells per axis");
        if (cfg->domain_lo[a] < -(1 << 20) || cfg->domain_hi[a] > (1 << 20) - 1)
            return fail(nullptr, MPM_ERR_INVALID_ARG, "domain outside the Eq. (key) range [-2^20, 2^20-1]");
        if (!std::isfinite(cfg->gravity[a])) return fail(nullptr, MPM_ERR_INVALID_ARG, "gravity not finite");
    }
    const int64_t B = cfg->block_size;
    int64_t nb = 1;
    for (int a = 0; a < 3; ++a) nb *= floordiv(cfg->domain_hi[a], B) - floordiv(cfg->domain_lo[a], B) + 1;
    if (nb * B * B * B >= (int64_t)1 << 32)
        return fail(nullptr, MPM_ERR_INVALID_ARG, "box has 2^32 or more nodes (32-bit sort keys)");
    if ((cfg->flags & MPM_SCAN_COMPACTION) && (cfg->flags & MPM_DENSE_GRID))
        return fail(nullptr, MPM_ERR_INVALID_ARG, "MPM_SCAN_COMPACTION is a sparse-grid mode");
    if (cfg->material != MPM_NEOHOOKEAN && cfg->material != MPM_DRUCKER_PRAGER)
        return fail(nullptr, MPM_ERR_INVALID_ARG, "unknown material");
    if (!(cfg->E >= 0.0) || !(cfg->nu >= 0.0 && cfg->nu < 0.5) || !(cfg->rho > 0.0))
        return fail(nullptr, MPM_ERR_INVALID_ARG, "need E >= 0, 0 <= nu < 0.5, rho > 0");
    if (cfg->material == MPM_DRUCKER_PRAGER && !(cfg->E > 0.0))
        return fail(nullptr, MPM_ERR_INVALID_ARG, "Drucker-Prager needs E > 0");
    if (cfg->floor_kind < MPM_FLOOR_NONE || cfg->floor_kind > MPM_FLOOR_COULOMB)
        return fail(nullptr, MPM_ERR_INVALID_ARG, "unknown floor kind");
    if (cfg->terrain_height) {
        if (cfg->terrain_nx != cfg->domain_hi[0] - cfg->domain_lo[0] + 1 ||
            cfg->terrain_ny != cfg->domain_hi[1] - cfg->domain_lo[1] + 1)
            return fail(nullptr, MPM_ERR_INVALID_ARG, "terrain must have one height per node column of the box");
    }
    if (cfg->hash_capacity && !is_pow2(cfg->hash_capacity))
        return fail(nullptr, MPM_ERR_INVALID_ARG, "hash_capacity must be a power of two");
    if (cfg->block_capacity < 0 || cfg->max_probe < 0 || cfg->max_rebuilds < 0 || cfg->wall_layers < 0)
        return fail(nullptr, MPM_ERR_INVALID_ARG, "negative capacity or limit");
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
        return fail(nullptr, MPM_ERR_INVALID_ARG, "alloc and free must be given together");
    return MPM_OK;
}

// Wait for the context's stream, giving up after a fixed time so that a
// stalled device reports an error instead of blocking the caller forever.
cudaError_t sync_wait(mpm_ctx* c) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->st);
        if (e != cudaErrorNotReady) return e;
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(20)) return cudaErrorLaunchTimeout;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

cudaError_t read_status(mpm_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->hstat, c->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->st);
    if (e != cudaSuccess) return e;
    return sync_wait(c);
}

cudaError_t alloc_hash(mpm_ctx* c, int64_t H, int64_t cap) {
    if (c->hkeys) dfree(c, c->hkeys, sizeof(unsigned long long) * c->H);
    if (c->hvals) dfree(c, c->hvals, sizeof(int) * c->H);
    c->hkeys = nullptr;
    c->hvals = nullptr;
    for (int k = 0; k < 2; ++k) {
        if (c->akey[k]) dfree(c, c->akey[k], sizeof(uint32_t) * c->block_cap);
        if (c->aslot[k]) dfree(c, c->aslot[k], sizeof(uint32_t) * c->block_cap);
        c->akey[k] = c->aslot[k] = nullptr;
    }
    c->H = H;
    c->block_cap = cap;
    cudaError_t e;
    if ((e = dalloc(c, (void**)&c->hkeys, sizeof(unsigned long long) * H)) != cudaSuccess) return e;
    if ((e = dalloc(c, (void**)&c->hvals, sizeof(int) * H)) != cudaSuccess) return e;
    for (int k = 0; k < 2; ++k) {
        if ((e = dalloc(c, (void**)&c->akey[k], sizeof(uint32_t) * cap)) != cudaSuccess) return e;
        if ((e = dalloc(c, (void**)&c->aslot[k], sizeof(uint32_t) * cap)) != cudaSuccess) return e;
    }
    c->P.max_probe = c->cfg.max_probe;
    return radix_reserve(c, std::max<int64_t>(c->n, cap));
}

cudaError_t ensure_grid(mpm_ctx* c, int64_t nodes) {
    if (nodes <= c->node_cap && c->gmv) return cudaSuccess;
    const int64_t nc = std::max<int64_t>(nodes, (int64_t)(1.25 * (double)c->node_cap));
    dfree(c, c->gmv, 0);
    dfree(c, c->gf, 0);
    dfree(c, c->gv, 0);
    dfree(c, c->bins, 0);
    dfree(c, c->cs, 0);
    dfree(c, c->tsum, 0);
    c->gmv = c->gf = c->gv = nullptr;
    c->bins = c->cs = c->tsum = nullptr;
    c->node_cap = 0;
    cudaError_t e;
    if ((e = dalloc(c, (void**)&c->gmv, sizeof(float4) * nc)) != cudaSuccess) return e;
    if ((e = dalloc(c, (void**)&c->gf, sizeof(float4) * nc)) != cudaSuccess) return e;
    if ((e = dalloc(c, (void**)&c->gv, sizeof(float4) * nc)) != cudaSuccess) return e;
    if (counting_sort(c)) {
        // one counting-sort bin per (block, cell), i.e. per node
        if ((e = dalloc(c, (void**)&c->bins, sizeof(int) * nc)) != cudaSuccess) return e;
        if ((e = dalloc(c, (void**)&c->cs, sizeof(int) * (nc + 1))) != cudaSuccess) return e;
        if ((e = dalloc(c, (void**)&c->tsum, sizeof(int) * (nc / 2048 + 2))) != cudaSuccess) return e;
    }
    c->node_cap = nc;
    return cudaSuccess;
}

cudaError_t ensure_block_arrays(mpm_ctx* c, int64_t nb) {
    if (nb <= c->brange_cap && c->bstart) return cudaSuccess;
    const int64_t nc = std::max<int64_t>(nb, (int64_t)(1.25 * (double)c->brange_cap));
    dfree(c, c->bstart, 0);
    dfree(c, c->bend, 0);
    dfree(c, c->pblocks, 0);
    dfree(c, c->bcoord, 0);
    dfree(c, c->nbr, 0);
    dfree(c, c->ccount, 0);
    dfree(c, c->cperm, 0);
    dfree(c, c->cslot, 0);
    dfree(c, c->kpre, 0);
    dfree(c, c->hasp, 0);
    c->bstart = c->bend = c->pblocks = c->nbr = c->ccount = c->hasp = c->kpre = nullptr;
    c->bcoord = nullptr;
    c->cperm = c->cslot = nullptr;
    c->brange_cap = 0;
    cudaError_t e;
    if ((e = dalloc(c, (void**)&c->bstart, sizeof(int) * nc)) != cudaSuccess) return e;
    if ((e = dalloc(c, (void**)&c->bend, sizeof(int) * nc)) != cudaSuccess) return e;
    if ((e = dalloc(c, (void**)&c->pblocks, sizeof(int) * nc)) != cudaSuccess) return e;
    if ((e = dalloc(c, (void**)&c->bcoord, sizeof(int4) * nc)) != cudaSuccess) return e;
    if (!c->dense && (e = dalloc(c, (void**)&c->nbr, sizeof(int) * nc * (c->B == 4 ? 8 : 27))) != cudaSuccess)
        return e;
    if ((e = dalloc(c, (void**)&c->ccount, sizeof(int) * nc * c->B3)) != cudaSuccess) return e;
    if ((e = dalloc(c, (void**)&c->cperm, sizeof(uint8_t) * nc * c->B3)) != cudaSuccess) return e;
    if (!c->dense && !c->det && c->B == 4) {   // the k-major scatter of the fast sparse mode
        if ((e = dalloc(c, (void**)&c->cslot, sizeof(uint8_t) * nc * c->B3)) != cudaSuccess) return e;
        if ((e = dalloc(c, (void**)&c->kpre, sizeof(int) * nc * c->B3)) != cudaSuccess) return e;
    }
    if ((e = dalloc(c, (void**)&c->hasp, sizeof(int) * nc)) != cudaSuccess) return e;
    // generation 0 never matches a live step: start from a clean table
    if ((e = cudaMemsetAsync(c->hasp, 0, sizeof(int) * nc, c->st)) != cudaSuccess) return e;
    c->brange_cap = nc;
    return cudaSuccess;
}

// Active blocks that every per-step array can hold.
void update_live_cap(mpm_ctx* c) {
    int64_t live = c->dense ? c->n_dom_blocks : c->block_cap;
    live = std::min(live, c->brange_cap);
    live = std::min(live, c->node_cap / c->B3);
    if (c->det) live = std::min<int64_t>(live, c->tbuf_cap / DET_TILE_FLOATS);
    c->live_cap = live;
    c->P.cap_blocks = (int)live;
}

// Clear the flags a step may raise and retry from (overflow, out of domain)
// and the abort word.  numeric and map_miss stay until they are reported.
cudaError_t clear_retry_flags(mpm_ctx* c) {
    cudaError_t e = cudaMemsetAsync(&c->dstat->overflow, 0, 2 * sizeof(unsigned int), c->st);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(&c->dstat->abort, 0, 2 * sizeof(unsigned int), c->st);   // abort, steps_done
}

// Numeric failure of the last G2P: fall back to the buffer it read.
void rollback_g2p(mpm_ctx* c) {
    if (c->g2p_swapped) {
        c->cur = 1 - c->cur;
        c->g2p_swapped = false;
        if (c->steps > 0) --c->steps;
    }
    cudaMemsetAsync(&c->dstat->numeric, 0, sizeof(unsigned int), c->st);
}

mpm_status do_rebuild(mpm_ctx* c) {
    // keep the table at most half full (Alg. 7 would recover too, at the cost
    // of a second insert)
    if (!c->dense && !c->scan && 2 * c->n_active > c->H)
        CK(alloc_hash(c, 2 * c->H, std::max<int64_t>(c->block_cap, 2 * c->n_active)));
    c->ls = c->st;
    for (int round = 0;; ++round) {
        CK(clear_retry_flags(c));
        if (c->dense) CK(launch_dense_codes(c));
        else CK(launch_insert(c, c->block_cap));
        CK(read_status(c));
        const DevStatus& s = *c->hstat;
        if (s.map_miss) {
            cudaMemsetAsync(&c->dstat->map_miss, 0, sizeof(unsigned int), c->st);
            return fail(c, MPM_ERR_CUDA, "internal error: inconsistent active map or particle order (code " +
                                             std::to_string(s.map_miss) + ")");
        }
        if (s.numeric) {
            rollback_g2p(c);
            return fail(c, MPM_ERR_NUMERIC, "non-finite or inverted particle state");
        }
        c->g2p_swapped = false;
        if (s.out_of_domain) return fail(c, MPM_ERR_OUT_OF_DOMAIN, "a particle stencil left the potential grid box");
        if (c->dense || c->scan || !s.overflow) break;   // a scan-mode count never exceeds the box
        // Alg. 7: enlarge and insert again
        if (round >= c->cfg.max_rebuilds)
            return fail(c, MPM_ERR_HASH_OVERFLOW, "hash table still overflows after max_rebuilds regrowth rounds");
        int64_t H = c->H, cap = c->block_cap;
        if (s.overflow & 1u) H *= 2;
        if ((s.overflow & 2u) || (int64_t)s.n_active > cap)
            cap = std::max<int64_t>(2 * cap, next_pow2((int64_t)s.n_active));
        CK(alloc_hash(c, H, cap));
        ++c->rebuild_rounds;
    }
    c->n_active = c->dense ? c->n_dom_blocks : (int64_t)c->hstat->n_active;
    const int64_t nodes = c->n_active * c->B3;
    CK(ensure_grid(c, nodes));
    CK(ensure_block_arrays(c, c->n_active));
    if (c->det) CK(grow(c, c->tbuf, c->tbuf_cap, c->n_active * DET_TILE_FLOATS, 1.25));
    update_live_cap(c);
    CK(launch_assign(c));
    CK(launch_particle_keys(c));
    CK(launch_ranges(c, c->pkey[c->sorted_sel]));
    c->phase = 1;
    return MPM_OK;
}

mpm_status do_p2g(mpm_ctx* c) {
    CK(launch_p2g(c));
    c->phase = 2;
    return MPM_OK;
}

mpm_status do_grid(mpm_ctx* c) {
    CK(launch_grid_update(c));
    c->phase = 3;
    return MPM_OK;
}

mpm_status do_g2p(mpm_ctx* c) {
    CK(launch_g2p(c));
    c->cur = 1 - c->cur;
    c->g2p_swapped = true;
    c->phase = 0;
    ++c->steps;
    return MPM_OK;
}

// Check the flags of the last G2P (one status read).
mpm_status settle(mpm_ctx* c) {
    CK(read_status(c));
    if (c->hstat->map_miss) {
        const unsigned code = c->hstat->map_miss;
        cudaMemsetAsync(&c->dstat->map_miss, 0, sizeof(unsigned int), c->st);
        return fail(c, MPM_ERR_CUDA, "internal error: inconsistent active map or particle order (code " +
                                         std::to_string(code) + ")");
    }
    if (c->hstat->numeric) {
        rollback_g2p(c);
        return fail(c, MPM_ERR_NUMERIC, "non-finite or inverted particle state");
    }
    c->g2p_swapped = false;
    return MPM_OK;
}

mpm_status sync_step(mpm_ctx* c) {
    mpm_status s = do_rebuild(c);
    if (s == MPM_OK) s = do_p2g(c);
    if (s == MPM_OK) s = do_grid(c);
    if (s == MPM_OK) s = do_g2p(c);
    return s;
}

// The kernels of one step on c->ls, reading particle buffer c->cur.
mpm_status queue_step(mpm_ctx* c) {
    if (c->dense) CK(launch_dense_codes(c));
    else CK(launch_insert(c, c->live_cap));
    CK(launch_assign(c));
    CK(launch_particle_keys(c));
    CK(launch_ranges(c, c->pkey[c->sorted_sel]));
    CK(launch_p2g(c));
    CK(launch_grid_update(c));
    CK(launch_g2p(c));
    CK(launch_step_done(c));
    return MPM_OK;
}

// Capture one step reading buffer `parity` into an executable graph.
mpm_status capture_step(mpm_ctx* c, int parity) {
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    if (c->graph[parity]) {
        CK(cudaGraphExecDestroy(c->graph[parity]));
        c->graph[parity] = nullptr;
    }
    const int saved_cur = c->cur;
    const int64_t l0 = c->launches;
    c->cur = parity;
    c->ls = c->cap_stream;
    cudaGraph_t g = nullptr;
    mpm_status s = MPM_OK;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        s = queue_step(c);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
        if (s == MPM_OK && e2 != cudaSuccess) e = e2;
    }
    c->ls = c->st;
    c->cur = saved_cur;
    const int64_t nl = c->launches - l0;
    c->launches = l0;
    if (s != MPM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return s != MPM_OK ? s : cuda_fail(c, e, "step capture");
    }
    e = cudaGraphInstantiate(&c->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph[parity] = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    c->graph_launches[parity] = nl;
    c->graph_version[parity] = c->cap_version;
    return MPM_OK;
}

// Capacities of a batch: the last block count plus half of it as headroom.
mpm_status prepare_batch(mpm_ctx* c) {
    const int64_t est = std::max(c->est_active, c->n_active);
    const int64_t want = c->dense ? c->n_dom_blocks : est + est / 2 + 64;
    if (!c->dense && !c->scan) {
        const int64_t H = std::max<int64_t>({next_pow2(2 * want), c->H, c->min_H});
        if (c->block_cap < want || c->H < H) CK(alloc_hash(c, H, std::max(c->block_cap, want)));
    }
    CK(ensure_grid(c, want * c->B3));
    CK(ensure_block_arrays(c, want));
    if (c->det) CK(grow(c, c->tbuf, c->tbuf_cap, want * DET_TILE_FLOATS, 1.25));
    update_live_cap(c);
    if (!(c->cfg.flags & MPM_NO_GRAPHS)) {
        for (int p = 0; p < 2; ++p)
            if (!c->graph[p] || c->graph_version[p] != c->cap_version) {
                mpm_status s = capture_step(c, p);
                if (s != MPM_OK) return s;
            }
    }
    return MPM_OK;
}

// `left` steps queued without host synchronisation; on return `left` holds
// the steps still to run (0 on success).
mpm_status run_batch(mpm_ctx* c, int32_t& left) {
    int failures = 0;
    while (left > 0) {
        mpm_status s = prepare_batch(c);
        if (s != MPM_OK) return s;
        CK(clear_retry_flags(c));
        const int c0 = c->cur;
        const bool graphs = !(c->cfg.flags & MPM_NO_GRAPHS);
        for (int32_t k = 0; k < left; ++k) {
            const int p = (c0 + k) & 1;
            if (graphs) {
                CK(cudaGraphLaunch(c->graph[p], c->st));
                c->launches += c->graph_launches[p];
            } else {
                c->cur = p;
                s = queue_step(c);
                if (s != MPM_OK) {
                    c->cur = c0;
                    return s;
                }
            }
        }
        c->cur = c0;
        CK(read_status(c));
        const DevStatus st = *c->hstat;
        const int32_t done = (int32_t)std::min<unsigned>(st.steps_done, (unsigned)left);
        c->cur = (c0 + done) & 1;
        c->steps += done;
        left -= done;
        c->phase = 0;
        c->g2p_swapped = false;
        if (done > 0) failures = 0;
        if (!st.abort) {
            c->n_active = std::min<int64_t>(st.n_active, c->live_cap);
            c->est_active = c->n_active;
            continue;
        }
        // the failing step's compaction may be partial: no active set is valid now
        c->n_active = c->dense ? c->n_dom_blocks : 0;
        if (st.map_miss) {
            cudaMemsetAsync(&c->dstat->map_miss, 0, sizeof(unsigned int), c->st);
            return fail(c, MPM_ERR_CUDA, "internal error: inconsistent active map or particle order (code " +
                                             std::to_string(st.map_miss) + ")");
        }
        if (st.numeric) {
            cudaMemsetAsync(&c->dstat->numeric, 0, sizeof(unsigned int), c->st);
            return fail(c, MPM_ERR_NUMERIC, "non-finite or inverted particle state");
        }
        if (st.out_of_domain) return fail(c, MPM_ERR_OUT_OF_DOMAIN, "a particle stencil left the potential grid box");
        if (!st.overflow) return fail(c, MPM_ERR_CUDA, "internal error: a step stopped without a reason");
        // Alg. 7: enlarge and run the remaining steps again
        if (++failures > c->cfg.max_rebuilds)
            return fail(c, MPM_ERR_HASH_OVERFLOW, "hash table still overflows after max_rebuilds regrowth rounds");
        ++c->rebuild_rounds;
        if (st.overflow & 1u) c->min_H = 2 * c->H;
        c->est_active = std::max<int64_t>(st.overflow & 2u ? 2 * c->live_cap : c->live_cap, (int64_t)st.n_active);
    }
    return MPM_OK;
}

mpm_status stage_in(mpm_ctx* c, const float* src, int64_t count, int on_device, const float** dev) {
    if (!src) {
        *dev = nullptr;
        return MPM_OK;
    }
    if (on_device) {
        *dev = src;
        return MPM_OK;
    }
    CK(grow(c, c->stage, c->stage_cap, count, 1.0));
    CK(cudaMemcpyAsync(c->stage, src, sizeof(float) * count, cudaMemcpyHostToDevice, c->st));
    *dev = c->stage;
    return MPM_OK;
}

mpm_status load_arrays(mpm_ctx* c, float* buf, const float* x, const float* v, const float* Cm, const float* F,
                       int on_device, bool fill_missing) {
    const float* d;
    struct Item {
        const float* src;
        int ncomp, comp0, identity;
    } items[4] = {{x, 3, PX, 0}, {v, 3, PV, 0}, {Cm, 9, PC, 0}, {F, 9, PF, 1}};
    for (auto& it : items) {
        if (!it.src && !fill_missing) continue;
        mpm_status s = stage_in(c, it.src, c->n * it.ncomp, on_device, &d);
        if (s != MPM_OK) return s;
        k_load_comp<<<nblk(c->n, 256), 256, 0, c->st>>>(d, it.ncomp, c->n, buf, c->pstride, it.comp0, it.identity);
        ++c->launches;
        CK(cudaGetLastError());
        // the staging buffer is reused by the next item: order on the stream suffices
    }
    return MPM_OK;
}

}  // namespace

namespace mpm {

// A host-side NVTX range over one entry point, so that a timeline profiler
// shows the library's calls (the kernels they queue carry their own names).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};


void set_noctx_error(const std::string& why) { g_create_error = why; }

cudaError_t dalloc(mpm_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c->cfg.alloc) {
        *p = c->cfg.alloc(bytes, (void*)c->st, c->cfg.alloc_user);
        if (!*p) return cudaErrorMemoryAllocation;
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            return e;
        }
    }
    registries()[c].sizes[*p] = bytes;
    c->device_bytes += (int64_t)bytes;
    ++c->cap_version;   // captured steps hold buffer addresses
    return cudaSuccess;
}

void dfree(mpm_ctx* c, void* p, size_t) {
    if (!p) return;
    auto& reg = registries()[c].sizes;
    auto it = reg.find(p);
    size_t bytes = it == reg.end() ? 0 : it->second;
    if (it != reg.end()) reg.erase(it);
    if (c->cfg.free) c->cfg.free(p, bytes, (void*)c->st, c->cfg.alloc_user);
    else cudaFree(p);
    c->device_bytes -= (int64_t)bytes;
    ++c->cap_version;
}

}  // namespace mpm

extern "C" {

mpm_status mpm_config_default(mpm_config* cfg) {
    if (!cfg) return MPM_ERR_INVALID_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->block_size = 4;
    cfg->material = MPM_NEOHOOKEAN;
    cfg->E = 1e6;
    cfg->nu = 0.3;
    cfg->rho = 1000.0;
    cfg->phi_deg = 30.0;
    cfg->wall_layers = 2;
    cfg->gravity[2] = -9.81;
    cfg->dx = 1.0 / 64.0;
    cfg->dt = 1e-4;
    for (int a = 0; a < 3; ++a) cfg->domain_hi[a] = 64;
    return MPM_OK;
}

const char* mpm_status_string(mpm_status s) {
    switch (s) {
        case MPM_OK: return "ok";
        case MPM_ERR_INVALID_ARG: return "invalid argument";
        case MPM_ERR_OOM: return "out of memory";
        case MPM_ERR_HASH_OVERFLOW: return "hash table overflow after regrowth";
        case MPM_ERR_OUT_OF_DOMAIN: return "particle stencil outside the potential grid";
        case MPM_ERR_NUMERIC: return "non-finite or inverted particle state";
        case MPM_ERR_CUDA: return "CUDA error";
        case MPM_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char* mpm_last_error(const mpm_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->last_error.c_str();
}

}  // extern "C"

static mpm_status create_impl(const mpm_config* cfg, int64_t n, const float* x, const float* v, const float* Cm,
                              const float* F, const float* phi, int on_device, void* stream, mpm_ctx* c,
                              int32_t n_scen, const int64_t* counts) {
    c->cfg = *cfg;
    c->cfg.terrain_height = nullptr;
    if (!c->cfg.max_probe) c->cfg.max_probe = 64;
    if (!c->cfg.max_rebuilds) c->cfg.max_rebuilds = 12;
    if (!c->cfg.wall_layers) c->cfg.wall_layers = 2;
    c->st = (cudaStream_t)stream;
    c->ls = c->st;
    CK(cudaGetDevice(&c->device));
    c->dense = (cfg->flags & MPM_DENSE_GRID) != 0;
    c->scan = (cfg->flags & MPM_SCAN_COMPACTION) != 0;
    c->det = (cfg->flags & MPM_DETERMINISTIC) != 0;
    c->B = cfg->block_size;
    c->B3 = c->B * c->B * c->B;
    c->n = n;
    c->pstride = (n + 31) / 32 * 32;

    Params& P = c->P;
    std::memset(&P, 0, sizeof(P));
    for (int a = 0; a < 3; ++a) {
        P.lo[a] = cfg->domain_lo[a];
        P.hi[a] = cfg->domain_hi[a];
        P.blo[a] = (int)floordiv(cfg->domain_lo[a], c->B);
        P.nb[a] = (int)(floordiv(cfg->domain_hi[a], c->B) - P.blo[a] + 1);
        P.g[a] = (float)cfg->gravity[a];
    }
    P.n_scen = 1;
    if (n_scen > 1) {
        // scenario s's blocks follow scenario s - 1's along x
        const int64_t nbx = (int64_t)P.nb[0] * n_scen;
        if ((int64_t)P.blo[0] + nbx - 1 > ((int64_t)1 << 20) / c->B - 1)
            return fail(c, MPM_ERR_INVALID_ARG, "the scenarios' boxes side by side leave the Eq. (key) range");
        if (nbx * P.nb[1] * P.nb[2] >= ((int64_t)1 << 32))
            return fail(c, MPM_ERR_INVALID_ARG, "the scenarios' boxes together hold 2^32 or more blocks");
        P.n_scen = n_scen;
        P.ens_pitch = P.nb[0];
        P.nb[0] = (int)nbx;
    }
    c->n_dom_blocks = (int64_t)P.nb[0] * P.nb[1] * P.nb[2];
    P.h = (float)cfg->dx;
    P.inv_h = (float)(1.0 / cfg->dx);
    P.dt = (float)cfg->dt;
    const double mu = cfg->E / (2.0 * (1.0 + cfg->nu));
    const double la = cfg->E * cfg->nu / ((1.0 + cfg->nu) * (1.0 - 2.0 * cfg->nu));
    P.mu = (float)mu;
    P.lambda = (float)la;
    const double V0 = cfg->particle_volume > 0 ? cfg->particle_volume : cfg->dx * cfg->dx * cfg->dx / 8.0;
    P.V0 = (float)V0;
    P.mp = (float)(cfg->rho * V0);
    P.phi_deg = (float)cfg->phi_deg;
    P.material = cfg->material;
    P.floor_kind = cfg->floor_kind;
    P.floor_z = (float)cfg->floor_z;
    P.floor_mu = (float)cfg->floor_mu;
    P.terrain_mu = (float)cfg->terrain_mu;
    P.wall_layers = c->cfg.wall_layers;
    P.block_shift = c->B == 4 ? 2 : 0;
    P.max_probe = c->cfg.max_probe;
    P.n_part = (int)n;

    CK(cudaMallocHost((void**)&c->hstat, sizeof(DevStatus)));
    std::memset(c->hstat, 0, sizeof(DevStatus));
    CK(dalloc(c, (void**)&c->dstat, sizeof(DevStatus)));
    CK(cudaMemsetAsync(c->dstat, 0, sizeof(DevStatus), c->st));
    for (int b = 0; b < 2; ++b) CK(dalloc(c, (void**)&c->ps[b], sizeof(float) * NF * c->pstride));
    CK(dalloc(c, (void**)&c->pcode, sizeof(uint32_t) * n));
    for (int b = 0; b < 2; ++b) {
        CK(dalloc(c, (void**)&c->pkey[b], sizeof(uint32_t) * n));
        CK(dalloc(c, (void**)&c->pval[b], sizeof(uint32_t) * n));
    }
    if (counting_sort(c)) CK(dalloc(c, (void**)&c->prank, sizeof(uint32_t) * n));
    if (n_scen > 1) {
        std::vector<uint32_t> start(n_scen + 1, 0u);
        for (int32_t k = 0; k < n_scen; ++k) start[k + 1] = start[k] + (uint32_t)counts[k];
        CK(dalloc(c, (void**)&c->scen_start, sizeof(uint32_t) * (n_scen + 1)));
        CK(cudaMemcpyAsync(c->scen_start, start.data(), sizeof(uint32_t) * (n_scen + 1), cudaMemcpyHostToDevice,
                           c->st));
        CK(cudaStreamSynchronize(c->st));   // the host vector goes out of scope
        P.scen_start = c->scen_start;
    }
    if (cfg->terrain_height) {
        const int64_t tn = (int64_t)cfg->terrain_nx * cfg->terrain_ny;
        CK(dalloc(c, (void**)&c->terrain, sizeof(float) * tn));
        CK(cudaMemcpyAsync(c->terrain, cfg->terrain_height, sizeof(float) * tn, cudaMemcpyHostToDevice, c->st));
        P.terrain = c->terrain;
        P.terrain_nx = cfg->terrain_nx;
        P.terrain_ny = cfg->terrain_ny;
    }
    if (c->dense) {
        c->block_cap = c->n_dom_blocks;
        CK(radix_reserve(c, std::max<int64_t>(n, c->block_cap)));
    } else {
        // bit mask over the box's blocks for the ranking, unless it would
        // exceed 64 MiB (then the keys are radix-sorted)
        const int64_t words = (c->n_dom_blocks + 31) / 32;
        if (words <= ((int64_t)1 << 24)) {
            c->bwords = words;
            CK(dalloc(c, (void**)&c->bmask, sizeof(uint32_t) * words));
            CK(dalloc(c, (void**)&c->bpre, sizeof(int) * (words + 1)));
            CK(dalloc(c, (void**)&c->btsum, sizeof(int) * (words / 2048 + 2)));
        } else if (c->scan) {
            return fail(c, MPM_ERR_INVALID_ARG, "MPM_SCAN_COMPACTION: the box's block mask would exceed 64 MiB");
        }
        if (c->scan) {   // no table: any block of the box may be marked
            c->block_cap = c->n_dom_blocks;
            CK(radix_reserve(c, n));
        } else {
            int64_t cap = cfg->block_capacity ? cfg->block_capacity : std::max<int64_t>(1024, n / 32);
            int64_t H = cfg->hash_capacity ? cfg->hash_capacity : next_pow2(2 * cap);
            CK(alloc_hash(c, H, cap));
        }
    }
    mpm_status s = load_arrays(c, c->ps[0], x, v, Cm, F, on_device, true);
    if (s != MPM_OK) return s;
    const float* dphi = nullptr;
    s = stage_in(c, phi, n, on_device, &dphi);
    if (s != MPM_OK) return s;
    k_load_alpha<<<nblk(n, 256), 256, 0, c->st>>>(dphi, (float)cfg->phi_deg, n, c->ps[0], c->pstride);
    ++c->launches;
    CK(cudaGetLastError());
    CK(launch_init_stress(c, c->ps[0]));
    CK(read_status(c));
    if (c->hstat->numeric) return fail(c, MPM_ERR_INVALID_ARG, "initial deformation gradient with J <= 0");
    c->cur = 0;
    return MPM_OK;
}

extern "C" {

mpm_status mpm_create(const mpm_config* cfg, int64_t n, const float* x, const float* v, const float* C,
                      const float* F, const float* phi_deg, int on_device, void* stream, mpm_ctx** out) {
    if (!out) return fail(nullptr, MPM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    mpm_status s = validate(cfg, n);
    if (s != MPM_OK) return s;
    if (!x) return fail(nullptr, MPM_ERR_INVALID_ARG, "x is NULL");
    mpm_ctx* c = new mpm_ctx();
    s = create_impl(cfg, n, x, v, C, F, phi_deg, on_device, stream, c, 1, nullptr);
    if (s != MPM_OK) {
        g_create_error = c->last_error;
        mpm_destroy(c);
        return s;
    }
    *out = c;
    return MPM_OK;
}

mpm_status mpm_create_ensemble(const mpm_config* cfg, int32_t n_scenarios, const int64_t* counts, const float* x,
                               const float* v, const float* C, const float* F, const float* phi_deg, int on_device,
                               void* stream, mpm_ctx** out) {
    if (!out) return fail(nullptr, MPM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_scenarios < 1 || !counts) return fail(nullptr, MPM_ERR_INVALID_ARG, "need n_scenarios >= 1 and counts");
    int64_t n = 0;
    for (int32_t k = 0; k < n_scenarios; ++k) {
        if (counts[k] < 1) return fail(nullptr, MPM_ERR_INVALID_ARG, "every scenario needs at least one particle");
        n += counts[k];
        if (n > (int64_t)INT32_MAX) return fail(nullptr, MPM_ERR_INVALID_ARG, "particle count out of range");
    }
    mpm_status s = validate(cfg, n);
    if (s != MPM_OK) return s;
    if (cfg->flags & MPM_DENSE_GRID) return fail(nullptr, MPM_ERR_INVALID_ARG, "ensembles run on the sparse grid only");
    if (!x) return fail(nullptr, MPM_ERR_INVALID_ARG, "x is NULL");
    mpm_ctx* c = new mpm_ctx();
    s = create_impl(cfg, n, x, v, C, F, phi_deg, on_device, stream, c, n_scenarios, counts);
    if (s != MPM_OK) {
        g_create_error = c->last_error;
        mpm_destroy(c);
        return s;
    }
    *out = c;
    return MPM_OK;
}

mpm_status mpm_rebuild_active(mpm_ctx* c, int64_t* n_blocks, int64_t* n_nodes) {
    const mpm::NvtxRange nvtx_range("mpm_rebuild_active");
    if (!c) return MPM_ERR_INVALID_ARG;
    mpm_status s = do_rebuild(c);
    if (s != MPM_OK) return s;
    if (n_blocks) *n_blocks = c->n_active;
    if (n_nodes) *n_nodes = c->n_active * c->B3;
    return MPM_OK;
}

mpm_status mpm_p2g(mpm_ctx* c) {
    const mpm::NvtxRange nvtx_range("mpm_p2g");
    if (!c) return MPM_ERR_INVALID_ARG;
    if (c->phase != 1) return fail(c, MPM_ERR_STATE, "mpm_p2g needs mpm_rebuild_active first");
    return do_p2g(c);
}

mpm_status mpm_grid_update(mpm_ctx* c) {
    const mpm::NvtxRange nvtx_range("mpm_grid_update");
    if (!c) return MPM_ERR_INVALID_ARG;
    if (c->phase != 2) return fail(c, MPM_ERR_STATE, "mpm_grid_update needs mpm_p2g first");
    return do_grid(c);
}

mpm_status mpm_g2p(mpm_ctx* c) {
    const mpm::NvtxRange nvtx_range("mpm_g2p");
    if (!c) return MPM_ERR_INVALID_ARG;
    if (c->phase != 3) return fail(c, MPM_ERR_STATE, "mpm_g2p needs mpm_grid_update first");
    return do_g2p(c);
}

mpm_status mpm_step(mpm_ctx* c, int32_t nsteps) {
    const mpm::NvtxRange nvtx_range("mpm_step");
    if (!c || nsteps < 0) return MPM_ERR_INVALID_ARG;
    int32_t left = nsteps;
    if (c->cfg.flags & MPM_SYNC_STEPS) {
        for (; left > 0; --left) {
            mpm_status s = sync_step(c);
            if (s != MPM_OK) return s;
        }
        return settle(c);
    }
    // a step cut short through the phase calls, or no block count yet: one
    // synchronous step (it also reports what an earlier G2P left pending)
    if (left > 0 && (c->phase != 0 || c->g2p_swapped || (!c->dense && c->n_active == 0))) {
        mpm_status s = sync_step(c);
        if (s == MPM_OK) s = settle(c);
        if (s != MPM_OK) return s;
        --left;
    }
    if (left == 0) return nsteps == 0 ? settle(c) : MPM_OK;
    return run_batch(c, left);
}

mpm_status mpm_read_particles(mpm_ctx* c, float* x, float* v, float* Cm, float* F, int on_device) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (c->g2p_swapped) {
        mpm_status s0 = settle(c);
        if (s0 != MPM_OK) return s0;
    }
    struct Item {
        float* dst;
        int ncomp, comp0;
    } items[4] = {{x, 3, PX}, {v, 3, PV}, {Cm, 9, PC}, {F, 9, PF}};
    for (auto& it : items) {
        if (!it.dst) continue;
        float* d = it.dst;
        if (!on_device) {
            CK(grow(c, c->stage, c->stage_cap, c->n * it.ncomp, 1.0));
            d = c->stage;
        }
        k_store_comp<<<nblk(c->n, 256), 256, 0, c->st>>>(c->ps[c->cur], c->pstride, c->n, it.comp0, it.ncomp, d);
        ++c->launches;
        CK(cudaGetLastError());
        if (!on_device)
            CK(cudaMemcpyAsync(it.dst, c->stage, sizeof(float) * c->n * it.ncomp, cudaMemcpyDeviceToHost, c->st));
    }
    CK(sync_wait(c));
    return MPM_OK;
}

mpm_status mpm_write_particles(mpm_ctx* c, const float* x, const float* v, const float* Cm, const float* F,
                               int on_device) {
    if (!c) return MPM_ERR_INVALID_ARG;
    float* cur = c->ps[c->cur];
    float* nxt = c->ps[1 - c->cur];
    k_to_id_order<<<nblk(c->n, 256), 256, 0, c->st>>>(cur, nxt, c->pstride, c->n);
    ++c->launches;
    CK(cudaGetLastError());
    c->cur = 1 - c->cur;
    c->g2p_swapped = false;
    mpm_status s = load_arrays(c, c->ps[c->cur], x, v, Cm, F, on_device, false);
    if (s != MPM_OK) return s;
    CK(launch_init_stress(c, c->ps[c->cur]));
    CK(read_status(c));
    if (c->hstat->numeric) {
        cudaMemsetAsync(&c->dstat->numeric, 0, sizeof(unsigned int), c->st);
        return fail(c, MPM_ERR_NUMERIC, "deformation gradient with J <= 0");
    }
    c->phase = 0;
    return MPM_OK;
}

mpm_status mpm_read_active(mpm_ctx* c, uint64_t* keys, int64_t cap, int64_t* n_out) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (n_out) *n_out = c->n_active;
    if (!keys) return MPM_OK;
    if (cap < c->n_active) return fail(c, MPM_ERR_INVALID_ARG, "cap smaller than the number of active blocks");
    if (c->dense) {
        for (int64_t r = 0; r < c->n_active; ++r) {
            int bi, bj, bk;
            rel_decode(c->P, (uint32_t)r, bi, bj, bk);
            keys[r] = pack_key(bi, bj, bk);
        }
        return MPM_OK;
    }
    std::vector<int4> bc(c->n_active);
    if (c->n_active) {
        CK(cudaMemcpyAsync(bc.data(), c->bcoord, sizeof(int4) * c->n_active, cudaMemcpyDeviceToHost, c->st));
        CK(sync_wait(c));
    }
    for (int64_t r = 0; r < c->n_active; ++r) keys[r] = pack_key(bc[r].x, bc[r].y, bc[r].z);
    return MPM_OK;
}

mpm_status mpm_read_grid(mpm_ctx* c, float* m, float* mv, float* f, float* v, int64_t cap) {
    if (!c) return MPM_ERR_INVALID_ARG;
    const int64_t nn = c->n_active * c->B3;
    if (cap < nn) return fail(c, MPM_ERR_INVALID_ARG, "cap smaller than the number of active nodes");
    if ((m || mv) && c->phase < 2 && c->phase != 0) return fail(c, MPM_ERR_STATE, "grid not filled yet");
    std::vector<float4> a(nn), b(nn), g(nn);
    if (nn) {
        CK(cudaMemcpyAsync(a.data(), c->gmv, sizeof(float4) * nn, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(b.data(), c->gf, sizeof(float4) * nn, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(g.data(), c->gv, sizeof(float4) * nn, cudaMemcpyDeviceToHost, c->st));
        CK(sync_wait(c));
    }
    for (int64_t i = 0; i < nn; ++i) {
        if (m) m[i] = a[i].x;
        if (mv) {
            mv[3 * i] = a[i].y;
            mv[3 * i + 1] = a[i].z;
            mv[3 * i + 2] = a[i].w;
        }
        if (f) {
            f[3 * i] = b[i].x;
            f[3 * i + 1] = b[i].y;
            f[3 * i + 2] = b[i].z;
        }
        if (v) {
            v[3 * i] = g[i].x;
            v[3 * i + 1] = g[i].y;
            v[3 * i + 2] = g[i].z;
        }
    }
    return MPM_OK;
}

}  // extern "C"

namespace {

void fill_tuning(const mpm_ctx* c, mpm_tuning* o) {
    std::memset(o, 0, sizeof(*o));
    o->p2g_ctas_per_sm = c->tune.p2g_ctas_per_sm;
    o->g2p_threads = c->tune.g2p_threads;
    o->g2p_regs = c->tune.g2p_regs;
}

// Median of the device times of `repeats` runs of `run` (each bracketed by
// events on the context's stream, after `prep`).
template <class Prep, class Run>
mpm_status time_median(mpm_ctx* c, int repeats, const Prep& prep, const Run& run, double* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<float> t;
    mpm_status s = MPM_OK;
    for (int k = 0; k < repeats && s == MPM_OK; ++k) {
        cudaError_t e = prep();
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
        if (e == cudaSuccess) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
        if (e == cudaSuccess) e = sync_wait(c);
        float x = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
        if (e != cudaSuccess) s = cuda_fail(c, e, "autotune timing");
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MPM_OK) return s;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return MPM_OK;
}

}  // namespace

extern "C" {

mpm_status mpm_autotune(mpm_ctx* c, int32_t repeats, mpm_tuning* out) {
    if (!c || repeats < 1) return MPM_ERR_INVALID_ARG;
    mpm_status s = do_rebuild(c);
    if (s != MPM_OK) return s;
    const int64_t nodes = c->n_active * c->B3;
    // P2G accumulates into the grid and draws work units from a counter:
    // both are reset before every run
    const auto p2g_prep = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (!c->det) {
            e = cudaMemsetAsync(c->gmv, 0, sizeof(float4) * nodes, c->st);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->gf, 0, sizeof(float4) * nodes, c->st);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(&c->dstat->work, 0, sizeof(unsigned int), c->st);
        return e;
    };
    const Tuning keep = c->tune;
    double best_p2g = 1e30, best_g2p = 1e30;
    Tuning best = keep;
    // The default shapes are timed first and another shape replaces the best
    // only when it is at least 3% faster: on small problems the kernels last
    // a few microseconds and their timings alone do not separate the shapes.
    const double margin = 0.97;
    for (int k = MPM_P2G_MAX_CTAS; k >= 1; --k) {
        c->tune.p2g_ctas_per_sm = k;
        double ms = 0;
        s = time_median(c, repeats, p2g_prep, [&]() { return launch_p2g(c); }, &ms);
        if (s != MPM_OK) {
            c->tune = keep;
            return s;
        }
        if (ms < best_p2g * margin) {
            best_p2g = ms;
            best.p2g_ctas_per_sm = k;
        }
    }
    c->tune.p2g_ctas_per_sm = best.p2g_ctas_per_sm;
    CK(p2g_prep());
    CK(launch_p2g(c));
    CK(launch_grid_update(c));
    // G2P reads the current buffer and writes the other one: reruns repeat it
    static const int shapes[][2] = {{128, 72}, {128, 80}, {128, 96}, {128, 128}, {256, 80}, {256, 128}};
    for (const auto& sh : shapes) {
        c->tune.g2p_threads = sh[0];
        c->tune.g2p_regs = sh[1];
        double ms = 0;
        s = time_median(c, repeats, []() { return cudaSuccess; }, [&]() { return launch_g2p(c); }, &ms);
        if (s != MPM_OK) {
            c->tune = keep;
            return s;
        }
        if (ms < best_g2p * margin) {
            best_g2p = ms;
            best.g2p_threads = sh[0];
            best.g2p_regs = sh[1];
        }
    }
    c->tune = best;
    c->phase = 0;          // the timed step is discarded; the state is the one before it
    ++c->cap_version;      // captured steps hold the old launch shapes
    if (out) {
        fill_tuning(c, out);
        out->p2g_ms = best_p2g;
        out->g2p_ms = best_g2p;
    }
    return MPM_OK;
}

mpm_status mpm_get_tuning(mpm_ctx* c, mpm_tuning* out) {
    if (!c || !out) return MPM_ERR_INVALID_ARG;
    fill_tuning(c, out);
    return MPM_OK;
}

mpm_status mpm_set_tuning(mpm_ctx* c, const mpm_tuning* in) {
    if (!c || !in) return MPM_ERR_INVALID_ARG;
    if (in->p2g_ctas_per_sm < 1 || in->p2g_ctas_per_sm > 8 || (in->g2p_threads != 128 && in->g2p_threads != 256) ||
        (in->g2p_regs != 72 && in->g2p_regs != 80 && in->g2p_regs != 96 && in->g2p_regs != 128) ||
        ((in->g2p_regs == 72 || in->g2p_regs == 96) && in->g2p_threads != 128))
        return fail(c, MPM_ERR_INVALID_ARG, "tuning outside p2g_ctas_per_sm 1..8, g2p_threads 128/256, "
                                            "g2p_regs 72 or 96 (128 threads only), 80, 128");
    c->tune.p2g_ctas_per_sm = in->p2g_ctas_per_sm;
    c->tune.g2p_threads = in->g2p_threads;
    c->tune.g2p_regs = in->g2p_regs;
    ++c->cap_version;
    return MPM_OK;
}

int64_t mpm_state_bytes(const mpm_ctx* c) { return c ? (int64_t)sizeof(float) * NF * c->pstride : 0; }

mpm_status mpm_save_state(mpm_ctx* c, void* dst) {
    if (!c || !dst) return MPM_ERR_INVALID_ARG;
    if (c->g2p_swapped) {
        mpm_status s = settle(c);
        if (s != MPM_OK) return s;
    }
    CK(cudaMemcpyAsync(dst, c->ps[c->cur], sizeof(float) * NF * c->pstride, cudaMemcpyDeviceToDevice, c->st));
    return MPM_OK;
}

mpm_status mpm_load_state(mpm_ctx* c, const void* src) {
    if (!c || !src) return MPM_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(c->ps[c->cur], src, sizeof(float) * NF * c->pstride, cudaMemcpyDeviceToDevice, c->st));
    c->phase = 0;
    c->g2p_swapped = false;
    return MPM_OK;
}

mpm_status mpm_adjoint_step(mpm_ctx* c, const float* adj_next, float* adj_cur, double* dE, double* dphi) {
    const mpm::NvtxRange nvtx_range("mpm_adjoint_step");
    if (!c || !adj_next || !adj_cur) return MPM_ERR_INVALID_ARG;
    if (!c->det || c->B != 4)
        return fail(c, MPM_ERR_INVALID_ARG, "the adjoint needs MPM_DETERMINISTIC and block_size 4");
    mpm_status s = do_rebuild(c);
    if (s == MPM_OK) s = do_p2g(c);
    if (s == MPM_OK) s = do_grid(c);
    if (s != MPM_OK) return s;
    const int64_t nodes = c->n_active * 64;
    if (nodes > c->adj_node_cap) {
        dfree(c, c->adj_nodes, 0);
        c->adj_nodes = nullptr;
        c->adj_node_cap = 0;
        CK(dalloc(c, (void**)&c->adj_nodes, sizeof(float4) * 3 * nodes));
        c->adj_node_cap = nodes;
    }
    if (!c->adj_dE) CK(dalloc(c, (void**)&c->adj_dE, 2 * sizeof(double)));
    CK(cudaMemsetAsync(c->adj_dE, 0, 2 * sizeof(double), c->st));
    float4* base = c->adj_nodes;
    CK(launch_adjoint(c, adj_next, adj_cur, base, base + c->adj_node_cap, base + 2 * c->adj_node_cap, c->adj_dE,
                      c->adj_dE + 1));
    double h[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(h, c->adj_dE, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(sync_wait(c));
    if (dE) *dE += h[0];
    if (dphi) *dphi += h[1];
    c->phase = 0;   // the step is not taken
    return MPM_OK;
}

mpm_status mpm_get_stats(mpm_ctx* c, mpm_stats* o) {
    if (!c || !o) return MPM_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->n_particles = c->n;
    o->n_active_blocks = c->n_active;
    o->n_active_nodes = c->n_active * c->B3;
    if (c->phase >= 1 || c->steps > 0) {
        CK(cudaMemcpyAsync(c->hstat, c->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->st));
        CK(sync_wait(c));
        o->n_particle_blocks = c->hstat->n_pblocks;
    }
    int64_t dn = 1;
    for (int a = 0; a < 3; ++a) dn *= (int64_t)c->P.hi[a] - c->P.lo[a] + 1;
    o->n_dense_nodes = dn;
    o->hash_capacity = c->H;
    o->block_capacity = c->block_cap;
    o->rebuild_rounds = c->rebuild_rounds;
    o->steps = c->steps;
    o->device_bytes = c->device_bytes;
    o->flags = (int32_t)c->cfg.flags;
    o->block_size = c->B;
    o->kernel_launches = c->launches;
    o->n_scenarios = c->P.n_scen;
    return MPM_OK;
}

void mpm_destroy(mpm_ctx* c) {
    if (!c) return;
    (void)sync_wait(c);
    for (int p = 0; p < 2; ++p)
        if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    auto it = registries().find(c);
    if (it != registries().end()) {
        for (auto& kv : it->second.sizes) {
            if (c->cfg.free) c->cfg.free(kv.first, kv.second, (void*)c->st, c->cfg.alloc_user);
            else cudaFree(kv.first);
        }
        registries().erase(it);
    }
    if (c->hstat) cudaFreeHost(c->hstat);
    delete c;
}

}  // extern "C"
