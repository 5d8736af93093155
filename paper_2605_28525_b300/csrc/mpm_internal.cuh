// Internal declarations of the sparse-grid MPM library (sm_103a).
//
// Data layout in HBM (one context):
//   particle state   two buffers (ping-pong) of NF = 32 floats per particle:
//                    x(3) alpha(1, Drucker-Prager cone constant from the
//                    friction angle) F(9, row-major) id(1, uint32 bits)
//                    tau(6, symmetric Kirchhoff stress xx xy xz yy yz zz)
//                    v(3) C(9, row-major), i.e. 8 planes of 4 floats, stored
//                    in tiles of 32 particles: tile p/32 holds its 8 planes
//                    one after the other, each plane 32 float4 in particle
//                    order (see pel).  A particle's planes lie 512 B apart
//                    from one address, and one plane of 32 consecutive
//                    particles is one 512 B run.  G2P reads planes 0-3 (x,
//                    alpha, F, id) and writes all 8; P2G reads planes 0, 5-7
//                    (x, v, C) and 0, 3-4 (x, tau).  G2P reads buffer `cur`
//                    through the sort permutation and writes buffer 1-cur in
//                    sorted (block, cell) order.
//   hash table       H slots of uint64 keys (EMPTY = all ones) and int32
//                    values = compact block index Phi (Sec. 4.3, Alg. 5-6).
//   active list      block_cap entries of (relative block key, slot), sorted
//                    by key, then block coordinates per Phi.
//   grid             n_active_blocks * B^3 nodes, node phi = Phi*B^3 + l,
//                    float4 (m, mv) and float4 (f, 0) accumulators and float4
//                    (v, m) after the grid update.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mpm.h"

namespace mpm {

// particle-state components (their order fixes the planes: plane = k / 4)
enum : int {
    PX = 0, PPHI = 3, PF = 4, PID = 13, PT = 14, PV = 20, PC = 23, NF = 32
};
constexpr int NPLANE = NF / 4;

// Float index of component k of the particle at storage index p: tile p / 32,
// plane k / 4, lane p % 32, slot k % 4.  The buffers hold pstride (a multiple
// of 32) particles.
__host__ __device__ __forceinline__ int64_t pel(int64_t p, int k) {
    return ((((p >> 5) * NPLANE + (k >> 2)) << 5) + (p & 31)) * 4 + (k & 3);
}

// float4 index of plane j of the particle at storage index p.
__host__ __device__ __forceinline__ int64_t pel4(int64_t p, int j) {
    return (((p >> 5) * NPLANE + j) << 5) + (p & 31);
}

constexpr uint64_t EMPTY_KEY = ~0ull;
constexpr int KEY_BITS = 21;               // m of Eq. (key)
constexpr int KEY_BIAS = 1 << 20;          // b of Eq. (key)

// Device status words.  Every error flag is sticky: the host clears it once
// it has reported it.  Setting one also sets `abort`, after which each later
// kernel of the step (and of every queued step) returns at entry, so a batch
// of steps queued without host synchronisation stops at the first failure.
struct DevStatus {
    unsigned int n_active;       // Alg. 6 counter (the box's block count on the dense grid)
    unsigned int overflow;       // bit 0: probe limit / table full, bit 1: block capacity
    unsigned int out_of_domain;
    unsigned int numeric;        // non-finite state
    unsigned int n_pblocks;      // blocks holding particles
    unsigned int map_miss;       // a stencil block missing from the map (must stay 0)
    unsigned int abort;          // any error flag above was raised
    unsigned int steps_done;     // steps completed without error since the host cleared it
    unsigned int gen;            // step generation (block "holds particles" marks)
    unsigned int go;             // the running step's insert may proceed (written by the table clear)
    unsigned int work;           // next P2G work unit (dynamic scheduling; zeroed by the table clear)
    unsigned int scan_done[2];   // tile-scan arrival counters (bit-mask scan, bin scan); left at 0
    unsigned int pad[3];
};

__device__ __forceinline__ void raise_flag(DevStatus* s, unsigned int* word, unsigned int bits) {
    atomicOr(word, bits);
    atomicOr(&s->abort, 1u);
}

// Status words that a kernel reads but that only earlier kernels write (or
// that it may read stale, like the abort word) are read with plain, L1-cached
// loads: writes of earlier kernels are visible at launch, and one address read
// by every warp from L2 would serialise all of them on one L2 slice.

// CTA-uniform test of the abort word at kernel entry.  Every thread of the
// CTA must call it (it holds a barrier).
__device__ __forceinline__ bool cta_aborted(const DevStatus* s) {
    __shared__ unsigned int ab;
    if (threadIdx.x == 0) ab = s->abort;
    __syncthreads();
    return ab != 0u;
}

// The checked build (MPM_CHECKED=1, a separate library): an index outside the
// buffer it addresses raises bit 4 of the map-error word (and the abort word)
// and the access is skipped, so a bad index reports instead of corrupting
// memory.  In the normal build the test compiles away.
#ifndef MPM_CHECKED
#define MPM_CHECKED 0
#endif

__device__ __forceinline__ bool index_ok(int64_t i, int64_t bound, DevStatus* st) {
    if (!MPM_CHECKED) return true;
    if (i >= 0 && i < bound) return true;
    raise_flag(st, &st->map_miss, 4u);
    return false;
}

// Live active-block count, clamped to the capacity the arrays were sized for.
__device__ __forceinline__ int64_t live_blocks(const DevStatus* s, int64_t cap) {
    const int64_t n = (int64_t)s->n_active;
    return n < cap ? n : cap;
}

// Scalar parameters handed to kernels by value.
struct Params {
    int lo[3], hi[3];            // node box
    int blo[3], nb[3];           // block box: first block and block counts
    float h, inv_h, dt;
    float g[3];
    float mu, lambda;            // Lame parameters
    float mp, V0;                // particle mass and initial volume
    float phi_deg;
    int material;
    int floor_kind;
    float floor_z, floor_mu;
    float terrain_mu;
    int terrain_nx, terrain_ny;
    const float* terrain;        // device, or nullptr
    int wall_layers;
    int block_shift;             // log2(B)
    int max_probe;
    // ensembles: scenario s occupies blocks [s * ens_pitch, (s + 1) * ens_pitch)
    // along x of the block box (relative to blo); its particles keep their own
    // frame and are the ids [scen_start[s], scen_start[s + 1]).
    int n_scen;                  // 1 for a single simulation
    int ens_pitch;               // blocks per scenario along x
    const uint32_t* scen_start;  // device, n_scen + 1 entries (nullptr when n_scen == 1)
    // sizes the checked build tests indices against
    int cap_blocks;              // blocks the per-block and grid arrays hold
    int n_part;                  // particles
};

// Scenario of the particle with this id (binary search over scen_start).
__device__ __forceinline__ int scenario_of(const Params& P, uint32_t id) {
    int lo = 0, hi = P.n_scen;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&P.scen_start[mid]) <= id) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Block lookup: the hash table (Sec. 4.3), or in scan mode the block bit
// mask and its word-count scan (Sec. 4.2), where Phi = set bits below.
struct HashView {
    unsigned long long* keys;
    int* vals;
    uint64_t mask;               // H - 1
    const uint32_t* bits = nullptr;   // scan mode: bit per block of the box
    const int* pre = nullptr;         // scan mode: exclusive scan of the words' bit counts
};

// ------------------------------------------------------------------ keys

// Eq. (key): ((i+b) << 2m) | ((j+b) << m) | (k+b), m = 21, b = 2^20.
__host__ __device__ inline uint64_t pack_key(int i, int j, int k) {
    return ((uint64_t)(uint32_t)(i + KEY_BIAS) << (2 * KEY_BITS)) |
           ((uint64_t)(uint32_t)(j + KEY_BIAS) << KEY_BITS) | (uint64_t)(uint32_t)(k + KEY_BIAS);
}

// Order-preserving compact key inside the block box (i-major, k fastest).
__host__ __device__ inline uint32_t rel_key(const Params& P, int bi, int bj, int bk) {
    return (uint32_t)(((uint64_t)(bi - P.blo[0]) * (uint64_t)P.nb[1] + (uint64_t)(bj - P.blo[1])) *
                          (uint64_t)P.nb[2] +
                      (uint64_t)(bk - P.blo[2]));
}

__host__ __device__ inline void rel_decode(const Params& P, uint32_t r, int& bi, int& bj, int& bk) {
    bk = (int)(r % (uint32_t)P.nb[2]) + P.blo[2];
    uint32_t q = r / (uint32_t)P.nb[2];
    bj = (int)(q % (uint32_t)P.nb[1]) + P.blo[1];
    bi = (int)(q / (uint32_t)P.nb[1]) + P.blo[0];
}

// 64-bit finaliser of SplitMix64 (Steele, Lea and Flood 2014), the mixing
// function the paper names for spreading structured keys over the table.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Lookup of Phi for a block key: linear probing from the hashed slot until the
// key or an empty slot; bounded by max_probe (Alg. 6 never places a key
// further than that from its home slot).
__device__ __forceinline__ int hash_find(const HashView& hv, uint64_t key, int max_probe) {
    uint64_t s = mix64(key) & hv.mask;
    for (int r = 0; r < max_probe; ++r) {
        unsigned long long k = __ldg(&hv.keys[s]);
        if (k == key) return __ldg(&hv.vals[s]);
        if (k == EMPTY_KEY) return -1;
        s = (s + 1) & hv.mask;
    }
    return -1;
}

// Scan mode: Phi of the block with relative key rel, -1 if it is not marked.
__device__ __forceinline__ int mask_rank(const HashView& hv, uint32_t rel) {
    const uint32_t w = rel >> 5, b = 1u << (rel & 31u);
    const uint32_t word = __ldg(&hv.bits[w]);
    if (!(word & b)) return -1;
    return __ldg(&hv.pre[w]) + __popc(word & (b - 1u));
}

// Phi of block (bi, bj, bk): the table or the scan; -1 if absent.
__device__ __forceinline__ int lookup_block(const Params& P, const HashView& hv, int bi, int bj, int bk) {
    if (hv.bits) {
        if (bi < P.blo[0] || bj < P.blo[1] || bk < P.blo[2] || bi >= P.blo[0] + P.nb[0] ||
            bj >= P.blo[1] + P.nb[1] || bk >= P.blo[2] + P.nb[2])
            return -1;
        return mask_rank(hv, rel_key(P, bi, bj, bk));
    }
    return hash_find(hv, pack_key(bi, bj, bk), P.max_probe);
}

// ||F F^T - I||_F up to which the Drucker-Prager return map and the Hencky
// stress take their power-series form (forward and adjoint alike).
#ifndef MPM_SERIES_MAX
#define MPM_SERIES_MAX 0.0625f
#endif

// ---------------------------------------------------- quadratic B-spline

// Cell/base index: floor(x/h - 1/2).  x/h is exact for power-of-two h and the
// subtraction of 1/2 is exact for |x/h| < 2^22, so this equals the FP64 value.
__device__ __forceinline__ int base_index(float fx) { return (int)floorf(fx - 0.5f); }

// Weights of the three stencil nodes base+a for d = x/h - base in [0.5, 1.5):
// a=0: (1.5-d)^2/2, a=1: 3/4-(d-1)^2, a=2: (d-1/2)^2/2, and their derivatives
// with respect to x/h.
__device__ __forceinline__ void bspline3(float d, float w[3], float dw[3]) {
    float t0 = 1.5f - d, t1 = d - 1.0f, t2 = d - 0.5f;
    w[0] = 0.5f * t0 * t0;
    w[1] = 0.75f - t1 * t1;
    w[2] = 0.5f * t2 * t2;
    dw[0] = -t0;
    dw[1] = -2.0f * t1;
    dw[2] = t2;
}

__device__ __forceinline__ void bspline_a(float d, int a, float& w, float& dw) {
    if (a == 0) {
        float t = 1.5f - d;
        w = 0.5f * t * t;
        dw = -t;
    } else if (a == 1) {
        float t = d - 1.0f;
        w = 0.75f - t * t;
        dw = -2.0f * t;
    } else {
        float t = d - 0.5f;
        w = 0.5f * t * t;
        dw = t;
    }
}

// ------------------------------------------------------------ host side

// CTAs of the P2G kernel that fit on one SM (registers and shared memory).
#ifndef MPM_P2G_MAX_CTAS
#define MPM_P2G_MAX_CTAS 3
#endif

// Launch shapes that change no result (mpm_autotune picks them).
struct Tuning {
    int p2g_ctas_per_sm = MPM_P2G_MAX_CTAS;   // persistent P2G grid: 148 x this many CTAs of 128 threads
    int g2p_threads = 128;       // G2P CTA size (128 or 256)
    int g2p_regs = 72;           // registers a G2P thread is compiled for: 72 (128 threads only), 80, 128
};

struct RadixScratch {
    uint32_t* counts = nullptr;   // [256][ntiles]
    uint32_t* totals = nullptr;   // [256]
    int64_t tiles_cap = 0;
};

}  // namespace mpm

// Deterministic mode: a block's two half-block partial tiles of 7 channels x
// 216 nodes each, stored by P2G and summed in a fixed order by its reduce.
constexpr int64_t DET_TILE_FLOATS = 2 * 7 * 216;

struct mpm_ctx {
    mpm_config cfg;
    mpm::Params P;
    cudaStream_t st = nullptr;
    int device = 0;
    bool dense = false, det = false;
    int B = 4, B3 = 64;
    int64_t n = 0;
    int64_t pstride = 0;
    float* ps[2] = {nullptr, nullptr};
    int cur = 0;

    // hash + active list
    unsigned long long* hkeys = nullptr;
    int* hvals = nullptr;
    int64_t H = 0;
    uint32_t* akey[2] = {nullptr, nullptr};
    uint32_t* aslot[2] = {nullptr, nullptr};
    int4* bcoord = nullptr;      // per Phi: block coordinates
    uint32_t* bmask = nullptr;   // bit per block of the box: set when the insert claims its key
    int* bpre = nullptr;         // exclusive scan of the words' bit counts (+ total): Phi = rank
    int* btsum = nullptr;        // scan tile totals
    int64_t bwords = 0;          // words of bmask (0: the block keys are radix-sorted instead)
    bool scan = false;           // MPM_SCAN_COMPACTION: no hash table, Phi and lookups from bmask
    int64_t block_cap = 0;
    int64_t live_cap = 0;        // active blocks every per-step array can hold (<= block_cap)
    int64_t n_dom_blocks = 0;
    int64_t n_active = 0;        // blocks after the last rebuild
    int64_t n_pblocks = 0;

    // per particle
    uint32_t* pcode = nullptr;   // sparse: slot*B3 + cell; dense: sort key
    uint32_t* pkey[2] = {nullptr, nullptr};
    uint32_t* pval[2] = {nullptr, nullptr};
    int sorted_sel = 0;          // which pkey/pval buffer holds the sorted result
    int* bstart = nullptr;       // per Phi (first sorted particle of the block)
    int* bend = nullptr;
    int* pblocks = nullptr;      // Phi of blocks holding particles
    int* ccount = nullptr;       // per (Phi, slot): particles in the slot's cell (k-major P2G order)
    uint8_t* cperm = nullptr;    // per (Phi, slot): the slot's cell (fast mode: cells by count)
    uint8_t* cslot = nullptr;    // per (Phi, cell): the cell's slot (fast sparse mode)
    int* kpre = nullptr;         // per (Phi, k < 64): particles of the block's rounds before round k (fast sparse mode)
    int* nbr = nullptr;          // per Phi: Phi of the blocks b + {0..R-1}^3 (R = 2 for B = 4, 3 for B = 1)
    int64_t brange_cap = 0;
    int* bins = nullptr;         // counting sort: particles per (Phi, cell) bin (one per node)
    int* cs = nullptr;           // counting sort: exclusive scan of bins (+ total)
    int* tsum = nullptr;         // counting sort: scan tile totals
    uint32_t* prank = nullptr;   // counting sort: rank of each particle in its bin
    float* tbuf = nullptr;       // deterministic mode: DET_TILE_FLOATS per block
    int64_t tbuf_cap = 0;
    int* hasp = nullptr;         // per Phi: generation (DevStatus.gen) of the last step the block held particles

    // grid
    float4* gmv = nullptr;
    float4* gf = nullptr;
    float4* gv = nullptr;
    int64_t node_cap = 0;

    // terrain
    float* terrain = nullptr;

    // ensemble
    uint32_t* scen_start = nullptr;

    // adjoint scratch: node adjoints (velocity; mass and momentum; force) and dL/dE
    float4* adj_nodes = nullptr;
    int64_t adj_node_cap = 0;
    double* adj_dE = nullptr;   // [dL/dE, dL/dphi]

    // status
    mpm::DevStatus* dstat = nullptr;
    mpm::DevStatus* hstat = nullptr;   // pinned

    mpm::RadixScratch rs;
    mpm::Tuning tune;

    // staging for host <-> device particle copies
    float* stage = nullptr;
    int64_t stage_cap = 0;

    int64_t rebuild_rounds = 0;
    int64_t launches = 0;              // kernels launched by this context
    cudaStream_t ls = nullptr;         // stream kernels are enqueued on (st, or the capture stream)
    cudaStream_t cap_stream = nullptr; // private stream for graph capture
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // one step, per parity of the read buffer
    int64_t graph_launches[2] = {0, 0};              // kernels in each captured step
    int64_t cap_version = 0;           // bumped whenever a buffer is reallocated
    int64_t graph_version[2] = {-1, -1};
    int64_t est_active = 0;            // active-block estimate the next batch is sized from
    int64_t min_H = 0;                 // table size a batch must have (raised by a probe overflow)
    int64_t steps = 0;
    int64_t device_bytes = 0;
    int phase = 0;                     // 0 idle, 1 rebuilt, 2 p2g done, 3 grid done
    bool g2p_swapped = false;          // last G2P wrote the buffer now current
    std::string last_error;
};

namespace mpm {

// ---- memory (api.cu)
cudaError_t dalloc(mpm_ctx* c, void** p, size_t bytes);
void dfree(mpm_ctx* c, void* p, size_t bytes);

// ---- radix sort (radix_sort.cu)
// Stable LSD sort of (key, value) pairs on `bits` low key bits.  n_dev (device)
// holds the live count when non-null, clamped to n_cap; otherwise n_cap is the
// count.  Buffers k[0]/v[0] hold the input; returns the index of the buffer
// pair that holds the result.
int radix_sort_pairs(mpm_ctx* c, uint32_t* k[2], uint32_t* v[2], int64_t n_cap,
                     const unsigned int* n_dev, int bits, cudaStream_t st, const unsigned int* abort = nullptr);
cudaError_t radix_reserve(mpm_ctx* c, int64_t n_cap);
int radix_sort_pairs_scratch(uint32_t* k[2], uint32_t* v[2], int64_t n_cap, const unsigned int* n_dev, int bits,
                             uint32_t* counts, uint32_t* totals, cudaStream_t st);

// ---- errors of calls made without a context (api.cu)
void set_noctx_error(const std::string& why);

// ---- rebuild (rebuild.cu)
cudaError_t launch_insert(mpm_ctx* c, int64_t ins_cap);
HashView hash_view(const mpm_ctx* c);
cudaError_t launch_dense_codes(mpm_ctx* c);
cudaError_t launch_assign(mpm_ctx* c);
cudaError_t launch_particle_keys(mpm_ctx* c);
cudaError_t launch_ranges(mpm_ctx* c, const uint32_t* skey);
bool counting_sort(const mpm_ctx* c);

// ---- transfers (transfer.cu)
cudaError_t launch_p2g(mpm_ctx* c);
cudaError_t launch_grid_update(mpm_ctx* c);
cudaError_t launch_g2p(mpm_ctx* c);
cudaError_t launch_init_stress(mpm_ctx* c, float* buf);
cudaError_t launch_step_done(mpm_ctx* c);

// ---- adjoint (adjoint.cu)
cudaError_t launch_adjoint(mpm_ctx* c, const float* adj_next, float* adj_cur, float4* gvbar, float4* gmbar,
                           float4* gfbar, double* dE, double* dphi);

}  // namespace mpm
