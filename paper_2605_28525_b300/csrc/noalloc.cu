// mpm_active_blocks_noalloc: the sorted active-block keys of a particle
// cloud, computed without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they need
// the active set: code that runs while a framework owns every byte of the
// GPU through its own pool, real-time loops that forbid allocation after
// start-up, or plug-ins that are handed device buffers but no allocator.
// This entry point serves them.  Its hash table, block list and sort scratch
// live in one file-scope device array of fixed size, held on every GPU where
// it has been loaded for as long as the process runs; the caller passes only
// the particle positions and the output buffer.
//
// Limits: at most NA_MAX_BLOCKS active blocks per call (65,536 blocks, i.e.
// 4.2 M nodes at block size 4) and a 2^17-slot table probed at most
// NA_MAX_PROBE slots from a key's home slot; larger sets, and sets whose keys
// crowd one part of the table, are rejected with MPM_ERR_INVALID_ARG.  All
// calls share the one array, so two calls whose GPU work overlaps (for
// example on two streams) race and produce garbage; serialise them.  The
// first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current; make that first call
// before any stream capture.  With CUDA's lazy module loading (the default)
// that lookup is also what loads the library's device code and places the
// array in device memory, so the first call on a device does need free
// device memory (the ~2 MiB array and the code): make it once at start-up,
// before the caller's pool takes the GPU.  Later calls allocate nothing.
// The address is kept for the life of the process: after a device reset
// (cudaDeviceReset) it is stale, so do not call this entry point again in a
// process that reset the device.
#include <cmath>
#include <mutex>

#include "mpm_internal.cuh"

namespace mpm {
namespace {

constexpr int64_t NA_MAX_BLOCKS = 1 << 16;
constexpr int64_t NA_SLOTS = 1 << 17;
constexpr int NA_MAX_PROBE = 128;
constexpr int64_t NA_TILES = NA_MAX_BLOCKS / 2048;   // radix tiles of 2048 keys

// byte offsets inside the scratch array
constexpr size_t OFF_KEYS = 0;                                            // uint64[NA_SLOTS]
constexpr size_t OFF_LKEY = OFF_KEYS + sizeof(unsigned long long) * NA_SLOTS;   // uint32[2][MAX]
constexpr size_t OFF_LVAL = OFF_LKEY + sizeof(uint32_t) * 2 * NA_MAX_BLOCKS;    // uint32[2][MAX]
constexpr size_t OFF_CNTS = OFF_LVAL + sizeof(uint32_t) * 2 * NA_MAX_BLOCKS;    // uint32[256 * TILES]
constexpr size_t OFF_TOTS = OFF_CNTS + sizeof(uint32_t) * 256 * NA_TILES;       // uint32[256]
constexpr size_t OFF_STAT = OFF_TOTS + sizeof(uint32_t) * 256;                  // NaStatus
constexpr size_t NA_SCRATCH_BYTES = OFF_STAT + 256;                             // about 2.0 MiB

struct NaStatus {
    unsigned int n_active;
    unsigned int overflow;   // 1: probe limit, 2: more than NA_MAX_BLOCKS blocks
    unsigned int outside;    // a stencil node outside the box
    unsigned int nonfinite;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

struct NaBox {
    int lo[3], hi[3], blo[3], nb[3];
    float inv_h;
    int shift;   // log2(block size)
};

__device__ __forceinline__ uint64_t na_mix(uint64_t z) {   // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Every call starts from an empty table and zero counters.
__global__ void k_na_clear(unsigned char* scratch) {
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(scratch + OFF_KEYS);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < NA_SLOTS; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = EMPTY_KEY;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        NaStatus* s = reinterpret_cast<NaStatus*>(scratch + OFF_STAT);
        s->n_active = s->overflow = s->outside = s->nonfinite = 0;
    }
}

// Per particle: the blocks of its 27 stencil nodes, inserted with CAS and
// linear probing; each newly claimed block appends its box-relative key.
__global__ void k_na_insert(const float* __restrict__ x, int64_t n, NaBox bx, unsigned char* scratch) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(scratch + OFF_KEYS);
    uint32_t* lkey = reinterpret_cast<uint32_t*>(scratch + OFF_LKEY);
    uint32_t* lval = reinterpret_cast<uint32_t*>(scratch + OFF_LVAL);
    NaStatus* s = reinterpret_cast<NaStatus*>(scratch + OFF_STAT);
    int base[3];
    for (int a = 0; a < 3; ++a) {
        const float fx = x[3 * p + a] * bx.inv_h;
        if (!isfinite(fx)) {
            atomicOr(&s->nonfinite, 1u);
            return;
        }
        if (!(fx >= (float)bx.lo[a] + 0.5f && fx < (float)(bx.hi[a] - 2) + 1.5f)) {
            atomicOr(&s->outside, 1u);
            return;
        }
        base[a] = (int)floorf(fx - 0.5f);
    }
    const int b0x = base[0] >> bx.shift, b1x = (base[0] + 2) >> bx.shift;
    const int b0y = base[1] >> bx.shift, b1y = (base[1] + 2) >> bx.shift;
    const int b0z = base[2] >> bx.shift, b1z = (base[2] + 2) >> bx.shift;
    for (int bi = b0x; bi <= b1x; ++bi)
        for (int bj = b0y; bj <= b1y; ++bj)
            for (int bk = b0z; bk <= b1z; ++bk) {
                const uint64_t key = pack_key(bi, bj, bk);
                uint64_t slot = na_mix(key) & (uint64_t)(NA_SLOTS - 1);
                bool placed = false;
                for (int r = 0; r < NA_MAX_PROBE && !placed; ++r) {
                    const unsigned long long old = atomicCAS(&keys[slot], EMPTY_KEY, (unsigned long long)key);
                    if (old == EMPTY_KEY) {
                        const unsigned idx = atomicAdd(&s->n_active, 1u);
                        if ((int64_t)idx < NA_MAX_BLOCKS) {
                            lkey[idx] = (uint32_t)((((uint64_t)(bi - bx.blo[0]) * (uint64_t)bx.nb[1] +
                                                     (uint64_t)(bj - bx.blo[1])) * (uint64_t)bx.nb[2]) +
                                                   (uint64_t)(bk - bx.blo[2]));
                            lval[idx] = idx;
                        } else {
                            atomicOr(&s->overflow, 2u);
                        }
                        placed = true;
                    } else if (old == key) {
                        placed = true;
                    } else {
                        slot = (slot + 1) & (uint64_t)(NA_SLOTS - 1);
                    }
                }
                if (!placed) atomicOr(&s->overflow, 1u);
            }
}

// Sorted box-relative keys -> Eq. (key) block keys in the caller's buffer.
__global__ void k_na_emit(const uint32_t* __restrict__ skey, NaBox bx, const NaStatus* __restrict__ s,
                          uint64_t* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)s->n_active || r >= NA_MAX_BLOCKS) return;
    const uint32_t q = skey[r];
    const int bk = (int)(q % (uint32_t)bx.nb[2]) + bx.blo[2];
    const uint32_t t = q / (uint32_t)bx.nb[2];
    const int bj = (int)(t % (uint32_t)bx.nb[1]) + bx.blo[1];
    const int bi = (int)(t / (uint32_t)bx.nb[1]) + bx.blo[0];
    out[r] = pack_key(bi, bj, bk);
}

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};

int64_t na_floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

mpm_status na_fail(mpm_status s, const std::string& why) {
    set_noctx_error(why);
    return s;
}

}  // namespace
}  // namespace mpm

using namespace mpm;

extern "C" mpm_status mpm_active_blocks_noalloc(const float* x, int64_t n, const int32_t domain_lo[3],
                                                const int32_t domain_hi[3], double dx, int32_t block_size,
                                                uint64_t* block_keys, int64_t cap, int64_t* n_active,
                                                void* stream) {
    if (!x || !domain_lo || !domain_hi || !block_keys || !n_active)
        return na_fail(MPM_ERR_INVALID_ARG, "mpm_active_blocks_noalloc: NULL pointer argument");
    if (n < 1 || n > (int64_t)INT32_MAX) return na_fail(MPM_ERR_INVALID_ARG, "mpm_active_blocks_noalloc: bad particle count");
    if (block_size != 1 && block_size != 4)
        return na_fail(MPM_ERR_INVALID_ARG, "mpm_active_blocks_noalloc: block_size must be 1 or 4");
    int ex;
    if (!(dx > 0.0) || std::frexp(dx, &ex) != 0.5)
        return na_fail(MPM_ERR_INVALID_ARG, "mpm_active_blocks_noalloc: dx must be a positive power of two");
    NaBox bx;
    int64_t nbox = 1;
    for (int a = 0; a < 3; ++a) {
        if (domain_lo[a] > domain_hi[a] - 3 || domain_lo[a] < -(1 << 20) || domain_hi[a] > (1 << 20) - 1)
            return na_fail(MPM_ERR_INVALID_ARG, "mpm_active_blocks_noalloc: invalid domain box");
        bx.lo[a] = domain_lo[a];
        bx.hi[a] = domain_hi[a];
        bx.blo[a] = (int)na_floordiv(domain_lo[a], block_size);
        bx.nb[a] = (int)(na_floordiv(domain_hi[a], block_size) - bx.blo[a] + 1);
        nbox *= bx.nb[a];
    }
    if (nbox >= ((int64_t)1 << 32))
        return na_fail(MPM_ERR_INVALID_ARG, "mpm_active_blocks_noalloc: box has 2^32 or more blocks");
    bx.inv_h = (float)(1.0 / dx);
    bx.shift = block_size == 4 ? 2 : 0;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(MPM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(MPM_ERR_INVALID_ARG, "mpm_active_blocks_noalloc: device index too large");
    unsigned char* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return na_fail(MPM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_ptr[dev] = static_cast<unsigned char*>(ptr);
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    NaStatus* sdev = reinterpret_cast<NaStatus*>(scratch + OFF_STAT);
    k_na_clear<<<128, 256, 0, st>>>(scratch);
    k_na_insert<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, bx, scratch);
    NaStatus hs;
    e = cudaMemcpyAsync(&hs, sdev, sizeof(NaStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(MPM_ERR_CUDA, std::string("insert: ") + cudaGetErrorString(e));
    if (hs.nonfinite) return na_fail(MPM_ERR_NUMERIC, "mpm_active_blocks_noalloc: non-finite particle position");
    if (hs.outside) return na_fail(MPM_ERR_OUT_OF_DOMAIN, "mpm_active_blocks_noalloc: a particle stencil left the box");
    if ((hs.overflow & 2u) || (int64_t)hs.n_active > NA_MAX_BLOCKS)
        return na_fail(MPM_ERR_INVALID_ARG,
                       "mpm_active_blocks_noalloc: more than 65536 active blocks (the fixed scratch limit); "
                       "use mpm_create / mpm_rebuild_active instead");
    if (hs.overflow)
        return na_fail(MPM_ERR_INVALID_ARG,
                       "mpm_active_blocks_noalloc: a block key found no free slot within 128 probes of its home "
                       "slot (the fixed 2^17-slot table); use mpm_create / mpm_rebuild_active instead");
    *n_active = (int64_t)hs.n_active;
    if ((int64_t)hs.n_active > cap) return na_fail(MPM_ERR_INVALID_ARG, "mpm_active_blocks_noalloc: cap too small");
    uint32_t* lk = reinterpret_cast<uint32_t*>(scratch + OFF_LKEY);
    uint32_t* lv = reinterpret_cast<uint32_t*>(scratch + OFF_LVAL);
    uint32_t* k2[2] = {lk, lk + NA_MAX_BLOCKS};
    uint32_t* v2[2] = {lv, lv + NA_MAX_BLOCKS};
    const int bits = 64 - __builtin_clzll((unsigned long long)(nbox > 1 ? nbox - 1 : 1));
    const int sel = radix_sort_pairs_scratch(k2, v2, NA_MAX_BLOCKS, &sdev->n_active, bits,
                                             reinterpret_cast<uint32_t*>(scratch + OFF_CNTS),
                                             reinterpret_cast<uint32_t*>(scratch + OFF_TOTS), st);
    k_na_emit<<<(unsigned)((hs.n_active + 255) / 256), 256, 0, st>>>(k2[sel], bx, sdev, block_keys);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(MPM_ERR_CUDA, std::string("sort: ") + cudaGetErrorString(e));
    return MPM_OK;
}
