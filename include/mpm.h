/*
 * mpm.h -- C-ABI of the B300 (sm_103a) sparse-grid explicit MPM step.
 *
 * One simulation = one opaque context on one GPU and one CUDA stream.  The
 * calls follow the paper's statement of the problem (Zhao et al., "Unified
 * sparse framework for large-scale simulations using the material point
 * method"):
 *   - Sec. 4.1: one explicit step = P2G, grid update, G2P over the active set
 *     A = U_p S(p) of the quadratic B-spline supports;
 *   - Sec. 4.1, compact indexing map phi: A -> {0..|A|-1};
 *   - Sec. 4.3, Alg. 5-7: block keys by Eq. (key), hashed insert with linear
 *     probing, overflow flag and table regrowth; phi(n) = Phi(b(n)) B^3 + l(n).
 * The library computes Phi in ascending Eq.-(key) order of the active blocks
 * (the order a scan of the dense block mask in Sec. 4.2 produces), so the
 * active set and its indices do not depend on the table size, the hash
 * function or thread timing.
 *
 * Conventions shared by every call:
 *   - Status: every call returns an mpm_status; no exception crosses the ABI.
 *     mpm_last_error() gives a human-readable reason for the last failure.
 *   - Streams: all device work runs on the stream given to mpm_create.  Calls
 *     that return data to the host synchronise that stream; the others do not
 *     wait for the GPU except where stated.
 *   - Particle arrays at the boundary are in particle-id order (the order of
 *     mpm_create's input), array-of-structs, float32: x[n][3], v[n][3],
 *     C[n][9] and F[n][9] (row-major 3x3), phi_deg[n].  "on_device" = 1 means
 *     the pointers are device pointers on the context's GPU, 0 means host
 *     memory (pinned or pageable).
 *   - Ownership: inputs are copied during the call; the library owns all of
 *     its device memory (optionally obtained through the caller's allocator,
 *     see mpm_config.alloc) and frees it in mpm_destroy.  Outputs go to
 *     caller-owned buffers.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef MPM_B300_H
#define MPM_B300_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPM_ABI_VERSION 1

typedef struct mpm_ctx mpm_ctx;

typedef enum {
    MPM_OK = 0,
    MPM_ERR_INVALID_ARG = 1,   /* bad config, size or pointer; nothing changed */
    MPM_ERR_OOM = 2,           /* a device or pinned allocation failed */
    MPM_ERR_HASH_OVERFLOW = 3, /* Alg. 7 regrowth still overflowed after max_rebuilds */
    MPM_ERR_OUT_OF_DOMAIN = 4, /* a stencil node left the potential grid box */
    MPM_ERR_NUMERIC = 5,       /* non-finite state or J <= 0; state rolled back */
    MPM_ERR_CUDA = 6,          /* a CUDA runtime call failed, or device work did not finish
                                  within 20 s of a wait (see mpm_last_error) */
    MPM_ERR_STATE = 7          /* call out of order (e.g. mpm_p2g before a rebuild) */
} mpm_status;

enum { MPM_NEOHOOKEAN = 0, MPM_DRUCKER_PRAGER = 1 };
enum { MPM_FLOOR_NONE = 0, MPM_FLOOR_STICKY = 1, MPM_FLOOR_SLIP = 2, MPM_FLOOR_COULOMB = 3 };

/* mpm_config.flags */
#define MPM_DETERMINISTIC 1u /* fixed-order P2G reduction and (block, cell, id) particle order:
                                results are bit-reproducible and identical between the sparse
                                and the dense grid; needs block_size 4 */
#define MPM_DENSE_GRID 2u    /* comparator: identity map over every block of the box; the grid
                                is cleared and updated over the whole potential domain */
#define MPM_SYNC_STEPS 4u    /* mpm_step reads the status after every insert (one host
                                synchronisation per step) instead of queueing the steps */
#define MPM_NO_GRAPHS 8u     /* mpm_step queues its steps as plain kernel launches instead of
                                replaying CUDA graphs (same kernels, same results) */
#define MPM_SCAN_COMPACTION 16u /* the paper's scan realisation (Sec. 4.2, Alg. 2-4) in place of
                                the hash (Sec. 4.3): a bit per block of the box, marked by every
                                particle's stencil, and Phi = a scan of the marks; lookups are
                                the scan itself, no table.  Same active set, same Phi, same
                                results; memory grows with the box (n_blocks / 4 bytes) */

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns a device pointer of at least `bytes` bytes usable on `stream`, or
 * NULL on failure; free releases it.  Both NULL: cudaMalloc / cudaFree. */
typedef void* (*mpm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*mpm_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

typedef struct mpm_config {
    int32_t domain_lo[3], domain_hi[3]; /* potential grid box in node indices, inclusive;
                                           |index| <= 2^20 - 1 (Sec. 4.3, Eq. (key)) */
    double dx;                          /* grid spacing h; must be a power of two so that
                                           x/h and the cell index are exact in float32 */
    double dt;                          /* time step */
    double gravity[3];                  /* body force per unit mass (f_ext = m g, Sec. 4.1) */
    int32_t block_size;                 /* B: 1 (node-level set) or 4 (paper's blocks) */
    int32_t material;                   /* MPM_NEOHOOKEAN or MPM_DRUCKER_PRAGER */
    double E, nu, rho;                  /* Young's modulus, Poisson ratio, density */
    double phi_deg;                     /* friction angle (DP) when no per-particle array */
    double particle_volume;             /* V0 per particle; m_p = rho V0.  0: dx^3 / 8 */
    int32_t floor_kind;                 /* MPM_FLOOR_* on nodes with z_n <= floor_z */
    double floor_z, floor_mu;
    const float* terrain_height;        /* optional host height map at node columns,
                                           index (i-lo0) + terrain_nx*(j-lo1); copied */
    int32_t terrain_nx, terrain_ny;     /* must equal the box's node counts in x and y */
    double terrain_mu;                  /* Coulomb coefficient on nodes with z_n <= H */
    int32_t wall_layers;                /* sticky node layers at each box face (0: 2) */
    uint32_t flags;                     /* MPM_DETERMINISTIC | MPM_DENSE_GRID | MPM_SYNC_STEPS |
                                           MPM_NO_GRAPHS | MPM_SCAN_COMPACTION */
    int64_t hash_capacity;              /* initial H, power of two (0: automatic) */
    int64_t block_capacity;             /* initial active-block capacity (0: automatic) */
    int32_t max_probe;                  /* n_probe of Alg. 6 (0: 64) */
    int32_t max_rebuilds;               /* cap on Alg. 7 regrowth rounds (0: 12) */
    mpm_alloc_fn alloc;                 /* optional allocator, see above */
    mpm_free_fn free;
    void* alloc_user;
} mpm_config;

typedef struct mpm_stats {
    int64_t n_particles;
    int64_t n_active_blocks;     /* |Phi| after the last rebuild */
    int64_t n_active_nodes;      /* n_active_blocks * B^3 */
    int64_t n_particle_blocks;   /* blocks that hold at least one particle's base cell */
    int64_t n_dense_nodes;       /* nodes of the whole potential box */
    int64_t hash_capacity;       /* current H */
    int64_t block_capacity;
    int64_t rebuild_rounds;      /* Alg. 7 regrowth rounds since create */
    int64_t steps;               /* completed steps */
    int64_t device_bytes;        /* device memory currently held */
    int64_t kernel_launches;     /* CUDA kernels this context has launched */
    int32_t flags;
    int32_t block_size;
    int32_t n_scenarios;         /* 1, or the scenarios of an ensemble context */
    int32_t reserved;
} mpm_stats;

/* Fill *cfg with defaults (zeros except: block_size 4, material NH, E 1e6,
 * nu 0.3, rho 1000, phi 30, wall_layers 2, gravity (0,0,-9.81)). */
mpm_status mpm_config_default(mpm_config* cfg);

/* Validate cfg and create a context with n >= 1 particles.  x is required;
 * v, C (zero when NULL), F (identity when NULL) and phi_deg (cfg->phi_deg
 * when NULL) are optional.  stream: a cudaStream_t, or NULL for the legacy
 * default stream.  Errors: INVALID_ARG (config or sizes), OOM, CUDA. */
mpm_status mpm_create(const mpm_config* cfg, int64_t n, const float* x, const float* v,
                      const float* C, const float* F, const float* phi_deg, int on_device,
                      void* stream, mpm_ctx** out);

/* An ensemble: n_scenarios independent simulations in one context, every
 * launch of a step covering all of them (the paper has no counterpart; it runs
 * one simulation).  Scenario s has counts[s] >= 1 particles (host array); the
 * particle arrays hold the scenarios one after another, in scenario order, and
 * the particle ids follow that order.  Every scenario uses cfg as if it were
 * alone: the same potential grid box, in its own frame (positions are never
 * shifted), and the same constants; per-scenario friction angles go through
 * phi_deg.  Inside the library scenario s's blocks sit s * (blocks of the box
 * along x) further along x, so the scenarios share one hash table, active
 * list and grid without touching each other, and boundary conditions are
 * applied in each scenario's frame.  In MPM_DETERMINISTIC mode every scenario
 * gives the same bits as a context holding that scenario alone.
 * mpm_read_active returns the shifted block keys.  Not with MPM_DENSE_GRID.
 * Errors: those of mpm_create; INVALID_ARG also when the shifted box leaves
 * the Eq.-(key) range. */
mpm_status mpm_create_ensemble(const mpm_config* cfg, int32_t n_scenarios, const int64_t* counts,
                               const float* x, const float* v, const float* C, const float* F,
                               const float* phi_deg, int on_device, void* stream, mpm_ctx** out);

/* Active-set rebuild (Alg. 5-7): cell keys, hashed insert of every particle's
 * stencil blocks, regrowth on overflow, compaction to Phi in key order,
 * particle reordering by (block, cell).  Synchronises once to read the block
 * count.  Outputs (nullable): number of active blocks and nodes.
 * Errors: OUT_OF_DOMAIN, NUMERIC (non-finite position), HASH_OVERFLOW. */
mpm_status mpm_rebuild_active(mpm_ctx* ctx, int64_t* n_active_blocks, int64_t* n_active_nodes);

/* P2G (Sec. 4.1): clear the active grid, scatter m, m v (APIC) and f_int.
 * Requires a rebuild since the last G2P (else STATE). */
mpm_status mpm_p2g(mpm_ctx* ctx);

/* Grid update (Sec. 4.1, explicit Euler) with gravity and the boundary
 * conditions; requires mpm_p2g. */
mpm_status mpm_grid_update(mpm_ctx* ctx);

/* G2P (Sec. 4.1) with the constitutive update (NH stress, or DP return map);
 * requires mpm_grid_update.  Completes the step without waiting for the GPU:
 * a non-finite result is reported (and the step undone) by the next call that
 * synchronises (mpm_rebuild_active, mpm_step, mpm_read_particles). */
mpm_status mpm_g2p(mpm_ctx* ctx);

/* nsteps full steps = rebuild + P2G + grid update + G2P each.  On error the
 * particle state is the one after the last completed step, and the stats'
 * step count says how many completed.  The steps are queued without host
 * synchronisation (as CUDA graphs, one per step) on capacities sized from
 * the last active-block count with headroom; the call synchronises once at
 * the end to read the status.  A step that outgrows the capacities stops the
 * queue on the device; the call then enlarges them (Alg. 7) and runs the
 * remaining steps again from the last completed one.  The first step of a
 * context, and a step after a partial phase sequence, run synchronously. */
mpm_status mpm_step(mpm_ctx* ctx, int32_t nsteps);

/* Copy the particle state out in id order (any pointer may be NULL). */
mpm_status mpm_read_particles(mpm_ctx* ctx, float* x, float* v, float* C, float* F, int on_device);

/* Overwrite the particle state (x, v, C, F in id order; NULL keeps the current
 * value).  phi stays.  The restart path of a checkpoint. */
mpm_status mpm_write_particles(mpm_ctx* ctx, const float* x, const float* v, const float* C,
                               const float* F, int on_device);

/* Active block keys by Eq. (key) with m = 21, b = 2^20, in Phi order (host
 * buffer of cap entries).  *n_out receives the count. */
mpm_status mpm_read_active(mpm_ctx* ctx, uint64_t* block_keys, int64_t cap, int64_t* n_out);

/* Grid values of the active nodes in phi order (host buffers, cap nodes each;
 * any may be NULL): m[cap], mv[cap][3], f[cap][3] (f_int) after mpm_p2g, and
 * v[cap][3] after mpm_grid_update.  A test hook. */
mpm_status mpm_read_grid(mpm_ctx* ctx, float* m, float* mv, float* f, float* v, int64_t cap);

mpm_status mpm_get_stats(mpm_ctx* ctx, mpm_stats* out);

/* The sorted active-block keys of a particle cloud, for callers that cannot
 * allocate device memory (the paper has no counterpart: it describes the
 * active set, not this interface).  Typical callers: code running while a
 * framework owns the whole GPU through its own memory pool, loops that must
 * not allocate after start-up, and plug-ins that receive device buffers but
 * no allocator.  Inputs: x = n particle positions (device, float32, [n][3]),
 * the potential grid box (domain_lo/hi, node indices, inclusive), dx (a
 * power of two) and block_size (1 or 4).  Output: block_keys (device,
 * cap entries) receives the Eq. (key) block keys in ascending key order -
 * the same list mpm_read_active gives after mpm_rebuild_active - and
 * *n_active (host) their count.  stream: a cudaStream_t or NULL; the call
 * waits for its own work on it.
 * No memory is allocated: the hash table, block list and sort scratch live
 * in one fixed device array of about 2 MiB, held on every GPU where it has
 * been loaded until the process exits.  Limit: 65,536 active blocks per
 * call, and no more than 128 keys crowding one stretch of its 2^17-slot
 * table; beyond that the call returns MPM_ERR_INVALID_ARG (use mpm_create
 * and mpm_rebuild_active instead).  Other errors: OUT_OF_DOMAIN, NUMERIC,
 * CUDA; the reason is in mpm_last_error(NULL).  Every call clears and
 * reuses the shared array, so calls whose GPU work overlaps (e.g. on two
 * streams) race: serialise them.  The first call on a device looks up the
 * array's address with that device current; make that first call before
 * any stream capture.  Under CUDA's lazy module loading (the default) that
 * first call is also what loads the library's device code and the array
 * onto the device, so it needs free device memory: make it once at
 * start-up, before a pool takes the GPU; later calls allocate nothing.  The
 * address is kept for the process's life: do not call this again after a
 * device reset (cudaDeviceReset). */
mpm_status mpm_active_blocks_noalloc(const float* x, int64_t n, const int32_t domain_lo[3],
                                     const int32_t domain_hi[3], double dx, int32_t block_size,
                                     uint64_t* block_keys, int64_t cap, int64_t* n_active, void* stream);

/* Launch shapes that change no result: how many P2G work CTAs run per SM,
 * the G2P CTA size, and the register budget G2P was compiled for (the paper
 * has no counterpart: these are this library's launch parameters). */
typedef struct mpm_tuning {
    int32_t p2g_ctas_per_sm;   /* 1..8 (default: the most that fit on an SM) */
    int32_t g2p_threads;       /* 128 (default) or 256 */
    int32_t g2p_regs;          /* registers a G2P thread is compiled for: 72 (default) or 96 (128 threads only), 80 or 128 */
    int32_t reserved;
    double p2g_ms, g2p_ms;     /* mpm_autotune: median device time of the chosen shapes */
} mpm_tuning;

/* Autotuner: runs one rebuild on the current state, then times P2G for each
 * p2g_ctas_per_sm from 1 to the most that fit on an SM, and G2P for each
 * (g2p_threads, g2p_regs) in
 * {(128, 72), (128, 80), (128, 96), (128, 128), (256, 80), (256, 128)}, `repeats` times each (CUDA events on the context's
 * stream; the grid is cleared before every P2G), and keeps the shapes with
 * the smallest median; the default shapes are timed first and are replaced
 * only by a shape at least 3% faster.  The particle state is not advanced: the step it
 * timed is discarded.  Synchronises.  *out (nullable) receives the choice.
 * Errors: those of mpm_rebuild_active; INVALID_ARG for repeats < 1. */
mpm_status mpm_autotune(mpm_ctx* ctx, int32_t repeats, mpm_tuning* out);

/* Read or set the launch shapes (set: INVALID_ARG outside the ranges above;
 * the time fields are ignored). */
mpm_status mpm_get_tuning(mpm_ctx* ctx, mpm_tuning* out);
mpm_status mpm_set_tuning(mpm_ctx* ctx, const mpm_tuning* in);

/* Differentiation: a hand-written adjoint (reverse mode) of one explicit
 * step, Sec. 4.1, with the Neo-Hookean stress or the Drucker-Prager return
 * map and Hencky stress, for contexts in MPM_DETERMINISTIC mode with
 * block_size 4 (other contexts: INVALID_ARG).  The paper has no counterpart.
 *
 * mpm_state_bytes / mpm_save_state / mpm_load_state copy the context's whole
 * particle state (internal layout and order, with the stored stress) to or
 * from a caller device buffer of mpm_state_bytes bytes: checkpoints for
 * recomputation.  Loading makes the next step repeat, bit for bit, the step
 * that followed the save.
 *
 * mpm_adjoint_step: with the context holding the state S_k of a step k (as
 * saved before that step), recompute step k's grid and apply the adjoint of
 * the step.  adj_next (device, read) holds dL/dS_{k+1} and adj_cur (device,
 * written) receives dL/dS_k, both in particle-id order with 24 floats a
 * particle: x(3) v(3) C(9) F(9, row-major).  Whatever L depends on through
 * the stress of S_{k+1} must already be in adj_next's F part (the adjoint of
 * step k+1 puts it there).  *dE and *dphi (host, nullable) are increased by
 * the step's part of dL/dE (Young's modulus, nu fixed) and, for
 * Drucker-Prager, of dL/dphi (degrees; every particle's friction angle moved
 * by the same amount).  The state is not advanced.  Synchronises. */
int64_t mpm_state_bytes(const mpm_ctx* ctx);
mpm_status mpm_save_state(mpm_ctx* ctx, void* dst);
mpm_status mpm_load_state(mpm_ctx* ctx, const void* src);
mpm_status mpm_adjoint_step(mpm_ctx* ctx, const float* adj_next, float* adj_cur, double* dE, double* dphi);

/* Static description of a status code; never NULL. */
const char* mpm_status_string(mpm_status s);

/* Reason for the last failure on ctx (or, when ctx is NULL, of the last
 * failed mpm_create or mpm_active_blocks_noalloc); never NULL. */
const char* mpm_last_error(const mpm_ctx* ctx);

/* Free every resource; NULL is ignored.  Synchronises the stream. */
void mpm_destroy(mpm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
