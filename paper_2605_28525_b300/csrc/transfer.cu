// Particle-grid transfers and the grid update (Sec. 4.1 of the paper).
//
// P2G  m_n  = sum_p N m_p
//      mv_n = sum_p N m_p [v_p + C_p (x_n - x_p)]          (APIC)
//      f_n  = -sum_p grad N sigma_p V_p = -sum_p grad N tau_p V0
// Grid v_n = mv_n/m_n + dt (f_n/m_n + g) for m_n > 0, else 0; boundary
//      conditions on the updated velocity.
// G2P  v_p = sum N v_n,  x_p += dt v_p,
//      C_p = (sum N v_n (x) (x_n - x_p)) D_p^-1 with D_p = (h^2/4) I,
//      F_p = (I + dt sum v_n (x) grad N) F_p, then the constitutive update,
//      which also stores the Kirchhoff stress tau for the next P2G.
//
// Two P2G variants:
//   k_p2g_cells   one warp per half block (32 cells) that holds particles,
//                 handed out dynamically, lane = cell, with
//                 the block's particles in k-major order; register sums per
//                 (cell, channel family) over the 27 stencil nodes and a
//                 warp-private shared tile updated without atomics, flushed
//                 with float4 global atomics into the active nodes.  Fast;
//                 the order of the global adds varies.
//   deterministic the same kernel with the block's particles in (cell, id)
//                 order; each block stores its tile and k_p2g_reduce sums
//                 the <= 8 tiles of every node in a fixed order: results are
//                 bit-identical between runs and between sparse and dense.
//   k_p2g_atomic  the node-level (B = 1) set: per-particle float4 atomics.
#include <algorithm>

#include "mpm_internal.cuh"

namespace mpm {

namespace {

// ------------------------------------------------------------ block maps

// Block coordinates of compact block r.
template <bool DENSE>
__device__ __forceinline__ void block_coords(const Params& P, const int4* __restrict__ bcoord, int r, int b[3]) {
    if (DENSE) {
        rel_decode(P, (uint32_t)r, b[0], b[1], b[2]);
    } else {
        int4 q = bcoord[r];
        b[0] = q.x;
        b[1] = q.y;
        b[2] = q.z;
    }
}

// Compact index of block (bi, bj, bk) or -1 when absent.
template <bool DENSE>
__device__ __forceinline__ int block_rank(const Params& P, const HashView& hv, int bi, int bj, int bk) {
    if (DENSE) {
        if (bi < P.blo[0] || bj < P.blo[1] || bk < P.blo[2] || bi >= P.blo[0] + P.nb[0] ||
            bj >= P.blo[1] + P.nb[1] || bk >= P.blo[2] + P.nb[2])
            return -1;
        return (int)rel_key(P, bi, bj, bk);
    }
    return lookup_block(P, hv, bi, bj, bk);
}

// ------------------------------------------------------- P2G: cell lanes

// Particles of a block are stored "k-major": the k-th particle of every cell
// (cells in slot order) before the (k+1)-th particle of any cell; ccount
// holds the particles per slot.  A warp takes a work unit of 32 slots (lane
// l owns slot 32h + l of unit h; the rebuild orders the slots by count in the
// fast sparse mode) with a private tile of (B+2)^3 = 216 nodes.  The unit
// runs two passes, momentum (m, m v) and force (f); in each the lanes walk
// rounds k = 0, 1, ...: the k-th particles of the 32 cells are consecutive
// in memory, and each lane sums its particle into the 27 nodes of its cell's
// stencil in registers (108 momentum or 81 force accumulators).  A round's
// particle planes are staged in shared memory by cp.async one round ahead.
// At the end of a pass the lanes hold distinct cells, so for each node
// offset their target nodes are distinct: the tile is updated with plain
// read-modify-write, one warp-synchronised step per offset, no atomics.  The
// finished tile is added to the active nodes with float4 global atomics.
struct CellTileCfg {
    static constexpr int T = 6;                    // tile edge (B + 2 with B = 4)
    static constexpr int SY = 8, SZ = 52;          // strides: conflict-free for one half's 32 cells
    static constexpr int TILE = (T - 1) * (SZ + SY) + T;
    static constexpr int WARPS = 4;
};

#ifndef MPM_P2G_MINB
#define MPM_P2G_MINB MPM_P2G_MAX_CTAS
#endif

// The y and z B-spline weights of one particle together, in packed FP32
// (d = (d_y, d_z)); the same formulas as bspline3.
__device__ __forceinline__ void bspline3_yz(float2 d, float wy[3], float dwy[3], float wz[3], float dwz[3]) {
    const float2 t0 = __ffma2_rn(d, make_float2(-1.f, -1.f), make_float2(1.5f, 1.5f));   // 1.5 - d
    const float2 t1 = __fadd2_rn(d, make_float2(-1.f, -1.f));
    const float2 t2 = __fadd2_rn(d, make_float2(-0.5f, -0.5f));
    const float2 w0 = __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), t0), t0);
    const float2 w1 = __ffma2_rn(__fmul2_rn(t1, make_float2(-1.f, -1.f)), t1, make_float2(0.75f, 0.75f));
    const float2 w2 = __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), t2), t2);
    wy[0] = w0.x; wy[1] = w1.x; wy[2] = w2.x;
    wz[0] = w0.y; wz[1] = w1.y; wz[2] = w2.y;
    dwy[0] = -t0.x; dwy[1] = -2.f * t1.x; dwy[2] = t2.x;
    dwz[0] = -t0.y; dwz[1] = -2.f * t1.y; dwz[2] = t2.y;
}

// ---- two channel passes: one pass per channel family over all 27 stencil
// nodes, so that each particle is loaded and its weights computed twice per
// work unit, and the per-particle work is mostly the node sums themselves.

// Momentum pass: m and m v (APIC) at the 27 nodes, in units of m_p.  With
// q0 = v - hC d, the momentum at node (a, b, c) is q0 + hC (a, b, c).
struct MomAcc {
    float2 m_mz, mxy;
};

__device__ __forceinline__ void p2g_momentum(const Params& P, const float4 (&pl)[4], MomAcc (&acc)[27]) {
    const float4 a0 = pl[0], a5 = pl[1], a6 = pl[2], a7 = pl[3];
    const float xs[3] = {a0.x, a0.y, a0.z};
    const float v[3] = {a5.x, a5.y, a5.z};
    const float cs[9] = {a5.w, a6.x, a6.y, a6.z, a6.w, a7.x, a7.y, a7.z, a7.w};
    float d[3], hc[9];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float fx = xs[q] * P.inv_h;
        d[q] = fx - (float)base_index(fx);      // exact
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) hc[q] = cs[q] * P.h;
    float wx[3], wy[3], wz[3], dw[3];
    bspline3(d[0], wx, dw);
    bspline3(d[1], wy, dw);
    bspline3(d[2], wz, dw);
    const float q0x = v[0] - hc[0] * d[0] - hc[1] * d[1] - hc[2] * d[2];
    const float q0y = v[1] - hc[3] * d[0] - hc[4] * d[1] - hc[5] * d[2];
    const float q0z = v[2] - hc[6] * d[0] - hc[7] * d[1] - hc[8] * d[2];
    const float2 hx = make_float2(hc[0], hc[3]), hy = make_float2(hc[1], hc[4]), hz = make_float2(hc[2], hc[5]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 qa = __ffma2_rn(hx, make_float2((float)a, (float)a), make_float2(q0x, q0y));
        const float qaz = fmaf(hc[6], (float)a, q0z);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float Pw = wx[a] * wy[b];
            const float2 qb = __ffma2_rn(hy, make_float2((float)b, (float)b), qa);
            const float qbz = fmaf(hc[7], (float)b, qaz);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float N = Pw * wz[c];
                const float2 NN = make_float2(N, N);
                const float2 qxy = __ffma2_rn(hz, make_float2((float)c, (float)c), qb);
                const float qz = fmaf(hc[8], (float)c, qbz);
                MomAcc& A = acc[(a * 3 + b) * 3 + c];
                A.m_mz = __ffma2_rn(NN, make_float2(1.f, qz), A.m_mz);   // m: N x 1 + m, exact as N + m
                A.mxy = __ffma2_rn(NN, qxy, A.mxy);
            }
        }
    }
}

// Force pass: tau . grad N at the 27 nodes, in units of -V0/h.  For node
// (a, b, c): f_r = wz (tau_r0 dwx wy + tau_r1 wx dwy) + dwz tau_r2 wx wy.
struct ForceAcc {
    float2 fxy;
    float fz;
};

__device__ __forceinline__ void p2g_force(const Params& P, const float4 (&pl)[4], ForceAcc (&acc)[27]) {
    const float4 a0 = pl[0], a3 = pl[1], a4 = pl[2];
    const float xs[3] = {a0.x, a0.y, a0.z};
    const float t[6] = {a3.z, a3.w, a4.x, a4.y, a4.z, a4.w};
    float d[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float fx = xs[q] * P.inv_h;
        d[q] = fx - (float)base_index(fx);
    }
    float wx[3], dwx[3], wy[3], dwy[3], wz[3], dwz[3];
    bspline3(d[0], wx, dwx);
    bspline3_yz(make_float2(d[1], d[2]), wy, dwy, wz, dwz);
    const float2 t01 = make_float2(t[0], t[1]), t13 = make_float2(t[1], t[3]), t24 = make_float2(t[2], t[4]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float Pw = wx[a] * wy[b], Gx = dwx[a] * wy[b], Gy = wx[a] * dwy[b];
            const float2 A01 = __ffma2_rn(t01, make_float2(Gx, Gx), __fmul2_rn(t13, make_float2(Gy, Gy)));
            const float2 B01 = __fmul2_rn(t24, make_float2(Pw, Pw));
            const float A2 = fmaf(t[2], Gx, t[4] * Gy), B2 = t[5] * Pw;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ForceAcc& A = acc[(a * 3 + b) * 3 + c];
                A.fxy = __ffma2_rn(make_float2(wz[c], wz[c]), A01,
                                   __ffma2_rn(make_float2(dwz[c], dwz[c]), B01, A.fxy));
                A.fz = fmaf(wz[c], A2, fmaf(dwz[c], B2, A.fz));
            }
        }
}

// 16-byte asynchronous copy global -> shared (L2 only), and its group fences.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Rounds each P2G pass stages ahead of the one it sums, plus one: the round
// being summed waits until at most MPM_P2G_STAGES - 1 later groups are open.
#ifndef MPM_P2G_STAGES
#define MPM_P2G_STAGES 2
#endif
__device__ __forceinline__ void cp_async_wait_stages() {
    asm volatile("cp.async.wait_group %0;" ::"n"(MPM_P2G_STAGES - 1) : "memory");
}

#ifndef MPM_P2G_PCACHE
#define MPM_P2G_PCACHE 12   // rounds whose particle indices a lane loads once per work unit
#endif

template <bool DENSE, bool DET>
__global__ void __launch_bounds__(CellTileCfg::WARPS * 32, MPM_P2G_MINB) k_p2g_cells(
    const float* __restrict__ ps, int64_t stride, const uint32_t* __restrict__ perm,
    const int* __restrict__ bstart, const int* __restrict__ bend, const int* __restrict__ pblocks,
    const int* __restrict__ ccount, const uint8_t* __restrict__ cperm, const DevStatus* __restrict__ stc, Params P,
    const int* __restrict__ nbr, float4* __restrict__ gmv, float4* __restrict__ gf, float* __restrict__ tbuf,
    DevStatus* st) {
    using K = CellTileCfg;
    // Work unit: half a block's cells, handed out dynamically (in the
    // deterministic mode each half stores its whole tile to tbuf, zeros
    // included, as one of the block's two partial tiles).  Slot j (lane
    // j % 32 of half j / 32) holds cell cperm[j] when the rebuild ordered the
    // cells by count (the fast mode on the sparse grid: the units span the
    // whole tile), else cell j (a half is then the z-layers 2h, 2h+1 and, in
    // the fast mode, its tile layers 2h..2h+3).
    constexpr int HU = 2;
    const bool by_count = !DET && cperm != nullptr;
    const int TZ = (DET || by_count) ? K::T : 4;
    __shared__ float tiles[K::WARPS][7][K::TILE];
#if MPM_P2G_PCACHE
    __shared__ uint32_t pcs[K::WARPS][MPM_P2G_PCACHE][32];   // the lanes' cached particle indices
#endif
    __shared__ __align__(16) float4 stage[K::WARPS][MPM_P2G_STAGES][4][32];   // the lanes' staged particle planes
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float(&tile)[7][K::TILE] = tiles[wid];
    if (cta_aborted(stc)) return;
    const int nunits = (int)stc->n_pblocks * HU;
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;

    for (int i = lane; i < 7 * K::TILE; i += 32) (&tile[0][0])[i] = 0.f;
    __syncwarp();
    // Map errors are noted here and raised once at the end: a flag raise
    // (two atomics) inside the loops would constrain how they are scheduled.
    unsigned int miss = 0u;

    for (;;) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(&st->work, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nunits) break;
        const int r = pblocks[u / HU];
        if (!index_ok(r, P.cap_blocks, st)) continue;
        const int h0 = u % HU, h1 = h0 + 1;
        const int zoff = (DET || by_count) ? 0 : 2 * h0;   // block z-layer of the tile's layer 0
        const int s = bstart[r], kcap = bend[r] - s;   // no cell holds more than the block's particles
        const int cnt0 = ccount[(int64_t)r * 64 + lane], cnt1 = ccount[(int64_t)r * 64 + 32 + lane];
        if (!DET && __ballot_sync(FULL, (h0 ? cnt1 : cnt0) > 0) == 0u) continue;   // empty half
#pragma unroll 1
        for (int h = h0; h < h1; ++h) {
            const int cnt = h ? cnt1 : cnt0;
            const int cell = by_count ? (int)cperm[(int64_t)r * 64 + 32 * h + lane] : 32 * h + lane;
            const int cx = cell & 3, cy = (cell >> 2) & 3, cz = (cell >> 4) - zoff;
#if MPM_P2G_PCACHE
            // storage indices of this lane's first rounds, loaded once for the
            // three x-offset passes (one dependent load less per round) and
            // kept in shared memory: a round reads its index with one load
            {
                int off = 0;
#pragma unroll
                for (int k = 0; k < MPM_P2G_PCACHE; ++k) {
                    const unsigned M0 = __ballot_sync(FULL, cnt0 > k), M1 = __ballot_sync(FULL, cnt1 > k);
                    const int idx = h ? __popc(M0) + __popc(M1 & lt) : __popc(M0 & lt);
                    const int nrun = __popc(M0) + __popc(M1);
                    pcs[wid][k][lane] = (cnt > k && off + nrun <= kcap) ? perm[s + off + idx] : 0u;
                    off += nrun;
                }
                __syncwarp();
            }
#endif
            // Rounds of the unit: the fullest cell of this half.  Round k's
            // particle of this lane: storage index and its offset in the
            // block's k-major order; `nrun` particles of both halves precede
            // round k + 1.  Each pass stages round k + 1's planes in the
            // lane's half of the double buffer (cp.async) while round k is
            // summed; every lane reads only its own staged planes.
            const int R = __reduce_max_sync(FULL, cnt);
            auto round_particle = [&](int k, int& off, uint32_t& p) -> bool {
                const unsigned M0 = __ballot_sync(FULL, cnt0 > k), M1 = __ballot_sync(FULL, cnt1 > k);
                const int nrun = __popc(M0) + __popc(M1);
                bool ok = cnt > k;
                if (k >= kcap || off + nrun > kcap) {   // inconsistent counts
                    miss |= 2u;
                    ok = false;
                }
                p = 0u;
                if (ok) {
#if MPM_P2G_PCACHE
                    if (k < MPM_P2G_PCACHE)
                        p = pcs[wid][k][lane];
                    else
#endif
                        p = perm[s + off + (h ? __popc(M0) + __popc(M1 & lt) : __popc(M0 & lt))];
                    ok = index_ok(p, P.n_part, st);
                }
                off += nrun;
                return ok;
            };
            float4(&sbuf)[MPM_P2G_STAGES][4][32] = stage[wid];
            const float4* ps4 = reinterpret_cast<const float4*>(ps);
            // the planes each pass reads: 0 (x), 5 (v, C0), 6 (C1..C4), 7 (C5..C8)
            // for the momentum; 0 (x), 3 (F8, id, tau xx, xy), 4 (tau xz, yy,
            // yz, zz) for the force
            auto stage_planes = [&](bool ok, uint32_t p, int buf, bool momentum) {
                if (ok) {
                    const float4* q4 = ps4 + pel4(p, 0);
                    cp_async16(&sbuf[buf][0][lane], q4);
                    if (momentum) {
                        cp_async16(&sbuf[buf][1][lane], q4 + 32 * 5);
                        cp_async16(&sbuf[buf][2][lane], q4 + 32 * 6);
                        cp_async16(&sbuf[buf][3][lane], q4 + 32 * 7);
                    } else {
                        cp_async16(&sbuf[buf][1][lane], q4 + 32 * 3);
                        cp_async16(&sbuf[buf][2][lane], q4 + 32 * 4);
                    }
                }
                cp_async_commit();
            };
            {
                // momentum pass, then force pass: the lanes' 27-node sums of
                // their cells, added to the tile one warp-ordered node offset
                // at a time (for one offset the lanes' targets are distinct)
                MomAcc macc[27];
#pragma unroll
                for (int q = 0; q < 27; ++q) macc[q].m_mz = macc[q].mxy = make_float2(0.f, 0.f);
                int off = 0;
                uint32_t p;
                unsigned okm = 0u;   // bit j: round k + j of this lane is staged
#pragma unroll
                for (int j = 0; j < MPM_P2G_STAGES - 1; ++j) {
                    const bool ok = j < R && round_particle(j, off, p);
                    okm |= (unsigned)ok << j;
                    stage_planes(ok, p, j, true);
                }
#pragma unroll 1
                for (int k = 0; k < R; ++k) {
                    const bool cur = okm & 1u;
                    const int kn = k + MPM_P2G_STAGES - 1;
                    const bool ok = kn < R && round_particle(kn, off, p);
                    okm = (okm >> 1) | ((unsigned)ok << (MPM_P2G_STAGES - 2));
                    stage_planes(ok, p, kn % MPM_P2G_STAGES, true);
                    cp_async_wait_stages();
                    const int kb = k % MPM_P2G_STAGES;
                    if (cur) {
                        const float4 pl[4] = {sbuf[kb][0][lane], sbuf[kb][1][lane], sbuf[kb][2][lane],
                                              sbuf[kb][3][lane]};
                        p2g_momentum(P, pl, macc);
                    }
                }
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    if (cnt > 0) {
                        const int ti = (cx + q / 9) + K::SY * (cy + (q / 3) % 3) + K::SZ * (cz + q % 3);
                        tile[0][ti] += macc[q].m_mz.x;
                        tile[1][ti] += macc[q].mxy.x;
                        tile[2][ti] += macc[q].mxy.y;
                        tile[3][ti] += macc[q].m_mz.y;
                    }
                    __syncwarp();
                }
            }
            {
                ForceAcc facc[27];
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    facc[q].fxy = make_float2(0.f, 0.f);
                    facc[q].fz = 0.f;
                }
                cp_async_wait0();
                int off = 0;
                uint32_t p;
                unsigned okm = 0u;   // bit j: round k + j of this lane is staged
#pragma unroll
                for (int j = 0; j < MPM_P2G_STAGES - 1; ++j) {
                    const bool ok = j < R && round_particle(j, off, p);
                    okm |= (unsigned)ok << j;
                    stage_planes(ok, p, j, false);
                }
#pragma unroll 1
                for (int k = 0; k < R; ++k) {
                    const bool cur = okm & 1u;
                    const int kn = k + MPM_P2G_STAGES - 1;
                    const bool ok = kn < R && round_particle(kn, off, p);
                    okm = (okm >> 1) | ((unsigned)ok << (MPM_P2G_STAGES - 2));
                    stage_planes(ok, p, kn % MPM_P2G_STAGES, false);
                    cp_async_wait_stages();
                    const int kb = k % MPM_P2G_STAGES;
                    if (cur) {
                        const float4 pl[4] = {sbuf[kb][0][lane], sbuf[kb][1][lane], sbuf[kb][2][lane],
                                              make_float4(0.f, 0.f, 0.f, 0.f)};
                        p2g_force(P, pl, facc);
                    }
                }
                cp_async_wait0();
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    if (cnt > 0) {
                        const int ti = (cx + q / 9) + K::SY * (cy + (q / 3) % 3) + K::SZ * (cz + q % 3);
                        tile[4][ti] += facc[q].fxy.x;
                        tile[5][ti] += facc[q].fxy.y;
                        tile[6][ti] += facc[q].fz;
                    }
                    __syncwarp();
                }
            }
        }
        // flush the tile: deterministic mode stores it for k_p2g_reduce, the
        // fast mode adds it to the active nodes of this block and its neighbours
        const float fs = -P.V0 * P.inv_h;
        for (int t = lane; t < K::T * K::T * TZ; t += 32) {
            const int tx = t % K::T, ty = (t / K::T) % K::T, tzl = t / (K::T * K::T);
            const int ti = tx + K::SY * ty + K::SZ * tzl;
            float v[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                v[k] = tile[k][ti];
                tile[k][ti] = 0.f;
            }
            if (DET) {
                float* T = tbuf + ((int64_t)r * 2 + h0) * (7 * 216);
#pragma unroll
                for (int k = 0; k < 7; ++k) T[k * 216 + t] = v[k];
                continue;
            }
            if (v[0] == 0.f && v[1] == 0.f && v[2] == 0.f && v[3] == 0.f && v[4] == 0.f && v[5] == 0.f &&
                v[6] == 0.f)
                continue;
            const int tz = tzl + zoff;
            const int ex = tx >> 2, ey = ty >> 2, ez = tz >> 2;
            int rank;
            if (DENSE) rank = r + (ex * P.nb[1] + ey) * P.nb[2] + ez;
            else rank = __ldg(&nbr[(int64_t)r * 8 + (ex * 2 + ey) * 2 + ez]);
            if (rank < 0) {
                miss |= 1u;
                continue;
            }
            if (!index_ok(rank, P.cap_blocks, st)) continue;
            const int l = (tx & 3) + 4 * ((ty & 3) + 4 * (tz & 3));
            const int64_t g = (int64_t)rank * 64 + l;
            atomicAdd(&gmv[g], make_float4(v[0] * P.mp, v[1] * P.mp, v[2] * P.mp, v[3] * P.mp));
            atomicAdd(&gf[g], make_float4(v[4] * fs, v[5] * fs, v[6] * fs, 0.f));
        }
        __syncwarp();
    }
    if (miss) raise_flag(st, &st->map_miss, miss);
}

// --------------------------------------------- P2G: deterministic reduce

// Deterministic mode: every half block writes its finished tile (7 channels
// x 216 nodes) to tbuf instead of adding it to the grid.  Each active node
// then sums the tiles of the (at most 8) blocks b - e, e in {0,1}^3, that
// cover it, in the fixed order e = 0..7 and, for each, half 0 then half 1,
// only for blocks that hold particles this step.  The result does not depend on thread timing, and the sparse and the
// dense grid produce the same bits (absent blocks hold no particles).
template <bool DENSE>
__global__ void __launch_bounds__(256) k_p2g_reduce(int64_t cap, const DevStatus* st, Params P, HashView hv,
                                                    const int4* __restrict__ bcoord, const float* __restrict__ tbuf,
                                                    const int* __restrict__ hasp, float4* __restrict__ gmv,
                                                    float4* __restrict__ gf) {
    if (cta_aborted(st)) return;
    const int64_t nnodes = live_blocks(st, cap) * 64;
    const int gen = (int)st->gen;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnodes) return;
    const int r = (int)(i >> 6), l = (int)(i & 63);
    const int lx = l & 3, ly = (l >> 2) & 3, lz = l >> 4;
    int bc[3];
    block_coords<DENSE>(P, bcoord, r, bc);
    float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int ex = e >> 2, ey = (e >> 1) & 1, ez = e & 1;
        if ((ex && lx > 1) || (ey && ly > 1) || (ez && lz > 1)) continue;   // outside that block's tile
        const int rs = block_rank<DENSE>(P, hv, bc[0] - ex, bc[1] - ey, bc[2] - ez);
        if (rs < 0 || hasp[rs] != gen) continue;
        const int t = (lx + 4 * ex) + 6 * ((ly + 4 * ey) + 6 * (lz + 4 * ez));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float* T = tbuf + ((int64_t)rs * 2 + h) * (7 * 216);
#pragma unroll
            for (int k = 0; k < 7; ++k) v[k] += T[k * 216 + t];
        }
    }
    const float fs = -P.V0 * P.inv_h;
    gmv[i] = make_float4(v[0] * P.mp, v[1] * P.mp, v[2] * P.mp, v[3] * P.mp);
    gf[i] = make_float4(v[4] * fs, v[5] * fs, v[6] * fs, 0.f);
}

// --------------------------------------------------- P2G: node-level sets

// B = 1 (every node its own block): one thread per particle, the 27 node
// contributions added with float4 global atomics into the nodes found
// through the particle's neighbour table.  A validation mode for the
// node-level active set; the grid was zeroed by the rebuild.
__global__ void __launch_bounds__(256) k_p2g_atomic(const float* __restrict__ ps, int64_t stride,
                                                    const uint32_t* __restrict__ perm,
                                                    const uint32_t* __restrict__ skey, int64_t n,
                                                    const int* __restrict__ nbr, Params P, float4* __restrict__ gmv,
                                                    float4* __restrict__ gf, DevStatus* st) {
    if (cta_aborted(st)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = perm[i];
    const int r = (int)skey[i];
    float d[3], v[3], hc[9], t[6];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float fx = ps[pel(p, PX + q)] * P.inv_h;
        d[q] = fx - (float)base_index(fx);
        v[q] = ps[pel(p, PV + q)];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) hc[q] = ps[pel(p, PC + q)] * P.h;
#pragma unroll
    for (int q = 0; q < 6; ++q) t[q] = ps[pel(p, PT + q)];
    float wx[3], dwx[3], wy[3], dwy[3], wz[3], dwz[3];
    bspline3(d[0], wx, dwx);
    bspline3(d[1], wy, dwy);
    bspline3(d[2], wz, dwz);
    const float fs = -P.V0 * P.inv_h;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int rank = __ldg(&nbr[(int64_t)r * 27 + (a * 3 + b) * 3 + c]);
                if (rank < 0) {
                    raise_flag(st, &st->map_miss, 1u);
                    continue;
                }
                const float N = wx[a] * wy[b] * wz[c];
                const float gx = dwx[a] * wy[b] * wz[c], gy = wx[a] * dwy[b] * wz[c], gz = wx[a] * wy[b] * dwz[c];
                const float ox = (float)a - d[0], oy = (float)b - d[1], oz = (float)c - d[2];
                const float mx = v[0] + hc[0] * ox + hc[1] * oy + hc[2] * oz;
                const float my = v[1] + hc[3] * ox + hc[4] * oy + hc[5] * oz;
                const float mz = v[2] + hc[6] * ox + hc[7] * oy + hc[8] * oz;
                atomicAdd(&gmv[rank], make_float4(N * P.mp, N * mx * P.mp, N * my * P.mp, N * mz * P.mp));
                atomicAdd(&gf[rank], make_float4((gx * t[0] + gy * t[1] + gz * t[2]) * fs,
                                                 (gx * t[1] + gy * t[3] + gz * t[4]) * fs,
                                                 (gx * t[2] + gy * t[4] + gz * t[5]) * fs, 0.f));
            }
}

// ------------------------------------------------------------ grid update

// Coulomb friction against a rigid boundary with outward unit normal n: only
// an approaching velocity changes; its normal part is removed and the
// tangential part shrinks by mu |v.n| or stops.
__device__ __forceinline__ void coulomb(float& vx, float& vy, float& vz, float nx, float ny, float nz, float mu) {
    const float vn = vx * nx + vy * ny + vz * nz;
    if (vn >= 0.f) return;
    const float tx = vx - vn * nx, ty = vy - vn * ny, tz = vz - vn * nz;
    const float tn = sqrtf(tx * tx + ty * ty + tz * tz);
    const float keep = tn + mu * vn;
    if (keep <= 0.f) {
        vx = vy = vz = 0.f;
        return;
    }
    const float s = keep / tn;
    vx = tx * s;
    vy = ty * s;
    vz = tz * s;
}

__device__ __forceinline__ float terrain_at(const Params& P, int ti, int tj) {
    ti = min(max(ti, 0), P.terrain_nx - 1);
    tj = min(max(tj, 0), P.terrain_ny - 1);
    return P.terrain[ti + (int64_t)P.terrain_nx * tj];
}

template <bool DENSE>
__global__ void __launch_bounds__(256) k_grid(int64_t cap, const DevStatus* st, int B, int S3, Params P,
                                              const int4* __restrict__ bcoord, const float4* __restrict__ gmv,
                                              const float4* __restrict__ gf, float4* __restrict__ gv) {
    if (cta_aborted(st)) return;
    const int64_t nnodes = live_blocks(st, cap) << S3;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnodes; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i >> S3), l = (int)(i & ((1 << S3) - 1));
        int bc[3];
        block_coords<DENSE>(P, bcoord, r, bc);
        if (P.n_scen > 1) bc[0] -= ((bc[0] - P.blo[0]) / P.ens_pitch) * P.ens_pitch;   // the scenario's own frame
        const int n0 = bc[0] * B + l % B, n1 = bc[1] * B + (l / B) % B, n2 = bc[2] * B + l / (B * B);
        const float4 a = gmv[i];
        const float m = a.x;
        float vx = 0.f, vy = 0.f, vz = 0.f;
        if (m > 0.f) {
            const float4 f = gf[i];
            const float im = 1.0f / m;
            vx = a.y * im + P.dt * (f.x * im + P.g[0]);
            vy = a.z * im + P.dt * (f.y * im + P.g[1]);
            vz = a.w * im + P.dt * (f.z * im + P.g[2]);
            const float z = (float)n2 * P.h;
            if (P.floor_kind != MPM_FLOOR_NONE && z <= P.floor_z) {
                if (P.floor_kind == MPM_FLOOR_STICKY) {
                    vx = vy = vz = 0.f;
                } else if (P.floor_kind == MPM_FLOOR_SLIP) {
                    vz = fmaxf(vz, 0.f);
                } else {
                    coulomb(vx, vy, vz, 0.f, 0.f, 1.f, P.floor_mu);
                }
            }
            if (P.terrain) {
                const int ti = n0 - P.lo[0], tj = n1 - P.lo[1];
                const float Hn = terrain_at(P, ti, tj);
                if (z <= Hn) {
                    const int i0 = ti > 0 ? ti - 1 : ti, i1 = ti < P.terrain_nx - 1 ? ti + 1 : ti;
                    const int j0 = tj > 0 ? tj - 1 : tj, j1 = tj < P.terrain_ny - 1 ? tj + 1 : tj;
                    const float hx = (terrain_at(P, i1, tj) - terrain_at(P, i0, tj)) / ((float)(i1 - i0) * P.h);
                    const float hy = (terrain_at(P, ti, j1) - terrain_at(P, ti, j0)) / ((float)(j1 - j0) * P.h);
                    const float il = rsqrtf(hx * hx + hy * hy + 1.f);
                    coulomb(vx, vy, vz, -hx * il, -hy * il, il, P.terrain_mu);
                }
            }
            const int w = P.wall_layers;
            if (n0 - P.lo[0] < w || P.hi[0] - n0 < w || n1 - P.lo[1] < w || P.hi[1] - n1 < w || n2 - P.lo[2] < w ||
                P.hi[2] - n2 < w)
                vx = vy = vz = 0.f;
        }
        gv[i] = make_float4(vx, vy, vz, m);
    }
}

// ------------------------------------------------------ constitutive (FP32)

struct Sym {
    float xx, xy, xz, yy, yz, zz;
};

__device__ __forceinline__ float det3(const float F[9]) {
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// Neo-Hookean Kirchhoff stress tau = mu (F F^T - I) + lambda ln J I.
__device__ __forceinline__ bool nh_tau(const Params& P, const float F[9], Sym& t) {
    const float J = det3(F);
    if (!(J > 0.f)) return false;
    const float lj = P.lambda * logf(J);
    t.xx = P.mu * (F[0] * F[0] + F[1] * F[1] + F[2] * F[2] - 1.f) + lj;
    t.yy = P.mu * (F[3] * F[3] + F[4] * F[4] + F[5] * F[5] - 1.f) + lj;
    t.zz = P.mu * (F[6] * F[6] + F[7] * F[7] + F[8] * F[8] - 1.f) + lj;
    t.xy = P.mu * (F[0] * F[3] + F[1] * F[4] + F[2] * F[5]);
    t.xz = P.mu * (F[0] * F[6] + F[1] * F[7] + F[2] * F[8]);
    t.yz = P.mu * (F[3] * F[6] + F[4] * F[7] + F[5] * F[8]);
    return true;
}

#ifndef MPM_JACOBI_SWEEPS
#define MPM_JACOBI_SWEEPS 4   // at most
#endif

// One Jacobi rotation of the symmetric S in the (p, q) plane, accumulated in
// V (columns).  The tangent of the rotation angle is the smaller root of
// t^2 + 2 theta t - 1 = 0 with theta = (S_qq - S_pp) / (2 S_pq), written as
// t = 2 S_pq sign(d) / (|d| + sqrt(d^2 + 4 S_pq^2)), d = S_qq - S_pp, which
// needs no division by S_pq.  Couplings below 1e-12 of the diagonal are
// treated as converged.
template <int p, int q, int r>
__device__ __forceinline__ void jacobi_rot(float S[3][3], float V[3][3]) {
    const float spq = S[p][q];
    // negligible coupling: no rotation (this also keeps the division below
    // away from denormal operands once the sweeps have converged)
    if (!(fabsf(spq) > 1e-12f * (fabsf(S[p][p]) + fabsf(S[q][q])))) return;
    const float dd = S[q][q] - S[p][p];
    const float den = fabsf(dd) + sqrtf(fmaf(dd, dd, 4.f * spq * spq));
    const float t = copysignf(2.f, dd) * __fdividef(spq, den);
    const float c = rsqrtf(fmaf(t, t, 1.f));
    const float s = t * c;
    S[p][p] -= t * spq;
    S[q][q] += t * spq;
    S[p][q] = S[q][p] = 0.f;
    const float srp = S[r][p], srq = S[r][q];
    S[r][p] = S[p][r] = c * srp - s * srq;
    S[r][q] = S[q][r] = s * srp + c * srq;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float vp = V[k][p], vq = V[k][q];
        V[k][p] = c * vp - s * vq;
        V[k][q] = s * vp + c * vq;
    }
}

#ifndef MPM_JACOBI_TOL
#define MPM_JACOBI_TOL 1e-7f
#endif

// Jacobi eigenanalysis of the symmetric S: on return its diagonal holds the
// eigenvalues (unordered) and the columns of U the eigenvectors.  From the
// third sweep on, a thread whose off-diagonal entries are all below
// MPM_JACOBI_TOL of the trace stops; the test is per thread, so a particle's
// result does not depend on the other particles of its warp.
__device__ __forceinline__ void jacobi_eig3(float S[3][3], float U[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) U[i][j] = (i == j) ? 1.f : 0.f;
#pragma unroll
    for (int sweep = 0; sweep < MPM_JACOBI_SWEEPS; ++sweep) {
        if (sweep >= 2) {
            const float tol = MPM_JACOBI_TOL * (fabsf(S[0][0]) + fabsf(S[1][1]) + fabsf(S[2][2]));
            if (fabsf(S[0][1]) <= tol && fabsf(S[0][2]) <= tol && fabsf(S[1][2]) <= tol) break;
        }
        jacobi_rot<0, 1, 2>(S, U);
        jacobi_rot<0, 2, 1>(S, U);
        jacobi_rot<1, 2, 0>(S, U);
    }
}

// Principal Hencky strains of F from the left Cauchy-Green tensor
// b = F F^T = U diag(exp(2 eps)) U^T.  False when det F <= 0 or b is not
// positive definite in FP32.
__device__ __forceinline__ bool left_hencky(const float F[9], float U[3][3], float eps[3]) {
    if (!(det3(F) > 0.f)) return false;
    float S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            S[i][j] = S[j][i] = F[i * 3 + 0] * F[j * 3 + 0] + F[i * 3 + 1] * F[j * 3 + 1] + F[i * 3 + 2] * F[j * 3 + 2];
    jacobi_eig3(S, U);
    if (!(S[0][0] > 0.f && S[1][1] > 0.f && S[2][2] > 0.f)) return false;
    eps[0] = 0.5f * logf(S[0][0]);
    eps[1] = 0.5f * logf(S[1][1]);
    eps[2] = 0.5f * logf(S[2][2]);
    return true;
}

// tau = U diag(2 mu H + lambda tr H) U^T, the Hencky Kirchhoff stress.
__device__ __forceinline__ void hencky_stress(const Params& P, const float U[3][3], const float H[3], Sym& t) {
    const float trH = H[0] + H[1] + H[2];
    const float d[3] = {2.f * P.mu * H[0] + P.lambda * trH, 2.f * P.mu * H[1] + P.lambda * trH,
                        2.f * P.mu * H[2] + P.lambda * trH};
    t.xx = U[0][0] * U[0][0] * d[0] + U[0][1] * U[0][1] * d[1] + U[0][2] * U[0][2] * d[2];
    t.yy = U[1][0] * U[1][0] * d[0] + U[1][1] * U[1][1] * d[1] + U[1][2] * U[1][2] * d[2];
    t.zz = U[2][0] * U[2][0] * d[0] + U[2][1] * U[2][1] * d[1] + U[2][2] * U[2][2] * d[2];
    t.xy = U[0][0] * U[1][0] * d[0] + U[0][1] * U[1][1] * d[1] + U[0][2] * U[1][2] * d[2];
    t.xz = U[0][0] * U[2][0] * d[0] + U[0][1] * U[2][1] * d[1] + U[0][2] * U[2][2] * d[2];
    t.yz = U[1][0] * U[2][0] * d[0] + U[1][1] * U[2][1] * d[1] + U[1][2] * U[2][2] * d[2];
}

// Drucker-Prager return map in principal Hencky strain (Klar et al. 2016) on
// the elastic trial F, through the left stretch: with F = U diag(e^eps) V^T,
// the projected F is U diag(e^H) V^T = U diag(e^(H - eps)) U^T F, so V is
// never formed and a state inside the cone keeps its F unchanged.  Writes the
// projected F and the Hencky Kirchhoff stress.
__device__ __forceinline__ bool dp_update_eig(const Params& P, float alpha, float F[9], Sym& t) {
    float U[3][3], eps[3];
    if (!left_hencky(F, U, eps)) return false;
    const float tr = eps[0] + eps[1] + eps[2];
    const float dev[3] = {eps[0] - tr * (1.f / 3.f), eps[1] - tr * (1.f / 3.f), eps[2] - tr * (1.f / 3.f)};
    const float nd = sqrtf(dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]);
    const float dgamma = nd + (3.f * P.lambda + 2.f * P.mu) / (2.f * P.mu) * tr * alpha;
    float H[3];
    if (tr < 0.f && dgamma <= 0.f) {
        H[0] = eps[0];                               // inside the cone: F unchanged
        H[1] = eps[1];
        H[2] = eps[2];
    } else {
        if (tr >= 0.f) {
            H[0] = H[1] = H[2] = 0.f;                // tip of the cone
        } else {
            const float k = dgamma / nd;             // onto the cone, volume kept
            H[0] = eps[0] - k * dev[0];
            H[1] = eps[1] - k * dev[1];
            H[2] = eps[2] - k * dev[2];
        }
        const float s[3] = {expf(H[0] - eps[0]), expf(H[1] - eps[1]), expf(H[2] - eps[2])};
        float M[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j)
                M[i][j] = M[j][i] = U[i][0] * s[0] * U[j][0] + U[i][1] * s[1] * U[j][1] + U[i][2] * s[2] * U[j][2];
        float G[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) G[i * 3 + j] = M[i][0] * F[0 * 3 + j] + M[i][1] * F[1 * 3 + j] + M[i][2] * F[2 * 3 + j];
#pragma unroll
        for (int k = 0; k < 9; ++k) F[k] = G[k];
    }
    hencky_stress(P, U, H, t);
    return true;
}

// ---- the same return map without an eigenanalysis, for a stretch near I
//
// All the map needs are isotropic matrix functions of b = F F^T: the Hencky
// strain eps = ln(b) / 2, and, since H and eps share their eigenvectors, the
// projected F = exp(H) exp(-eps) F = exp(H - eps) F with H - eps = -k dev eps
// on the cone and -eps at its tip.  When X = b - I is small, ln(I + X) and
// exp come from their power series, with products of symmetric matrices that
// commute (polynomials in X); larger stretches take the Jacobi path above.

// A B for symmetric A and B that commute: the product is symmetric.
__device__ __forceinline__ Sym sym_mul(const Sym& a, const Sym& b) {
    Sym r;
    r.xx = a.xx * b.xx + a.xy * b.xy + a.xz * b.xz;
    r.xy = a.xx * b.xy + a.xy * b.yy + a.xz * b.yz;
    r.xz = a.xx * b.xz + a.xy * b.yz + a.xz * b.zz;
    r.yy = a.xy * b.xy + a.yy * b.yy + a.yz * b.yz;
    r.yz = a.xy * b.xz + a.yy * b.yz + a.yz * b.zz;
    r.zz = a.xz * b.xz + a.yz * b.yz + a.zz * b.zz;
    return r;
}

__device__ __forceinline__ Sym sym_axpi(const Sym& a, float s, float d) {   // s A + d I
    return Sym{s * a.xx + d, s * a.xy, s * a.xz, s * a.yy + d, s * a.yz, s * a.zz + d};
}

__device__ __forceinline__ float sym_norm2(const Sym& a) {   // squared Frobenius norm
    return a.xx * a.xx + a.yy * a.yy + a.zz * a.zz + 2.f * (a.xy * a.xy + a.xz * a.xz + a.yz * a.yz);
}

// X = F F^T - I.  The diagonal is formed as (F_ii - 1)(F_ii + 1) + the other
// two squares, so the cancellation against 1 happens exactly.
__device__ __forceinline__ Sym left_cg_minus_i(const float F[9]) {
    Sym X;
    X.xx = fmaf(F[0] - 1.f, F[0] + 1.f, F[1] * F[1] + F[2] * F[2]);
    X.yy = fmaf(F[4] - 1.f, F[4] + 1.f, F[3] * F[3] + F[5] * F[5]);
    X.zz = fmaf(F[8] - 1.f, F[8] + 1.f, F[6] * F[6] + F[7] * F[7]);
    X.xy = F[0] * F[3] + F[1] * F[4] + F[2] * F[5];
    X.xz = F[0] * F[6] + F[1] * F[7] + F[2] * F[8];
    X.yz = F[3] * F[6] + F[4] * F[7] + F[5] * F[8];
    return X;
}

// eps = ln(I + X) / 2 from X - X^2/2 + X^3/3 - X^4/4 + X^5/5 (Horner).  At
// ||X||_F <= 1/16 the first omitted term is below 2e-8 in eps.
__device__ __forceinline__ Sym hencky_series(const Sym& X) {
    Sym q = sym_axpi(X, 0.2f, -0.25f);
    q = sym_axpi(sym_mul(q, X), 1.f, 1.f / 3.f);
    q = sym_axpi(sym_mul(q, X), 1.f, -0.5f);
    q = sym_axpi(sym_mul(q, X), 1.f, 1.f);
    return sym_axpi(sym_mul(q, X), 0.5f, 0.f);
}

// exp(Y) = I + Y + Y^2/2 + Y^3/6 + Y^4/24 (Horner), for ||Y||_F <= 1/32 here,
// where the first omitted term is below 3e-10.
__device__ __forceinline__ Sym exp_series(const Sym& Y) {
    Sym e = sym_axpi(Y, 0.25f, 1.f);
    e = sym_axpi(sym_mul(Y, e), 1.f / 3.f, 1.f);
    e = sym_axpi(sym_mul(Y, e), 0.5f, 1.f);
    return sym_axpi(sym_mul(Y, e), 1.f, 1.f);
}

__device__ __forceinline__ void hencky_stress_sym(const Params& P, const Sym& H, Sym& t) {
    const float l = P.lambda * (H.xx + H.yy + H.zz), m2 = 2.f * P.mu;
    t = Sym{m2 * H.xx + l, m2 * H.xy, m2 * H.xz, m2 * H.yy + l, m2 * H.yz, m2 * H.zz + l};
}

// Drucker-Prager return map (the reading above): the series form when
// ||F F^T - I||_F <= MPM_SERIES_MAX, else the eigenanalysis.
__device__ __forceinline__ bool dp_update(const Params& P, float alpha, float F[9], Sym& t) {
    const Sym X = left_cg_minus_i(F);
    if (!(sym_norm2(X) <= MPM_SERIES_MAX * MPM_SERIES_MAX)) return dp_update_eig(P, alpha, F, t);
    if (!(det3(F) > 0.f)) return false;
    const Sym e = hencky_series(X);
    const float tr = e.xx + e.yy + e.zz;
    const Sym dev = sym_axpi(e, 1.f, -tr * (1.f / 3.f));
    const float nd = sqrtf(sym_norm2(dev));
    const float dgamma = nd + (3.f * P.lambda + 2.f * P.mu) / (2.f * P.mu) * tr * alpha;
    Sym H = e;                                       // inside the cone: F unchanged
    if (!(tr < 0.f && dgamma <= 0.f)) {
        Sym Y;                                       // H - eps
        if (tr >= 0.f) {
            Y = sym_axpi(e, -1.f, 0.f);              // tip of the cone: H = 0
            H = Sym{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        } else {
            const float k = dgamma / nd;             // onto the cone, volume kept
            Y = sym_axpi(dev, -k, 0.f);
            H = Sym{e.xx + Y.xx, e.xy + Y.xy, e.xz + Y.xz, e.yy + Y.yy, e.yz + Y.yz, e.zz + Y.zz};
        }
        const Sym E = exp_series(Y);
        const float M[9] = {E.xx, E.xy, E.xz, E.xy, E.yy, E.yz, E.xz, E.yz, E.zz};
        float G[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                G[i * 3 + j] = M[i * 3 + 0] * F[0 * 3 + j] + M[i * 3 + 1] * F[1 * 3 + j] + M[i * 3 + 2] * F[2 * 3 + j];
#pragma unroll
        for (int k = 0; k < 9; ++k) F[k] = G[k];
    }
    hencky_stress_sym(P, H, t);
    return true;
}

// Hencky stress of an F without plastic projection (initial state).
__device__ __forceinline__ bool hencky_tau(const Params& P, const float F[9], Sym& t) {
    const Sym X = left_cg_minus_i(F);
    if (sym_norm2(X) <= MPM_SERIES_MAX * MPM_SERIES_MAX) {
        if (!(det3(F) > 0.f)) return false;
        hencky_stress_sym(P, hencky_series(X), t);
        return true;
    }
    float U[3][3], eps[3];
    if (!left_hencky(F, U, eps)) return false;
    hencky_stress(P, U, eps, t);
    return true;
}

// ------------------------------------------------------------------- G2P

// Compact index of the neighbour block e = (ex, ey, ez) (each 0..R-1) of
// block r: the per-block table (sparse) or the box arithmetic (dense).
template <int B, bool DENSE>
struct Neighbours {
    static constexpr int R = (B == 4) ? 2 : 3;
    static constexpr int NNB = R * R * R;
    int q[NNB];
    __device__ __forceinline__ void load(const Params& P, const int* __restrict__ nbr, int r) {
        if (DENSE) {
            const int sx = P.nb[1] * P.nb[2], sy = P.nb[2];
#pragma unroll
            for (int e = 0; e < NNB; ++e) q[e] = r + (e / (R * R)) * sx + ((e / R) % R) * sy + (e % R);
        } else {
            if (B == 4) {
                const int4 a = __ldg(reinterpret_cast<const int4*>(nbr) + 2 * r);
                const int4 b = __ldg(reinterpret_cast<const int4*>(nbr) + 2 * r + 1);
                q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
                q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
            } else {
#pragma unroll
                for (int e = 0; e < NNB; ++e) q[e] = __ldg(&nbr[(int64_t)r * NNB + e]);
            }
        }
    }
};

// G2P: one thread per particle in sorted order, no shared memory and no
// barriers.  The 27 node velocities come from the grid through the
// neighbour table (L1-resident for the particles of one block).  The node
// sums are factored over z: for each (a, b) the three z-nodes are first
// reduced with w_z, dw_z and c w_z, then scattered into v_p, B_p and L_p.
// G2P of the particle at sorted position i (storage index p, block r).
template <int B, bool DENSE, int MAT>
__device__ __forceinline__ void g2p_particle(const float* __restrict__ ps, float* __restrict__ po, int64_t stride,
                                             int64_t p, int64_t i, int r, const int* __restrict__ nbr,
                                             const Params& P, const float4* __restrict__ gv, DevStatus* st) {
    constexpr int NC = B * B * B;
    Neighbours<B, DENSE> nb;
    nb.load(P, nbr, r);
    // planes 0 (x, alpha), 1-2 (F0..F7), 3 (F8, id, tau xx, xy)
    const float4* q4 = reinterpret_cast<const float4*>(ps) + pel4(p, 0);
    const float4 a0 = q4[0];
    float d[3];
    int loc[3];
    const float xp[3] = {a0.x, a0.y, a0.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fx = xp[a] * P.inv_h;
        const int bi = base_index(fx);
        d[a] = fx - (float)bi;
        loc[a] = bi & (B - 1);
    }
    float wx[3], dwx[3], wy[3], dwy[3], wz[3], dwz[3];
    bspline3(d[0], wx, dwx);
    bspline3(d[1], wy, dwy);
    bspline3(d[2], wz, dwz);
    float vp[3] = {0.f, 0.f, 0.f}, Bx[3] = {0.f, 0.f, 0.f}, By[3] = {0.f, 0.f, 0.f}, Bz[3] = {0.f, 0.f, 0.f};
    float Lx[3] = {0.f, 0.f, 0.f}, Ly[3] = {0.f, 0.f, 0.f}, Lz[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int lx = loc[0] + a;
        const int ex = lx / B, mx = lx % B;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int ly = loc[1] + b;
            const int ey = ly / B, my = ly % B;
            int q0, q1, q2;
            if (B == 4) {
                q0 = ex ? (ey ? nb.q[6] : nb.q[4]) : (ey ? nb.q[2] : nb.q[0]);
                q1 = ex ? (ey ? nb.q[7] : nb.q[5]) : (ey ? nb.q[3] : nb.q[1]);
                q2 = q1;
            } else {
                q0 = nb.q[(a * 3 + b) * 3 + 0];
                q1 = nb.q[(a * 3 + b) * 3 + 1];
                q2 = nb.q[(a * 3 + b) * 3 + 2];
            }
            float Sw[3] = {0.f, 0.f, 0.f}, Sd[3] = {0.f, 0.f, 0.f}, Sc[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int lz = loc[2] + c;
                const int ez = lz / B, mz = lz % B;
                const int q = (B == 4) ? (ez ? q1 : q0) : (c == 0 ? q0 : (c == 1 ? q1 : q2));
                if (!index_ok(q, P.cap_blocks, st)) continue;   // a stencil block must be in the table
                const float4 v = __ldg(&gv[(int64_t)q * NC + mx + B * (my + B * mz)]);
                Sw[0] = fmaf(wz[c], v.x, Sw[0]);
                Sw[1] = fmaf(wz[c], v.y, Sw[1]);
                Sw[2] = fmaf(wz[c], v.z, Sw[2]);
                Sd[0] = fmaf(dwz[c], v.x, Sd[0]);
                Sd[1] = fmaf(dwz[c], v.y, Sd[1]);
                Sd[2] = fmaf(dwz[c], v.z, Sd[2]);
                if (c > 0) {
                    const float cw = (float)c * wz[c];
                    Sc[0] = fmaf(cw, v.x, Sc[0]);
                    Sc[1] = fmaf(cw, v.y, Sc[1]);
                    Sc[2] = fmaf(cw, v.z, Sc[2]);
                }
            }
            const float Pw = wx[a] * wy[b];
            const float gxw = dwx[a] * wy[b], gyw = wx[a] * dwy[b];
            const float oa = (float)a - d[0], ob = (float)b - d[1];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float Q = Pw * Sw[k];
                vp[k] += Q;
                Bx[k] = fmaf(oa, Q, Bx[k]);
                By[k] = fmaf(ob, Q, By[k]);
                Bz[k] = fmaf(Pw, fmaf(-d[2], Sw[k], Sc[k]), Bz[k]);
                Lx[k] = fmaf(gxw, Sw[k], Lx[k]);
                Ly[k] = fmaf(gyw, Sw[k], Ly[k]);
                Lz[k] = fmaf(Pw, Sd[k], Lz[k]);
            }
        }
    }
    // C = B D^-1 with B = h [Bx By Bz] and D = h^2/4 I; L = [Lx Ly Lz] / h.
    // x, v and C are written before the constitutive update, so that they
    // hold no registers through it; one sum of every output tests them all
    // for NaN or infinity.
    const float cs = 4.f * P.inv_h;
    const float ls = P.dt * P.inv_h;
    float4* o4 = reinterpret_cast<float4*>(po) + pel4(i, 0);
    float sum = 0.f;
    float xo[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xo[a] = xp[a] + P.dt * vp[a];
        sum += xo[a] + vp[a];
    }
    float Cn[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Cn[3 * k + 0] = cs * Bx[k];
        Cn[3 * k + 1] = cs * By[k];
        Cn[3 * k + 2] = cs * Bz[k];
        sum += Cn[3 * k + 0] + Cn[3 * k + 1] + Cn[3 * k + 2];
    }
    o4[0] = make_float4(xo[0], xo[1], xo[2], a0.w);
    o4[5 * 32] = make_float4(vp[0], vp[1], vp[2], Cn[0]);
    o4[6 * 32] = make_float4(Cn[1], Cn[2], Cn[3], Cn[4]);
    o4[7 * 32] = make_float4(Cn[5], Cn[6], Cn[7], Cn[8]);
    const float4 a1 = q4[32], a2 = q4[2 * 32], a3 = q4[3 * 32];
    float F[9] = {a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w, a3.x}, Fn[9];
    const float L[9] = {Lx[0], Ly[0], Lz[0], Lx[1], Ly[1], Lz[1], Lx[2], Ly[2], Lz[2]};
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2)
            Fn[i2 * 3 + j2] = F[i2 * 3 + j2] + ls * (L[i2 * 3 + 0] * F[0 * 3 + j2] + L[i2 * 3 + 1] * F[1 * 3 + j2] +
                                                    L[i2 * 3 + 2] * F[2 * 3 + j2]);
    const float alpha = a0.w;
    Sym tau;
    bool ok;
    if (MAT == MPM_NEOHOOKEAN) ok = nh_tau(P, Fn, tau);
    else ok = dp_update(P, alpha, Fn, tau);
    sum += tau.xx + tau.yy + tau.zz + tau.xy + tau.xz + tau.yz;
#pragma unroll
    for (int k = 0; k < 9; ++k) sum += Fn[k];
    const bool bad = !(ok && isfinite(sum));
    o4[32] = make_float4(Fn[0], Fn[1], Fn[2], Fn[3]);
    o4[2 * 32] = make_float4(Fn[4], Fn[5], Fn[6], Fn[7]);
    o4[3 * 32] = make_float4(Fn[8], a3.y, tau.xx, tau.xy);   // a3.y: the id
    o4[4 * 32] = make_float4(tau.xz, tau.yy, tau.yz, tau.zz);
    if (bad) raise_flag(st, &st->numeric, 1u);   // after the stores, which it then does not hold back
}

// THREADS x REGS: the CTA size and the registers a thread is compiled for
// (at most REGS: 65536 / (THREADS x REGS) CTAs fit on an SM); the autotuner
// picks one pair per context.
template <int B, bool DENSE, int MAT, int THREADS, int REGS>
__global__ void __launch_bounds__(THREADS, 65536 / (THREADS * REGS)) k_g2p(const float* __restrict__ ps, float* __restrict__ po, int64_t stride,
                                              const uint32_t* __restrict__ perm, const uint32_t* __restrict__ skey,
                                              int64_t n, const int* __restrict__ nbr, Params P,
                                              const float4* __restrict__ gv, DevStatus* st) {
    constexpr int S3 = (B == 4) ? 6 : 0;
    // the permutation and key are read before the abort test (in bounds
    // whatever they hold), so that their latency overlaps it; nothing they
    // index is read before it
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t p = 0u, sk = 0u;
    if (i < n) {
        p = perm[i];
        sk = skey[i];
    }
    if (cta_aborted(st)) return;
    if (i >= n) return;
    const int r = (int)(sk >> S3);
    if (!index_ok(p, n, st) || !index_ok(r, P.cap_blocks, st)) return;
    g2p_particle<B, DENSE, MAT>(ps, po, stride, p, i, r, nbr, P, gv, st);
}


// tau (and the cone constant alpha) of an unprojected state.
__global__ void k_init_stress(float* __restrict__ ps, int64_t stride, int64_t n, Params P, DevStatus* st) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = ps[pel(p, PF + k)];
    Sym t;
    const bool ok = (P.material == MPM_NEOHOOKEAN) ? nh_tau(P, F, t) : hencky_tau(P, F, t);
    if (!ok) {
        atomicOr(&st->numeric, 1u);
        t = Sym{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    }
    ps[pel(p, PT + 0)] = t.xx;
    ps[pel(p, PT + 1)] = t.xy;
    ps[pel(p, PT + 2)] = t.xz;
    ps[pel(p, PT + 3)] = t.yy;
    ps[pel(p, PT + 4)] = t.yz;
    ps[pel(p, PT + 5)] = t.zz;
}

// End of a step: count it unless something raised the abort word.
__global__ void k_step_done(DevStatus* st) {
    if (st->abort == 0u) st->steps_done += 1u;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int NUM_SMS = 148;

}  // namespace

cudaError_t launch_p2g(mpm_ctx* c) {
    const float* ps = c->ps[c->cur];
    const uint32_t* perm = c->pval[c->sorted_sel];
    const HashView hv = hash_view(c);
    if (c->B == 1) {
        k_p2g_atomic<<<blocks_for(c->n, 256), 256, 0, c->ls>>>(ps, c->pstride, perm, c->pkey[c->sorted_sel], c->n,
                                                              c->nbr, c->P, c->gmv, c->gf, c->dstat);
        ++c->launches;
        return cudaGetLastError();
    }
    const uint8_t* cp = (counting_sort(c) && !c->det) ? c->cperm : nullptr;   // cells ordered by count (fast sparse mode)
#define MPM_CELLS(D_, T_)                                                                                         \
    k_p2g_cells<D_, T_><<<NUM_SMS * c->tune.p2g_ctas_per_sm, CellTileCfg::WARPS * 32, 0, c->ls>>>(ps, c->pstride, perm, c->bstart, c->bend, \
                                                                       c->pblocks, c->ccount, cp, c->dstat, c->P, \
                                                                       c->nbr, c->gmv, c->gf, c->tbuf, c->dstat)
    if (c->dense) {
        if (c->det) MPM_CELLS(true, true);
        else MPM_CELLS(true, false);
    } else {
        if (c->det) MPM_CELLS(false, true);
        else MPM_CELLS(false, false);
    }
#undef MPM_CELLS
    ++c->launches;
    if (c->det) {
        const int64_t cap = c->live_cap;
        if (c->dense)
            k_p2g_reduce<true><<<blocks_for(cap * 64, 256), 256, 0, c->ls>>>(cap, c->dstat, c->P, hv, c->bcoord, c->tbuf,
                                                                            c->hasp, c->gmv, c->gf);
        else
            k_p2g_reduce<false><<<blocks_for(cap * 64, 256), 256, 0, c->ls>>>(cap, c->dstat, c->P, hv, c->bcoord,
                                                                             c->tbuf, c->hasp, c->gmv, c->gf);
        ++c->launches;
    }
    return cudaGetLastError();
}

cudaError_t launch_grid_update(mpm_ctx* c) {
    const int64_t cap = c->live_cap;
    const int S3 = (c->B == 4) ? 6 : 0;
    const unsigned g = (unsigned)std::min<int64_t>(blocks_for(cap * c->B3, 256), 148 * 16);
    if (c->dense) k_grid<true><<<g, 256, 0, c->ls>>>(cap, c->dstat, c->B, S3, c->P, c->bcoord, c->gmv, c->gf, c->gv);
    else k_grid<false><<<g, 256, 0, c->ls>>>(cap, c->dstat, c->B, S3, c->P, c->bcoord, c->gmv, c->gf, c->gv);
    ++c->launches;
    return cudaGetLastError();
}

cudaError_t launch_g2p(mpm_ctx* c) {
    const float* ps = c->ps[c->cur];
    float* po = c->ps[1 - c->cur];
    const uint32_t* perm = c->pval[c->sorted_sel];
    const uint32_t* skey = c->pkey[c->sorted_sel];
    const int threads = c->tune.g2p_threads, regs = c->tune.g2p_regs;
    const unsigned g = blocks_for(c->n, threads);
#define MPM_G2P_TR(B_, D_, M_, T_, R_)                                                                          \
    k_g2p<B_, D_, M_, T_, R_><<<g, T_, 0, c->ls>>>(ps, po, c->pstride, perm, skey, c->n, c->nbr, c->P, c->gv,   \
                                                  c->dstat)
#define MPM_G2P(B_, D_, M_)                                                                                      \
    do {                                                                                                         \
        if (threads == 256) {                                                                                    \
            if (regs == 128) MPM_G2P_TR(B_, D_, M_, 256, 128);                                                   \
            else MPM_G2P_TR(B_, D_, M_, 256, 80);                                                                \
        } else {                                                                                                 \
            if (regs == 128) MPM_G2P_TR(B_, D_, M_, 128, 128);                                                   \
            else if (regs == 96) MPM_G2P_TR(B_, D_, M_, 128, 96);                                                \
            else if (regs == 80) MPM_G2P_TR(B_, D_, M_, 128, 80);                                                \
            else MPM_G2P_TR(B_, D_, M_, 128, 72);                                                                \
        }                                                                                                        \
    } while (0)
    const int mat = c->P.material;
    if (c->B == 4) {
        if (c->dense) {
            if (mat == MPM_NEOHOOKEAN) MPM_G2P(4, true, MPM_NEOHOOKEAN);
            else MPM_G2P(4, true, MPM_DRUCKER_PRAGER);
        } else {
            if (mat == MPM_NEOHOOKEAN) MPM_G2P(4, false, MPM_NEOHOOKEAN);
            else MPM_G2P(4, false, MPM_DRUCKER_PRAGER);
        }
    } else {
        if (c->dense) {
            if (mat == MPM_NEOHOOKEAN) MPM_G2P(1, true, MPM_NEOHOOKEAN);
            else MPM_G2P(1, true, MPM_DRUCKER_PRAGER);
        } else {
            if (mat == MPM_NEOHOOKEAN) MPM_G2P(1, false, MPM_NEOHOOKEAN);
            else MPM_G2P(1, false, MPM_DRUCKER_PRAGER);
        }
    }
#undef MPM_G2P
#undef MPM_G2P_TR
    ++c->launches;
    return cudaGetLastError();
}

cudaError_t launch_step_done(mpm_ctx* c) {
    k_step_done<<<1, 1, 0, c->ls>>>(c->dstat);
    ++c->launches;
    return cudaGetLastError();
}

cudaError_t launch_init_stress(mpm_ctx* c, float* buf) {
    k_init_stress<<<blocks_for(c->n, 256), 256, 0, c->st>>>(buf, c->pstride, c->n, c->P, c->dstat);
    ++c->launches;
    return cudaGetLastError();
}

}  // namespace mpm
