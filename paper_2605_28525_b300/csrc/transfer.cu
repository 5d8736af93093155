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
//   k_p2g_tile    one CTA per block that holds particles.  The block's
//                 particles (sorted by cell) are staged in shared memory; work
//                 item (x-offset a, cell) sums the cell's particles into the 9
//                 nodes (a, 0..2, 0..2) in registers, then adds them to a
//                 (B+2)^3 shared tile; the tile is flushed with float4 global
//                 atomics into the active nodes of the block and its +1
//                 neighbours.  Fast; summation order varies between runs.
//   k_p2g_gather  one thread per active node; sums the particles of its 27
//                 neighbouring cells in a fixed order (cell offset, then
//                 sorted particle order = (block, cell, id)).  Deterministic,
//                 and bit-identical between the sparse and the dense grid.
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
    return hash_find(hv, pack_key(bi, bj, bk), P.max_probe);
}

__device__ __forceinline__ int first_geq(const uint32_t* __restrict__ skey, int lo, int hi, uint32_t q) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (skey[mid] < q) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------- P2G: block tile

template <int B>
struct TileCfg {
    static constexpr int T = B + 2;                 // tile edge in nodes
    static constexpr int NC = B * B * B;            // cells per block
    static constexpr int NI = 3 * NC;               // (a, cell) work items
    static constexpr int NT = (B == 4) ? 192 : 32;  // threads per CTA
    static constexpr int CH = (B == 4) ? 384 : 64;  // particles staged at once
    static constexpr int CHP = CH + CH / 8;         // padded stride (bank swizzle)
    static constexpr int SY = (B == 4) ? 8 : 3;     // tile strides (conflict-free for
    static constexpr int SZ = (B == 4) ? 68 : 9;    // 32 consecutive cells)
    static constexpr int TILE = (T - 1) * (SZ + SY) + T;
    static constexpr int R = (B == 4) ? 2 : 3;      // neighbour blocks per axis
    static constexpr int NNB = R * R * R;
};

__device__ __forceinline__ int swz(int t) { return t + (t >> 3); }

template <int B, bool DENSE>
__global__ void __launch_bounds__(TileCfg<B>::NT) k_p2g_tile(
    const float* __restrict__ ps, int64_t stride, const uint32_t* __restrict__ skey,
    const uint32_t* __restrict__ perm, const int* __restrict__ bstart, const int* __restrict__ bend,
    const int* __restrict__ pblocks, const DevStatus* __restrict__ stc, Params P, HashView hv,
    const int4* __restrict__ bcoord, float4* __restrict__ gmv, float4* __restrict__ gf, DevStatus* st) {
    using K = TileCfg<B>;
    __shared__ float s_d[3][K::CHP];
    __shared__ float s_v[3][K::CHP];
    __shared__ float s_c[9][K::CHP];
    __shared__ float s_t[6][K::CHP];
    __shared__ float s_tile[7][K::TILE];
    __shared__ int s_cs[K::NC + 1];
    __shared__ int s_nb[K::NNB];
    const int tid = threadIdx.x;
    const int nblk = (int)stc->n_pblocks;

    for (int i = tid; i < 7 * K::TILE; i += K::NT) (&s_tile[0][0])[i] = 0.f;

    for (int kb = blockIdx.x; kb < nblk; kb += gridDim.x) {
        const int r = pblocks[kb];
        const int s = bstart[r], e = bend[r];
        int bc[3];
        block_coords<DENSE>(P, bcoord, r, bc);
        if (tid < K::NNB) {
            const int jx = tid / (K::R * K::R), jy = (tid / K::R) % K::R, jz = tid % K::R;
            s_nb[tid] = block_rank<DENSE>(P, hv, bc[0] + jx, bc[1] + jy, bc[2] + jz);
        }
        for (int c = tid; c <= K::NC; c += K::NT)
            s_cs[c] = first_geq(skey, s, e, (uint32_t)r * K::NC + (uint32_t)c) - s;
        __syncthreads();

        const int np = e - s;
        for (int c0 = 0; c0 < np; c0 += K::CH) {
            const int cn = min(K::CH, np - c0);
            for (int t = tid; t < cn; t += K::NT) {
                const int64_t p = perm[s + c0 + t];
                const int q = swz(t);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float fx = ps[(PX + a) * stride + p] * P.inv_h;
                    s_d[a][q] = fx - (float)base_index(fx);    // exact
                    s_v[a][q] = ps[(PV + a) * stride + p];
                }
#pragma unroll
                for (int a = 0; a < 9; ++a) s_c[a][q] = ps[(PC + a) * stride + p] * P.h;
#pragma unroll
                for (int a = 0; a < 6; ++a) s_t[a][q] = ps[(PT + a) * stride + p];
            }
            __syncthreads();
            for (int it = tid; it < K::NI; it += K::NT) {
                const int a = it / K::NC, cell = it % K::NC;
                const int cx = cell % B, cy = (cell / B) % B, cz = cell / (B * B);
                const int lo = max(s_cs[cell], c0), hi = min(s_cs[cell + 1], c0 + cn);
                if (lo >= hi) continue;
                float acc[3][3][7];
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc)
#pragma unroll
                        for (int k = 0; k < 7; ++k) acc[b][cc][k] = 0.f;
                for (int j = lo; j < hi; ++j) {
                    const int q = swz(j - c0);
                    const float dx = s_d[0][q], dy = s_d[1][q], dz = s_d[2][q];
                    float wx, dwx, wy[3], dwy[3], wz[3], dwz[3];
                    bspline_a(dx, a, wx, dwx);
                    bspline3(dy, wy, dwy);
                    bspline3(dz, wz, dwz);
                    const float ox = (float)a - dx;
                    float hc[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) hc[k] = s_c[k][q];
                    const float t00 = s_t[0][q], t01 = s_t[1][q], t02 = s_t[2][q];
                    const float t11 = s_t[3][q], t12 = s_t[4][q], t22 = s_t[5][q];
                    const float q0x = fmaf(hc[0], ox, s_v[0][q]);
                    const float q0y = fmaf(hc[3], ox, s_v[1][q]);
                    const float q0z = fmaf(hc[6], ox, s_v[2][q]);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const float oy = (float)b - dy;
                        const float qbx = fmaf(hc[1], oy, q0x), qby = fmaf(hc[4], oy, q0y), qbz = fmaf(hc[7], oy, q0z);
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) {
                            const float oz = (float)cc - dz;
                            const float wyz = wy[b] * wz[cc];
                            const float N = wx * wyz;
                            const float gx = dwx * wyz, gy = wx * dwy[b] * wz[cc], gz = wx * wy[b] * dwz[cc];
                            const float mx = fmaf(hc[2], oz, qbx), my = fmaf(hc[5], oz, qby), mz = fmaf(hc[8], oz, qbz);
                            acc[b][cc][0] += N;
                            acc[b][cc][1] = fmaf(N, mx, acc[b][cc][1]);
                            acc[b][cc][2] = fmaf(N, my, acc[b][cc][2]);
                            acc[b][cc][3] = fmaf(N, mz, acc[b][cc][3]);
                            acc[b][cc][4] += gx * t00 + gy * t01 + gz * t02;
                            acc[b][cc][5] += gx * t01 + gy * t11 + gz * t12;
                            acc[b][cc][6] += gx * t02 + gy * t12 + gz * t22;
                        }
                    }
                }
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        const int ti = (cx + a) + K::SY * (cy + b) + K::SZ * (cz + cc);
#pragma unroll
                        for (int k = 0; k < 7; ++k) atomicAdd(&s_tile[k][ti], acc[b][cc][k]);
                    }
            }
            __syncthreads();
        }

        // flush the tile into the active nodes of this block and its neighbours
        const float fs = -P.V0 * P.inv_h;
        for (int t = tid; t < K::T * K::T * K::T; t += K::NT) {
            const int tx = t % K::T, ty = (t / K::T) % K::T, tz = t / (K::T * K::T);
            const int ti = tx + K::SY * ty + K::SZ * tz;
            float v[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                v[k] = s_tile[k][ti];
                s_tile[k][ti] = 0.f;
            }
            if (v[0] == 0.f && v[1] == 0.f && v[2] == 0.f && v[3] == 0.f && v[4] == 0.f && v[5] == 0.f &&
                v[6] == 0.f)
                continue;
            const int nbx = tx / B, nby = ty / B, nbz = tz / B;
            const int rank = s_nb[(nbx * K::R + nby) * K::R + nbz];
            if (rank < 0) {
                atomicOr(&st->map_miss, 1u);
                continue;
            }
            const int l = (tx % B) + B * ((ty % B) + B * (tz % B));
            const int64_t g = (int64_t)rank * K::NC + l;
            atomicAdd(&gmv[g], make_float4(v[0] * P.mp, v[1] * P.mp, v[2] * P.mp, v[3] * P.mp));
            atomicAdd(&gf[g], make_float4(v[4] * fs, v[5] * fs, v[6] * fs, 0.f));
        }
        __syncthreads();
    }
}

// ----------------------------------------------------- P2G: fixed order

template <int B, bool DENSE>
__global__ void __launch_bounds__(128) k_p2g_gather(
    const float* __restrict__ ps, int64_t stride, const uint32_t* __restrict__ perm,
    const int* __restrict__ cellstart, int64_t nnodes, Params P, HashView hv, const int4* __restrict__ bcoord,
    float4* __restrict__ gmv, float4* __restrict__ gf) {
    constexpr int S = (B == 4) ? 2 : 0;
    constexpr int NC = B * B * B;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnodes) return;
    const int r = (int)(i / NC), l = (int)(i % NC);
    int bc[3];
    block_coords<DENSE>(P, bcoord, r, bc);
    const int n[3] = {bc[0] * B + l % B, bc[1] * B + (l / B) % B, bc[2] * B + l / (B * B)};
    float m = 0.f, mvx = 0.f, mvy = 0.f, mvz = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                const int ci = n[0] - a, cj = n[1] - b, ck = n[2] - c;   // cell whose stencil holds n at (a,b,c)
                const int rank = block_rank<DENSE>(P, hv, ci >> S, cj >> S, ck >> S);
                if (rank < 0) continue;
                const int lc = (ci & (B - 1)) + B * ((cj & (B - 1)) + B * (ck & (B - 1)));
                const int q = rank * NC + lc;
                const int lo = cellstart[q], hi = cellstart[q + 1];
                for (int j = lo; j < hi; ++j) {
                    const int64_t p = perm[j];
                    const float dx = ps[(PX + 0) * stride + p] * P.inv_h - (float)ci;
                    const float dy = ps[(PX + 1) * stride + p] * P.inv_h - (float)cj;
                    const float dz = ps[(PX + 2) * stride + p] * P.inv_h - (float)ck;
                    float wx, dwx, wy, dwy, wz, dwz;
                    bspline_a(dx, a, wx, dwx);
                    bspline_a(dy, b, wy, dwy);
                    bspline_a(dz, c, wz, dwz);
                    const float N = wx * wy * wz;
                    const float gx = dwx * wy * wz, gy = wx * dwy * wz, gz = wx * wy * dwz;
                    const float ox = ((float)a - dx) * P.h, oy = ((float)b - dy) * P.h, oz = ((float)c - dz) * P.h;
                    const float* Cp = ps + PC * stride + p;
                    const float mx = ps[(PV + 0) * stride + p] + Cp[0] * ox + Cp[1 * stride] * oy + Cp[2 * stride] * oz;
                    const float my = ps[(PV + 1) * stride + p] + Cp[3 * stride] * ox + Cp[4 * stride] * oy + Cp[5 * stride] * oz;
                    const float mz = ps[(PV + 2) * stride + p] + Cp[6 * stride] * ox + Cp[7 * stride] * oy + Cp[8 * stride] * oz;
                    const float t00 = ps[(PT + 0) * stride + p], t01 = ps[(PT + 1) * stride + p];
                    const float t02 = ps[(PT + 2) * stride + p], t11 = ps[(PT + 3) * stride + p];
                    const float t12 = ps[(PT + 4) * stride + p], t22 = ps[(PT + 5) * stride + p];
                    m += N;
                    mvx += N * mx;
                    mvy += N * my;
                    mvz += N * mz;
                    g0 += gx * t00 + gy * t01 + gz * t02;
                    g1 += gx * t01 + gy * t11 + gz * t12;
                    g2 += gx * t02 + gy * t12 + gz * t22;
                }
            }
    const float fs = -P.V0 * P.inv_h;
    gmv[i] = make_float4(m * P.mp, mvx * P.mp, mvy * P.mp, mvz * P.mp);
    gf[i] = make_float4(g0 * fs, g1 * fs, g2 * fs, 0.f);
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
__global__ void __launch_bounds__(256) k_grid(int64_t nnodes, int B, int S3, Params P,
                                              const int4* __restrict__ bcoord, const float4* __restrict__ gmv,
                                              const float4* __restrict__ gf, float4* __restrict__ gv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnodes; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i >> S3), l = (int)(i & ((1 << S3) - 1));
        int bc[3];
        block_coords<DENSE>(P, bcoord, r, bc);
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

// One Jacobi rotation of the symmetric S in the (p, q) plane, accumulated in
// V (columns).  Standard cyclic Jacobi for symmetric eigenproblems.
template <int p, int q, int r>
__device__ __forceinline__ void jacobi_rot(float S[3][3], float V[3][3]) {
    const float spq = S[p][q];
    if (spq == 0.f) return;
    const float theta = (S[q][q] - S[p][p]) / (2.f * spq);
    const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
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

// SVD F = U diag(sig) V^T in FP32 (McAdams et al. 2011 structure: Jacobi
// eigenanalysis of F^T F for V, then an orthogonalisation of F V for U).
// sig is descending with sig[2] carrying the sign of det F.
__device__ __forceinline__ bool svd3(const float F[9], float U[3][3], float sig[3], float V[3][3]) {
    float S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            S[i][j] = F[0 * 3 + i] * F[0 * 3 + j] + F[1 * 3 + i] * F[1 * 3 + j] + F[2 * 3 + i] * F[2 * 3 + j];
            V[i][j] = (i == j) ? 1.f : 0.f;
        }
#pragma unroll
    for (int sweep = 0; sweep < 5; ++sweep) {
        jacobi_rot<0, 1, 2>(S, V);
        jacobi_rot<0, 2, 1>(S, V);
        jacobi_rot<1, 2, 0>(S, V);
    }
    float ev[3] = {S[0][0], S[1][1], S[2][2]};
    // sort eigenvalues (and columns of V) descending
#define MPM_SWAPCOL(a, b)                              \
    {                                                  \
        float te = ev[a];                              \
        ev[a] = ev[b];                                 \
        ev[b] = te;                                    \
        for (int k = 0; k < 3; ++k) {                  \
            float tv = V[k][a];                        \
            V[k][a] = V[k][b];                         \
            V[k][b] = tv;                              \
        }                                              \
    }
    if (ev[0] < ev[1]) MPM_SWAPCOL(0, 1);
    if (ev[0] < ev[2]) MPM_SWAPCOL(0, 2);
    if (ev[1] < ev[2]) MPM_SWAPCOL(1, 2);
#undef MPM_SWAPCOL
    // make V a rotation
    const float dv = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                     V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    if (dv < 0.f) {
        V[0][2] = -V[0][2];
        V[1][2] = -V[1][2];
        V[2][2] = -V[2][2];
    }
    float Bc[3][3];   // B = F V, columns b_j
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Bc[i][j] = F[i * 3 + 0] * V[0][j] + F[i * 3 + 1] * V[1][j] + F[i * 3 + 2] * V[2][j];
    const float n0 = sqrtf(Bc[0][0] * Bc[0][0] + Bc[1][0] * Bc[1][0] + Bc[2][0] * Bc[2][0]);
    if (!(n0 > 0.f)) return false;
    float u0[3] = {Bc[0][0] / n0, Bc[1][0] / n0, Bc[2][0] / n0};
    const float d01 = u0[0] * Bc[0][1] + u0[1] * Bc[1][1] + u0[2] * Bc[2][1];
    float u1[3] = {Bc[0][1] - d01 * u0[0], Bc[1][1] - d01 * u0[1], Bc[2][1] - d01 * u0[2]};
    const float n1 = sqrtf(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    if (!(n1 > 0.f)) return false;
    u1[0] /= n1;
    u1[1] /= n1;
    u1[2] /= n1;
    const float u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
    sig[0] = n0;
    sig[1] = n1;
    sig[2] = u2[0] * Bc[0][2] + u2[1] * Bc[1][2] + u2[2] * Bc[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        U[i][0] = u0[i];
        U[i][1] = u1[i];
        U[i][2] = u2[i];
    }
    return true;
}

// Drucker-Prager return map in principal Hencky strain (Klar et al. 2016) on
// the elastic trial F; writes the projected F and the Hencky Kirchhoff stress.
__device__ __forceinline__ bool dp_update(const Params& P, float alpha, float F[9], Sym& t) {
    float U[3][3], sig[3], V[3][3];
    if (!svd3(F, U, sig, V)) return false;
    if (!(sig[2] > 0.f)) return false;
    float eps[3] = {logf(sig[0]), logf(sig[1]), logf(sig[2])};
    const float tr = eps[0] + eps[1] + eps[2];
    const float dev[3] = {eps[0] - tr * (1.f / 3.f), eps[1] - tr * (1.f / 3.f), eps[2] - tr * (1.f / 3.f)};
    const float nd = sqrtf(dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]);
    const float dgamma = nd + (3.f * P.lambda + 2.f * P.mu) / (2.f * P.mu) * tr * alpha;
    float H[3];
    if (tr >= 0.f) {
        H[0] = H[1] = H[2] = 0.f;                   // tip of the cone
    } else if (dgamma <= 0.f) {
        H[0] = eps[0];                               // inside the cone
        H[1] = eps[1];
        H[2] = eps[2];
    } else {
        const float k = dgamma / nd;                 // onto the cone, volume kept
        H[0] = eps[0] - k * dev[0];
        H[1] = eps[1] - k * dev[1];
        H[2] = eps[2] - k * dev[2];
    }
    const float e[3] = {expf(H[0]), expf(H[1]), expf(H[2])};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i * 3 + j] = U[i][0] * e[0] * V[j][0] + U[i][1] * e[1] * V[j][1] + U[i][2] * e[2] * V[j][2];
    const float trH = H[0] + H[1] + H[2];
    const float d[3] = {2.f * P.mu * H[0] + P.lambda * trH, 2.f * P.mu * H[1] + P.lambda * trH,
                        2.f * P.mu * H[2] + P.lambda * trH};
    t.xx = U[0][0] * U[0][0] * d[0] + U[0][1] * U[0][1] * d[1] + U[0][2] * U[0][2] * d[2];
    t.yy = U[1][0] * U[1][0] * d[0] + U[1][1] * U[1][1] * d[1] + U[1][2] * U[1][2] * d[2];
    t.zz = U[2][0] * U[2][0] * d[0] + U[2][1] * U[2][1] * d[1] + U[2][2] * U[2][2] * d[2];
    t.xy = U[0][0] * U[1][0] * d[0] + U[0][1] * U[1][1] * d[1] + U[0][2] * U[1][2] * d[2];
    t.xz = U[0][0] * U[2][0] * d[0] + U[0][1] * U[2][1] * d[1] + U[0][2] * U[2][2] * d[2];
    t.yz = U[1][0] * U[2][0] * d[0] + U[1][1] * U[2][1] * d[1] + U[1][2] * U[2][2] * d[2];
    return true;
}

// Hencky stress of an F without plastic projection (initial state).
__device__ __forceinline__ bool hencky_tau(const Params& P, const float F[9], Sym& t) {
    float U[3][3], sig[3], V[3][3];
    if (!svd3(F, U, sig, V) || !(sig[2] > 0.f)) return false;
    const float H[3] = {logf(sig[0]), logf(sig[1]), logf(sig[2])};
    const float trH = H[0] + H[1] + H[2];
    const float d[3] = {2.f * P.mu * H[0] + P.lambda * trH, 2.f * P.mu * H[1] + P.lambda * trH,
                        2.f * P.mu * H[2] + P.lambda * trH};
    t.xx = U[0][0] * U[0][0] * d[0] + U[0][1] * U[0][1] * d[1] + U[0][2] * U[0][2] * d[2];
    t.yy = U[1][0] * U[1][0] * d[0] + U[1][1] * U[1][1] * d[1] + U[1][2] * U[1][2] * d[2];
    t.zz = U[2][0] * U[2][0] * d[0] + U[2][1] * U[2][1] * d[1] + U[2][2] * U[2][2] * d[2];
    t.xy = U[0][0] * U[1][0] * d[0] + U[0][1] * U[1][1] * d[1] + U[0][2] * U[1][2] * d[2];
    t.xz = U[0][0] * U[2][0] * d[0] + U[0][1] * U[2][1] * d[1] + U[0][2] * U[2][2] * d[2];
    t.yz = U[1][0] * U[2][0] * d[0] + U[1][1] * U[2][1] * d[1] + U[1][2] * U[2][2] * d[2];
    return true;
}

// ------------------------------------------------------------------- G2P

template <int B, bool DENSE, int MAT>
__global__ void __launch_bounds__(256) k_g2p(const float* __restrict__ ps, float* __restrict__ po, int64_t stride,
                                              const uint32_t* __restrict__ perm, const int* __restrict__ bstart,
                                              const int* __restrict__ bend, const int* __restrict__ pblocks,
                                              const DevStatus* __restrict__ stc, Params P, HashView hv,
                                              const int4* __restrict__ bcoord, const float4* __restrict__ gv,
                                              DevStatus* st) {
    constexpr int T = B + 2;
    constexpr int NC = B * B * B;
    constexpr int R = (B == 4) ? 2 : 3;
    __shared__ float4 s_v[T * T * T];
    __shared__ int s_nb[R * R * R];
    const int tid = threadIdx.x;
    const int nblk = (int)stc->n_pblocks;
    for (int kb = blockIdx.x; kb < nblk; kb += gridDim.x) {
        const int r = pblocks[kb];
        const int s = bstart[r], e = bend[r];
        int bc[3];
        block_coords<DENSE>(P, bcoord, r, bc);
        if (tid < R * R * R) {
            const int jx = tid / (R * R), jy = (tid / R) % R, jz = tid % R;
            s_nb[tid] = block_rank<DENSE>(P, hv, bc[0] + jx, bc[1] + jy, bc[2] + jz);
        }
        __syncthreads();
        for (int t = tid; t < T * T * T; t += blockDim.x) {
            const int tx = t % T, ty = (t / T) % T, tz = t / (T * T);
            const int rank = s_nb[((tx / B) * R + ty / B) * R + tz / B];
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rank >= 0) v = gv[(int64_t)rank * NC + (tx % B) + B * ((ty % B) + B * (tz % B))];
            s_v[t] = v;
        }
        __syncthreads();
        for (int i = s + tid; i < e; i += blockDim.x) {
            const int64_t p = perm[i];
            float d[3];
            int loc[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float fx = ps[(PX + a) * stride + p] * P.inv_h;
                const int bi = base_index(fx);
                d[a] = fx - (float)bi;
                loc[a] = bi - bc[a] * B;
            }
            if (loc[0] < 0 || loc[0] >= B || loc[1] < 0 || loc[1] >= B || loc[2] < 0 || loc[2] >= B) {
                atomicOr(&st->map_miss, 1u);   // cannot happen with a consistent sort
                continue;
            }
            float wx[3], dwx[3], wy[3], dwy[3], wz[3], dwz[3];
            bspline3(d[0], wx, dwx);
            bspline3(d[1], wy, dwy);
            bspline3(d[2], wz, dwz);
            float vp[3] = {0.f, 0.f, 0.f};
            float Bm[9], L[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) Bm[k] = L[k] = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float ox = (float)a - d[0];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float oy = (float)b - d[1];
                    const float wxy = wx[a] * wy[b];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float oz = (float)c - d[2];
                        const float4 vn = s_v[(loc[0] + a) + T * ((loc[1] + b) + T * (loc[2] + c))];
                        const float N = wxy * wz[c];
                        const float gx = dwx[a] * wy[b] * wz[c], gy = wx[a] * dwy[b] * wz[c], gz = wxy * dwz[c];
                        const float nvx = N * vn.x, nvy = N * vn.y, nvz = N * vn.z;
                        vp[0] += nvx;
                        vp[1] += nvy;
                        vp[2] += nvz;
                        Bm[0] = fmaf(nvx, ox, Bm[0]);
                        Bm[1] = fmaf(nvx, oy, Bm[1]);
                        Bm[2] = fmaf(nvx, oz, Bm[2]);
                        Bm[3] = fmaf(nvy, ox, Bm[3]);
                        Bm[4] = fmaf(nvy, oy, Bm[4]);
                        Bm[5] = fmaf(nvy, oz, Bm[5]);
                        Bm[6] = fmaf(nvz, ox, Bm[6]);
                        Bm[7] = fmaf(nvz, oy, Bm[7]);
                        Bm[8] = fmaf(nvz, oz, Bm[8]);
                        L[0] = fmaf(vn.x, gx, L[0]);
                        L[1] = fmaf(vn.x, gy, L[1]);
                        L[2] = fmaf(vn.x, gz, L[2]);
                        L[3] = fmaf(vn.y, gx, L[3]);
                        L[4] = fmaf(vn.y, gy, L[4]);
                        L[5] = fmaf(vn.y, gz, L[5]);
                        L[6] = fmaf(vn.z, gx, L[6]);
                        L[7] = fmaf(vn.z, gy, L[7]);
                        L[8] = fmaf(vn.z, gz, L[8]);
                    }
                }
            }
            // C = B D^-1 with B = h Bm (offsets in cells) and D = h^2/4 I
            const float cs = 4.f * P.inv_h;
            // F <- (I + dt L) F with L = (sum v (x) grad N) (1/h)
            const float ls = P.dt * P.inv_h;
            float F[9], Fn[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) F[k] = ps[(PF + k) * stride + p];
#pragma unroll
            for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
                for (int j2 = 0; j2 < 3; ++j2)
                    Fn[i2 * 3 + j2] = F[i2 * 3 + j2] + ls * (L[i2 * 3 + 0] * F[0 * 3 + j2] + L[i2 * 3 + 1] * F[1 * 3 + j2] +
                                                            L[i2 * 3 + 2] * F[2 * 3 + j2]);
            const float alpha = ps[PPHI * stride + p];
            Sym tau;
            bool ok;
            if (MAT == MPM_NEOHOOKEAN) ok = nh_tau(P, Fn, tau);
            else ok = dp_update(P, alpha, Fn, tau);
            float xo[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) xo[a] = ps[(PX + a) * stride + p] + P.dt * vp[a];
            bool fin = ok;
#pragma unroll
            for (int k = 0; k < 9; ++k) fin = fin && isfinite(Fn[k]) && isfinite(Bm[k]);
            fin = fin && isfinite(xo[0]) && isfinite(xo[1]) && isfinite(xo[2]) && isfinite(tau.xx) &&
                  isfinite(tau.yy) && isfinite(tau.zz) && isfinite(tau.xy) && isfinite(tau.xz) && isfinite(tau.yz);
            if (!fin) atomicOr(&st->numeric, 1u);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                po[(PX + a) * stride + i] = xo[a];
                po[(PV + a) * stride + i] = vp[a];
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                po[(PC + k) * stride + i] = cs * Bm[k];
                po[(PF + k) * stride + i] = Fn[k];
            }
            po[(PT + 0) * stride + i] = tau.xx;
            po[(PT + 1) * stride + i] = tau.xy;
            po[(PT + 2) * stride + i] = tau.xz;
            po[(PT + 3) * stride + i] = tau.yy;
            po[(PT + 4) * stride + i] = tau.yz;
            po[(PT + 5) * stride + i] = tau.zz;
            po[PPHI * stride + i] = alpha;
            po[PID * stride + i] = ps[PID * stride + p];
        }
        __syncthreads();
    }
}

// tau (and the cone constant alpha) of an unprojected state.
__global__ void k_init_stress(float* __restrict__ ps, int64_t stride, int64_t n, Params P, DevStatus* st) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = ps[(PF + k) * stride + p];
    Sym t;
    const bool ok = (P.material == MPM_NEOHOOKEAN) ? nh_tau(P, F, t) : hencky_tau(P, F, t);
    if (!ok) {
        atomicOr(&st->numeric, 1u);
        t = Sym{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    }
    ps[(PT + 0) * stride + p] = t.xx;
    ps[(PT + 1) * stride + p] = t.xy;
    ps[(PT + 2) * stride + p] = t.xz;
    ps[(PT + 3) * stride + p] = t.yy;
    ps[(PT + 4) * stride + p] = t.yz;
    ps[(PT + 5) * stride + p] = t.zz;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int PERSIST = 148 * 8;   // CTAs for the block loops (grid-stride over a device count)

}  // namespace

cudaError_t launch_p2g(mpm_ctx* c) {
    const float* ps = c->ps[c->cur];
    const uint32_t* skey = c->pkey[c->sorted_sel];
    const uint32_t* perm = c->pval[c->sorted_sel];
    HashView hv{c->hkeys, c->hvals, (uint64_t)(c->H ? c->H - 1 : 0)};
    if (c->det) {
        const int64_t nn = c->n_active * c->B3;
#define MPM_GATHER(B_, D_)                                                                                     \
    k_p2g_gather<B_, D_><<<blocks_for(nn, 128), 128, 0, c->st>>>(ps, c->pstride, perm, c->cellstart, nn, c->P, \
                                                                  hv, c->bcoord, c->gmv, c->gf)
        if (c->B == 4) {
            if (c->dense) MPM_GATHER(4, true);
            else MPM_GATHER(4, false);
        } else {
            if (c->dense) MPM_GATHER(1, true);
            else MPM_GATHER(1, false);
        }
#undef MPM_GATHER
        ++c->launches;
        return cudaGetLastError();
    }
#define MPM_TILE(B_, D_)                                                                                             \
    k_p2g_tile<B_, D_><<<PERSIST, TileCfg<B_>::NT, 0, c->st>>>(ps, c->pstride, skey, perm, c->bstart, c->bend,     \
                                                                c->pblocks, c->dstat, c->P, hv, c->bcoord, c->gmv, \
                                                                c->gf, c->dstat)
    if (c->B == 4) {
        if (c->dense) MPM_TILE(4, true);
        else MPM_TILE(4, false);
    } else {
        if (c->dense) MPM_TILE(1, true);
        else MPM_TILE(1, false);
    }
#undef MPM_TILE
    ++c->launches;
    return cudaGetLastError();
}

cudaError_t launch_grid_update(mpm_ctx* c) {
    const int64_t nn = c->n_active * c->B3;
    const int S3 = (c->B == 4) ? 6 : 0;
    const unsigned g = (unsigned)std::min<int64_t>(blocks_for(nn, 256), 148 * 16);
    if (c->dense) k_grid<true><<<g, 256, 0, c->st>>>(nn, c->B, S3, c->P, c->bcoord, c->gmv, c->gf, c->gv);
    else k_grid<false><<<g, 256, 0, c->st>>>(nn, c->B, S3, c->P, c->bcoord, c->gmv, c->gf, c->gv);
    ++c->launches;
    return cudaGetLastError();
}

cudaError_t launch_g2p(mpm_ctx* c) {
    const float* ps = c->ps[c->cur];
    float* po = c->ps[1 - c->cur];
    const uint32_t* perm = c->pval[c->sorted_sel];
    HashView hv{c->hkeys, c->hvals, (uint64_t)(c->H ? c->H - 1 : 0)};
    const int nt = (c->B == 4) ? 256 : 32;
#define MPM_G2P(B_, D_, M_)                                                                                          \
    k_g2p<B_, D_, M_><<<PERSIST, nt, 0, c->st>>>(ps, po, c->pstride, perm, c->bstart, c->bend, c->pblocks, c->dstat, \
                                                  c->P, hv, c->bcoord, c->gv, c->dstat)
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
    ++c->launches;
    return cudaGetLastError();
}

cudaError_t launch_init_stress(mpm_ctx* c, float* buf) {
    k_init_stress<<<blocks_for(c->n, 256), 256, 0, c->st>>>(buf, c->pstride, c->n, c->P, c->dstat);
    ++c->launches;
    return cudaGetLastError();
}

}  // namespace mpm
