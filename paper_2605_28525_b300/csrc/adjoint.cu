// Hand-written adjoint (reverse mode) of one explicit MPM step, Sec. 4.1:
//
//   P2G   m_n = sum_p m_p N,  p_n = sum_p m_p N (v_p + C_p (x_n - x_p)),
//         f_n = -V0 sum_p tau_p grad N
//   grid  v^_n = p_n / m_n + dt (f_n / m_n + g), then the boundary conditions
//   G2P   v_p' = sum_n N v_n,  C_p' = 4/h^2 sum_n N v_n (x_n - x_p)^T,
//         F_p' = (I + dt sum_n v_n grad N^T) F_p,  x_p' = x_p + dt v_p',
//         tau_p' = mu (F' F'^T - I) + lambda ln J' I   (Neo-Hookean)
//
// Given the adjoint of the state after the step (x', v', C', F'; the stress
// the next step's P2G reads is folded into F' by that step's adjoint), the
// kernels below produce the adjoint of the state before it and dL/dE.  N and
// grad N depend on x_p, so the x adjoint carries the B-spline gradient and
// Hessian terms.  The grid of the step is recomputed first (rebuild, P2G,
// grid update from the saved state), in deterministic mode, so it is the grid
// the forward step used.
//
//   k_adj_g2p    per particle: adjoint of G2P; scatters the adjoint of the
//                node velocities (float atomics) and writes the particle's
//                x and F adjoints
//   k_adj_grid   per node: through the boundary conditions (Jacobians of the
//                sticky, slip and Coulomb rules) and the momentum division
//   k_adj_p2g    per particle: adjoint of P2G gathered from the 27 nodes,
//                then of the stress; dL/dE summed in double
#include <algorithm>

#include "mpm_internal.cuh"

namespace mpm {

namespace {

// Per-particle adjoint record, particle-id order: x(3) v(3) C(9) F(9).
enum : int { AX = 0, AV = 3, AC = 6, AF = 15, ANF = 24 };

__device__ __forceinline__ void spline_d(float d, float w[3], float dw[3]) {
    const float t0 = 1.5f - d, t1 = d - 1.0f, t2 = d - 0.5f;
    w[0] = 0.5f * t0 * t0;
    w[1] = 0.75f - t1 * t1;
    w[2] = 0.5f * t2 * t2;
    dw[0] = -t0;
    dw[1] = -2.0f * t1;
    dw[2] = t2;
}
// second derivatives of the three weights with respect to d
__device__ __forceinline__ float spline_dd(int a) { return a == 1 ? -2.f : 1.f; }

// Node index of stencil node (a, b, c) of a particle whose base node sits at
// cell loc of its block; q = Phi of the blocks b + {0,1}^3 (B = 4).
__device__ __forceinline__ int64_t stencil_node(const int q[8], const int loc[3], int a, int b, int c) {
    const int lx = loc[0] + a, ly = loc[1] + b, lz = loc[2] + c;
    const int e = ((lx >> 2) * 2 + (ly >> 2)) * 2 + (lz >> 2);
    return (int64_t)q[e] * 64 + (lx & 3) + 4 * ((ly & 3) + 4 * (lz & 3));
}

template <bool DENSE>
__device__ __forceinline__ void block_neighbours(const Params& P, const int* __restrict__ nbr, int r, int q[8]) {
    if (DENSE) {
        const int sx = P.nb[1] * P.nb[2], sy = P.nb[2];
#pragma unroll
        for (int e = 0; e < 8; ++e) q[e] = r + (e >> 2) * sx + ((e >> 1) & 1) * sy + (e & 1);
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) q[e] = __ldg(&nbr[(int64_t)r * 8 + e]);
    }
}

// N, grad N (1/h units applied) and the Hessian of N at stencil node (a, b, c).
struct NodeWeights {
    float N, g[3], H[3][3];
};
__device__ __forceinline__ NodeWeights node_weights(const float w[3][3], const float dw[3][3], float inv_h, int a,
                                                    int b, int c) {
    NodeWeights r;
    const int o[3] = {a, b, c};
    const float W[3] = {w[0][a], w[1][b], w[2][c]};
    const float D[3] = {dw[0][a], dw[1][b], dw[2][c]};
    r.N = W[0] * W[1] * W[2];
    r.g[0] = D[0] * W[1] * W[2] * inv_h;
    r.g[1] = W[0] * D[1] * W[2] * inv_h;
    r.g[2] = W[0] * W[1] * D[2] * inv_h;
    const float ih2 = inv_h * inv_h;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            float v;
            if (k == l) {
                v = spline_dd(o[k]);
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    if (m != k) v *= W[m];
            } else {
                v = D[k] * D[l];
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    if (m != k && m != l) v *= W[m];
            }
            r.H[k][l] = v * ih2;
        }
    return r;
}

__device__ __forceinline__ void particle_geometry(const Params& P, const float x[3], float d[3], int loc[3],
                                                  float w[3][3], float dw[3][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float fx = x[k] * P.inv_h;
        const int b = base_index(fx);
        d[k] = fx - (float)b;
        loc[k] = b & 3;
        spline_d(d[k], w[k], dw[k]);
    }
}

template <bool DENSE>
__global__ void __launch_bounds__(128) k_adj_g2p(const float* __restrict__ ps, int64_t stride,
                                                 const uint32_t* __restrict__ perm, const uint32_t* __restrict__ skey,
                                                 int64_t n, const int* __restrict__ nbr, Params P,
                                                 const float4* __restrict__ gv, const float* __restrict__ adj_next,
                                                 float* __restrict__ adj_cur, float4* __restrict__ gvbar) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = perm[i];
    const int64_t id = (int64_t)__float_as_uint(ps[PID * stride + p]);
    int q[8];
    block_neighbours<DENSE>(P, nbr, (int)(skey[i] >> 6), q);
    float x[3], F[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = ps[(PX + k) * stride + p];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = ps[(PF + k) * stride + p];
    float d[3], w[3][3], dw[3][3];
    int loc[3];
    particle_geometry(P, x, d, loc, w, dw);
    const float* an = adj_next + id * ANF;
    float xb_n[3], vb[3], Cb[9], Fb_n[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xb_n[k] = an[AX + k];
        vb[k] = an[AV + k] + P.dt * an[AX + k];   // x' = x + dt v'
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Cb[k] = an[AC + k];
        Fb_n[k] = an[AF + k];
    }
    // L = sum v_n grad N^T (forward), needed for (I + dt L)^T F'bar
    float L[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                const NodeWeights nw = node_weights(w, dw, P.inv_h, a, b, c);
                const float4 vn = gv[stencil_node(q, loc, a, b, c)];
                const float v3[3] = {vn.x, vn.y, vn.z};
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int s = 0; s < 3; ++s) L[r * 3 + s] += v3[r] * nw.g[s];
            }
    // Lbar = dt F'bar F^T
    float Lb[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s)
            Lb[r * 3 + s] = P.dt * (Fb_n[r * 3 + 0] * F[s * 3 + 0] + Fb_n[r * 3 + 1] * F[s * 3 + 1] +
                                    Fb_n[r * 3 + 2] * F[s * 3 + 2]);
    float xb[3] = {xb_n[0], xb_n[1], xb_n[2]};
    const float c4 = 4.f * P.inv_h * P.inv_h;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                const NodeWeights nw = node_weights(w, dw, P.inv_h, a, b, c);
                const int64_t node = stencil_node(q, loc, a, b, c);
                const float4 vn = gv[node];
                const float v3[3] = {vn.x, vn.y, vn.z};
                const float dx[3] = {((float)a - d[0]) * P.h, ((float)b - d[1]) * P.h, ((float)c - d[2]) * P.h};
                float Cd[3], CtV[3], LtV[3], Lg[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    Cd[r] = Cb[r * 3 + 0] * dx[0] + Cb[r * 3 + 1] * dx[1] + Cb[r * 3 + 2] * dx[2];
                    CtV[r] = Cb[0 * 3 + r] * v3[0] + Cb[1 * 3 + r] * v3[1] + Cb[2 * 3 + r] * v3[2];
                    LtV[r] = Lb[0 * 3 + r] * v3[0] + Lb[1 * 3 + r] * v3[1] + Lb[2 * 3 + r] * v3[2];
                    Lg[r] = Lb[r * 3 + 0] * nw.g[0] + Lb[r * 3 + 1] * nw.g[1] + Lb[r * 3 + 2] * nw.g[2];
                }
                // adjoint of the node velocity
                float gb[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) gb[r] = nw.N * vb[r] + c4 * nw.N * Cd[r] + Lg[r];
                atomicAdd(&gvbar[node].x, gb[0]);
                atomicAdd(&gvbar[node].y, gb[1]);
                atomicAdd(&gvbar[node].z, gb[2]);
                // adjoint of x through N, grad N and (x_n - x_p)
                const float vdot = vb[0] * v3[0] + vb[1] * v3[1] + vb[2] * v3[2];
                const float cdot = v3[0] * Cd[0] + v3[1] * Cd[1] + v3[2] * Cd[2];
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    xb[r] += nw.g[r] * (vdot + c4 * cdot) - c4 * nw.N * CtV[r] + nw.H[r][0] * LtV[0] +
                             nw.H[r][1] * LtV[1] + nw.H[r][2] * LtV[2];
            }
    float* ac = adj_cur + id * ANF;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ac[AX + k] = xb[k];
        ac[AV + k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) ac[AC + k] = 0.f;
    // F'bar through F' = (I + dt L) F
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            float v = Fb_n[r * 3 + s];
#pragma unroll
            for (int k = 0; k < 3; ++k) v += P.dt * L[k * 3 + r] * Fb_n[k * 3 + s];
            ac[AF + r * 3 + s] = v;
        }
}

// Jacobian-transpose of the Coulomb rule at velocity v (before the rule)
// with outward normal n, applied to the adjoint vb in place.
__device__ __forceinline__ void coulomb_adj(const float v[3], const float n[3], float mu, float vb[3]) {
    const float vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
    if (vn >= 0.f) return;   // unchanged: identity
    const float t[3] = {v[0] - vn * n[0], v[1] - vn * n[1], v[2] - vn * n[2]};
    const float tn = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    const float keep = tn + mu * vn;
    if (keep <= 0.f) {       // stopped
        vb[0] = vb[1] = vb[2] = 0.f;
        return;
    }
    // v' = t s, s = keep / tn: J^T vb = s (I - n n^T) vb + (mu / tn) n (t.vb) - (mu vn / tn^3) t (t.vb)
    const float s = keep / tn;
    const float tb = t[0] * vb[0] + t[1] * vb[1] + t[2] * vb[2];
    const float nb = n[0] * vb[0] + n[1] * vb[1] + n[2] * vb[2];
    float o[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        o[k] = s * (vb[k] - nb * n[k]) + (mu / tn) * n[k] * tb - (mu * vn / (tn * tn * tn)) * t[k] * tb;
    vb[0] = o[0];
    vb[1] = o[1];
    vb[2] = o[2];
}

__device__ __forceinline__ float terrain_h(const Params& P, int ti, int tj) {
    ti = min(max(ti, 0), P.terrain_nx - 1);
    tj = min(max(tj, 0), P.terrain_ny - 1);
    return P.terrain[ti + (int64_t)P.terrain_nx * tj];
}

// Coulomb rule forward (the same rule as the grid update), for the Jacobian's
// evaluation point of the next rule.
__device__ __forceinline__ void coulomb_fwd(float v[3], const float n[3], float mu) {
    const float vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
    if (vn >= 0.f) return;
    const float t[3] = {v[0] - vn * n[0], v[1] - vn * n[1], v[2] - vn * n[2]};
    const float tn = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    const float keep = tn + mu * vn;
    if (keep <= 0.f) {
        v[0] = v[1] = v[2] = 0.f;
        return;
    }
    const float s = keep / tn;
    v[0] = t[0] * s;
    v[1] = t[1] * s;
    v[2] = t[2] * s;
}

template <bool DENSE>
__global__ void __launch_bounds__(256) k_adj_grid(int64_t cap, const DevStatus* st, Params P,
                                                  const int4* __restrict__ bcoord, const float4* __restrict__ gmv,
                                                  const float4* __restrict__ gf, const float4* __restrict__ gvbar,
                                                  float4* __restrict__ gmbar, float4* __restrict__ gfbar) {
    const int64_t nn = live_blocks(st, cap) * 64;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = gmv[i];
        const float m = a.x;
        if (!(m > 0.f)) {
            gmbar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            gfbar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const int r = (int)(i >> 6), l = (int)(i & 63);
        int bc[3];
        if (DENSE) {
            rel_decode(P, (uint32_t)r, bc[0], bc[1], bc[2]);
        } else {
            const int4 b = bcoord[r];
            bc[0] = b.x;
            bc[1] = b.y;
            bc[2] = b.z;
        }
        if (P.n_scen > 1) bc[0] -= ((bc[0] - P.blo[0]) / P.ens_pitch) * P.ens_pitch;
        const int n0 = bc[0] * 4 + (l & 3), n1 = bc[1] * 4 + ((l >> 2) & 3), n2 = bc[2] * 4 + (l >> 4);
        const float4 f = gf[i];
        const float im = 1.f / m;
        // forward: the velocity before each rule
        float v0[3] = {a.y * im + P.dt * (f.x * im + P.g[0]), a.z * im + P.dt * (f.y * im + P.g[1]),
                       a.w * im + P.dt * (f.z * im + P.g[2])};
        const float z = (float)n2 * P.h;
        const bool floor_on = P.floor_kind != MPM_FLOOR_NONE && z <= P.floor_z;
        float v1[3] = {v0[0], v0[1], v0[2]};
        const float up[3] = {0.f, 0.f, 1.f};
        if (floor_on) {
            if (P.floor_kind == MPM_FLOOR_STICKY) v1[0] = v1[1] = v1[2] = 0.f;
            else if (P.floor_kind == MPM_FLOOR_SLIP) v1[2] = fmaxf(v1[2], 0.f);
            else coulomb_fwd(v1, up, P.floor_mu);
        }
        bool terr_on = false;
        float tnrm[3] = {0.f, 0.f, 1.f};
        if (P.terrain) {
            const int ti = n0 - P.lo[0], tj = n1 - P.lo[1];
            if (z <= terrain_h(P, ti, tj)) {
                terr_on = true;
                const int i0 = ti > 0 ? ti - 1 : ti, i1 = ti < P.terrain_nx - 1 ? ti + 1 : ti;
                const int j0 = tj > 0 ? tj - 1 : tj, j1 = tj < P.terrain_ny - 1 ? tj + 1 : tj;
                const float hx = (terrain_h(P, i1, tj) - terrain_h(P, i0, tj)) / ((float)(i1 - i0) * P.h);
                const float hy = (terrain_h(P, ti, j1) - terrain_h(P, ti, j0)) / ((float)(j1 - j0) * P.h);
                const float il = rsqrtf(hx * hx + hy * hy + 1.f);
                tnrm[0] = -hx * il;
                tnrm[1] = -hy * il;
                tnrm[2] = il;
            }
        }
        const int w = P.wall_layers;
        const bool wall = n0 - P.lo[0] < w || P.hi[0] - n0 < w || n1 - P.lo[1] < w || P.hi[1] - n1 < w ||
                          n2 - P.lo[2] < w || P.hi[2] - n2 < w;
        // backward through walls, terrain, floor
        const float4 gb = gvbar[i];
        float vb[3] = {gb.x, gb.y, gb.z};
        if (wall) vb[0] = vb[1] = vb[2] = 0.f;
        if (terr_on) coulomb_adj(v1, tnrm, P.terrain_mu, vb);
        if (floor_on) {
            if (P.floor_kind == MPM_FLOOR_STICKY) vb[0] = vb[1] = vb[2] = 0.f;
            else if (P.floor_kind == MPM_FLOOR_SLIP) vb[2] = v0[2] > 0.f ? vb[2] : 0.f;
            else coulomb_adj(v0, up, P.floor_mu, vb);
        }
        // v0 = p / m + dt (f / m + g)
        const float pd[3] = {a.y + P.dt * f.x, a.z + P.dt * f.y, a.w + P.dt * f.z};
        const float mb = -(pd[0] * vb[0] + pd[1] * vb[1] + pd[2] * vb[2]) * im * im;
        gmbar[i] = make_float4(mb, vb[0] * im, vb[1] * im, vb[2] * im);
        gfbar[i] = make_float4(P.dt * vb[0] * im, P.dt * vb[1] * im, P.dt * vb[2] * im, 0.f);
    }
}

template <bool DENSE>
__global__ void __launch_bounds__(128) k_adj_p2g(const float* __restrict__ ps, int64_t stride,
                                                 const uint32_t* __restrict__ perm, const uint32_t* __restrict__ skey,
                                                 int64_t n, const int* __restrict__ nbr, Params P,
                                                 const float4* __restrict__ gmbar, const float4* __restrict__ gfbar,
                                                 float* __restrict__ adj_cur, double dmu_dE, double dla_dE,
                                                 double* __restrict__ dE) {
    __shared__ double red[4];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e_part = 0.0;
    if (i < n) {
        const int64_t p = perm[i];
        const int64_t id = (int64_t)__float_as_uint(ps[PID * stride + p]);
        int q[8];
        block_neighbours<DENSE>(P, nbr, (int)(skey[i] >> 6), q);
        float x[3], v[3], C[9], F[9], t6[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            x[k] = ps[(PX + k) * stride + p];
            v[k] = ps[(PV + k) * stride + p];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            C[k] = ps[(PC + k) * stride + p];
            F[k] = ps[(PF + k) * stride + p];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) t6[k] = ps[(PT + k) * stride + p];
        const float tau[9] = {t6[0], t6[1], t6[2], t6[1], t6[3], t6[4], t6[2], t6[4], t6[5]};
        float d[3], w[3][3], dw[3][3];
        int loc[3];
        particle_geometry(P, x, d, loc, w, dw);
        const float m = P.mp, V0 = P.V0;
        float xb[3] = {0.f, 0.f, 0.f}, vb[3] = {0.f, 0.f, 0.f}, Cb[9], tb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Cb[k] = tb[k] = 0.f;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) {
                    const NodeWeights nw = node_weights(w, dw, P.inv_h, a, b, c);
                    const int64_t node = stencil_node(q, loc, a, b, c);
                    const float4 mp = gmbar[node], fb4 = gfbar[node];
                    const float pb[3] = {mp.y, mp.z, mp.w}, fb[3] = {fb4.x, fb4.y, fb4.z};
                    const float dx[3] = {((float)a - d[0]) * P.h, ((float)b - d[1]) * P.h, ((float)c - d[2]) * P.h};
                    float u[3], Ctp[3], tf[3];
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        u[r] = v[r] + C[r * 3 + 0] * dx[0] + C[r * 3 + 1] * dx[1] + C[r * 3 + 2] * dx[2];
                        Ctp[r] = C[0 * 3 + r] * pb[0] + C[1 * 3 + r] * pb[1] + C[2 * 3 + r] * pb[2];
                        tf[r] = tau[r * 3 + 0] * fb[0] + tau[r * 3 + 1] * fb[1] + tau[r * 3 + 2] * fb[2];
                    }
                    const float pu = pb[0] * u[0] + pb[1] * u[1] + pb[2] * u[2];
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        xb[r] += m * nw.g[r] * (mp.x + pu) - m * nw.N * Ctp[r] -
                                 V0 * (nw.H[r][0] * tf[0] + nw.H[r][1] * tf[1] + nw.H[r][2] * tf[2]);
                        vb[r] += m * nw.N * pb[r];
#pragma unroll
                        for (int s = 0; s < 3; ++s) {
                            Cb[r * 3 + s] += m * nw.N * pb[r] * dx[s];
                            tb[r * 3 + s] -= V0 * fb[r] * nw.g[s];
                        }
                    }
                }
        // stress: tau = mu (F F^T - I) + lambda ln J I
        //   Fbar += mu (taubar + taubar^T) F + lambda tr(taubar) F^-T
        const float J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                        F[2] * (F[3] * F[7] - F[4] * F[6]);
        const float cof[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                              F[2] * F[7] - F[1] * F[8], F[0] * F[8] - F[2] * F[6], F[1] * F[6] - F[0] * F[7],
                              F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
        const float trb = tb[0] + tb[4] + tb[8];
        float* ac = adj_cur + id * ANF;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                float sym = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) sym += (tb[r * 3 + k] + tb[k * 3 + r]) * F[k * 3 + s];
                ac[AF + r * 3 + s] += P.mu * sym + P.lambda * trb * cof[r * 3 + s] / J;
            }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ac[AX + k] += xb[k];
            ac[AV + k] += vb[k];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) ac[AC + k] += Cb[k];
        // dE: taubar : (F F^T - I) dmu/dE + tr(taubar) ln J dlambda/dE
        double bb = 0.0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const double ffT = (double)F[r * 3 + 0] * F[s * 3 + 0] + (double)F[r * 3 + 1] * F[s * 3 + 1] +
                                   (double)F[r * 3 + 2] * F[s * 3 + 2] - (r == s ? 1.0 : 0.0);
                bb += (double)tb[r * 3 + s] * ffT;
            }
        e_part = bb * dmu_dE + (double)trb * log((double)J) * dla_dE;
    }
    // block sum, one double atomic per block
    for (int o = 16; o > 0; o >>= 1) e_part += __shfl_down_sync(0xffffffffu, e_part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e_part;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(dE, red[0] + red[1] + red[2] + red[3]);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Adjoint of the step whose grid the phase calls just built (rebuild, P2G
// and grid update on the saved state, deterministic mode, B = 4).
cudaError_t launch_adjoint(mpm_ctx* c, const float* adj_next, float* adj_cur, float4* gvbar, float4* gmbar,
                           float4* gfbar, double* dE) {
    const float* ps = c->ps[c->cur];
    const uint32_t* perm = c->pval[c->sorted_sel];
    const uint32_t* skey = c->pkey[c->sorted_sel];
    const int64_t nodes = c->n_active * 64;
    cudaError_t e = cudaMemsetAsync(gvbar, 0, sizeof(float4) * nodes, c->st);
    if (e != cudaSuccess) return e;
    const unsigned g = blocks_for(c->n, 128);
    const double nu = c->cfg.nu;
    const double dmu = 1.0 / (2.0 * (1.0 + nu)), dla = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const unsigned gg = (unsigned)std::min<int64_t>(blocks_for(nodes, 256), 148 * 16);
    if (c->dense) {
        k_adj_g2p<true><<<g, 128, 0, c->st>>>(ps, c->pstride, perm, skey, c->n, c->nbr, c->P, c->gv, adj_next, adj_cur,
                                              gvbar);
        k_adj_grid<true><<<gg, 256, 0, c->st>>>(c->live_cap, c->dstat, c->P, c->bcoord, c->gmv, c->gf, gvbar, gmbar,
                                                gfbar);
        k_adj_p2g<true><<<g, 128, 0, c->st>>>(ps, c->pstride, perm, skey, c->n, c->nbr, c->P, gmbar, gfbar, adj_cur,
                                              dmu, dla, dE);
    } else {
        k_adj_g2p<false><<<g, 128, 0, c->st>>>(ps, c->pstride, perm, skey, c->n, c->nbr, c->P, c->gv, adj_next,
                                               adj_cur, gvbar);
        k_adj_grid<false><<<gg, 256, 0, c->st>>>(c->live_cap, c->dstat, c->P, c->bcoord, c->gmv, c->gf, gvbar, gmbar,
                                                 gfbar);
        k_adj_p2g<false><<<g, 128, 0, c->st>>>(ps, c->pstride, perm, skey, c->n, c->nbr, c->P, gmbar, gfbar, adj_cur,
                                               dmu, dla, dE);
    }
    c->launches += 3;
    return cudaGetLastError();
}

}  // namespace mpm
