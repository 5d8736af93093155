// Hand-written adjoint (reverse mode) of one explicit MPM step, Sec. 4.1:
//
//   P2G   m_n = sum_p m_p N,  p_n = sum_p m_p N (v_p + C_p (x_n - x_p)),
//         f_n = -V0 sum_p tau_p grad N
//   grid  v^_n = p_n / m_n + dt (f_n / m_n + g), then the boundary conditions
//   G2P   v_p' = sum_n N v_n,  C_p' = 4/h^2 sum_n N v_n (x_n - x_p)^T,
//         F_p' = (I + dt sum_n v_n grad N^T) F_p,  x_p' = x_p + dt v_p',
//         tau_p' = mu (F' F'^T - I) + lambda ln J' I   (Neo-Hookean), or for
//         Drucker-Prager F' = U exp(H(ln S)) V^T (the return map of F_tr =
//         U S V^T) and tau' = U diag(2 mu H + lambda tr H) U^T
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
//
// The Drucker-Prager return map and the Hencky stress are isotropic functions
// of F.  Their adjoints come from the SVD differential: with P = U^T dF V,
// a function U diag(g(S)) V^T has the differential U K V^T with
// K_ii = sum_j dg_i/dS_j P_jj and, for i != j, K_ij = a P_ij + b P_ji,
// a, b = ((g_i - g_j)/(S_i - S_j) +- (g_i + g_j)/(S_i + S_j)) / 2, and the
// stress U diag(s) U^T has off-diagonal terms
// (s_j - s_i)/(S_j - S_i) (S_j P_ij + S_i P_ji)/(S_i + S_j).  The divided
// differences are taken in FP64 on an FP64 SVD of the FP32 state, with their
// limits where two singular values coincide.
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

// ---------------------------------------------------------- FP64 SVD

// One Jacobi rotation of the symmetric S in the (p, q) plane, accumulated
// in the columns of V (classical formulas, t = the smaller root).
__device__ void djacobi(double S[3][3], double V[3][3], int p, int q) {
    const double spq = S[p][q];
    if (fabs(spq) <= 1e-300) return;
    const double theta = (S[q][q] - S[p][p]) / (2.0 * spq);
    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
    const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
    for (int k = 0; k < 3; ++k) {
        const double skp = S[k][p], skq = S[k][q];
        S[k][p] = c * skp - s * skq;
        S[k][q] = s * skp + c * skq;
    }
    for (int k = 0; k < 3; ++k) {
        const double spk = S[p][k], sqk = S[q][k];
        S[p][k] = c * spk - s * sqk;
        S[q][k] = s * spk + c * sqk;
    }
    for (int k = 0; k < 3; ++k) {
        const double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
    }
}

// F = U diag(sg) V^T with U, V rotations and sg descending (sg[2] carries
// the sign of det F); Jacobi eigenanalysis of F^T F for V, then U by
// orthonormalising F V.  False for a rank-deficient F.
__device__ bool dsvd3(const float Ff[9], double U[3][3], double sg[3], double V[3][3]) {
    double F[9], S[3][3];
    for (int k = 0; k < 9; ++k) F[k] = (double)Ff[k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            S[i][j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
            V[i][j] = i == j ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 10; ++sweep) {   // quadratic convergence: a few sweeps reach FP64 rounding
        const double off = fabs(S[0][1]) + fabs(S[0][2]) + fabs(S[1][2]);
        if (off <= 1e-16 * (fabs(S[0][0]) + fabs(S[1][1]) + fabs(S[2][2]))) break;
        djacobi(S, V, 0, 1);
        djacobi(S, V, 0, 2);
        djacobi(S, V, 1, 2);
    }
    double ev[3] = {S[0][0], S[1][1], S[2][2]};
    for (int a = 0; a < 2; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (ev[a] < ev[b]) {
                const double t = ev[a];
                ev[a] = ev[b];
                ev[b] = t;
                for (int k = 0; k < 3; ++k) {
                    const double tv = V[k][a];
                    V[k][a] = V[k][b];
                    V[k][b] = tv;
                }
            }
    const double dv = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
                      V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                      V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    if (dv < 0.0)
        for (int k = 0; k < 3; ++k) V[k][2] = -V[k][2];
    double Bc[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Bc[i][j] = F[i * 3] * V[0][j] + F[i * 3 + 1] * V[1][j] + F[i * 3 + 2] * V[2][j];
    const double n0 = sqrt(Bc[0][0] * Bc[0][0] + Bc[1][0] * Bc[1][0] + Bc[2][0] * Bc[2][0]);
    if (!(n0 > 0.0)) return false;
    const double u0[3] = {Bc[0][0] / n0, Bc[1][0] / n0, Bc[2][0] / n0};
    const double d01 = u0[0] * Bc[0][1] + u0[1] * Bc[1][1] + u0[2] * Bc[2][1];
    double u1[3] = {Bc[0][1] - d01 * u0[0], Bc[1][1] - d01 * u0[1], Bc[2][1] - d01 * u0[2]};
    const double n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    if (!(n1 > 0.0)) return false;
    for (int k = 0; k < 3; ++k) u1[k] /= n1;
    const double u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
    sg[0] = n0;
    sg[1] = n1;
    sg[2] = u2[0] * Bc[0][2] + u2[1] * Bc[1][2] + u2[2] * Bc[2][2];
    for (int i = 0; i < 3; ++i) {
        U[i][0] = u0[i];
        U[i][1] = u1[i];
        U[i][2] = u2[i];
    }
    return true;
}

// (a_i - a_j) / (x_i - x_j), or lim when the x are (nearly) equal.
__device__ __forceinline__ double ddiff(double ai, double aj, double xi, double xj, double lim) {
    const double dx = xi - xj;
    return fabs(dx) > 1e-10 * fmax(fabs(xi), fabs(xj)) ? (ai - aj) / dx : lim;
}

// The forward's Drucker-Prager return map in principal stretches:
// g_i = exp(H_i(ln sg)), its Jacobian Jg[i][j] = dg_i/dsg_j and dg/dalpha.
__device__ void dp_map(const double sg[3], double alpha, double kappa, double g[3], double Jg[3][3],
                       double dga[3]) {
    double e[3], dev[3];
    for (int k = 0; k < 3; ++k) e[k] = log(sg[k]);
    const double tr = e[0] + e[1] + e[2];
    for (int k = 0; k < 3; ++k) dev[k] = e[k] - tr / 3.0;
    const double nd = sqrt(dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]);
    const double dgam = nd + kappa * tr * alpha;
    double H[3], dH[3][3], dHa[3];
    if (tr >= 0.0) {                      // tip of the cone
        for (int i = 0; i < 3; ++i) {
            H[i] = 0.0;
            dHa[i] = 0.0;
            for (int j = 0; j < 3; ++j) dH[i][j] = 0.0;
        }
    } else if (dgam <= 0.0) {             // inside the cone
        for (int i = 0; i < 3; ++i) {
            H[i] = e[i];
            dHa[i] = 0.0;
            for (int j = 0; j < 3; ++j) dH[i][j] = i == j ? 1.0 : 0.0;
        }
    } else {                              // onto the cone: H = tr/3 - beta dev
        const double beta = kappa * alpha * tr / nd;
        for (int i = 0; i < 3; ++i) {
            H[i] = tr / 3.0 - beta * dev[i];
            dHa[i] = -(kappa * tr / nd) * dev[i];
            for (int j = 0; j < 3; ++j) {
                const double dbeta = kappa * alpha * (1.0 / nd - tr * dev[j] / (nd * nd * nd));
                dH[i][j] = 1.0 / 3.0 - (dbeta * dev[i] + beta * ((i == j ? 1.0 : 0.0) - 1.0 / 3.0));
            }
        }
    }
    for (int i = 0; i < 3; ++i) {
        g[i] = exp(H[i]);
        dga[i] = g[i] * dHa[i];
        for (int j = 0; j < 3; ++j) Jg[i][j] = g[i] * dH[i][j] / sg[j];
    }
}

// Fbar_tr = (d returnmap / dF at F_tr)^T Fbar' and dL/dalpha.  False if F_tr
// has no usable SVD (the forward step would have failed).
__device__ bool dp_map_adjoint(const float Ftr[9], double alpha, double kappa, const float Fb[9], float Fb_tr[9],
                               double* abar) {
    double U[3][3], sg[3], V[3][3];
    if (!dsvd3(Ftr, U, sg, V) || !(sg[2] > 0.0)) return false;
    double g[3], Jg[3][3], dga[3];
    dp_map(sg, alpha, kappa, g, Jg, dga);
    double Gb[3][3];   // U^T Fbar V
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) v += U[k][i] * (double)Fb[k * 3 + l] * V[l][j];
            Gb[i][j] = v;
        }
    double M[3][3];
    for (int i = 0; i < 3; ++i) {
        double v = 0.0;
        for (int j = 0; j < 3; ++j) v += Gb[j][j] * Jg[j][i];
        M[i][i] = v;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (i == j) continue;
            const double lim = 0.5 * ((Jg[i][i] - Jg[j][i]) + (Jg[j][j] - Jg[i][j]));
            const double q = ddiff(g[i], g[j], sg[i], sg[j], lim);
            const double r = (g[i] + g[j]) / (sg[i] + sg[j]);
            M[i][j] = 0.5 * (q + r) * Gb[i][j] + 0.5 * (q - r) * Gb[j][i];
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) v += U[a][i] * M[i][j] * V[b][j];
            Fb_tr[a * 3 + b] = (float)v;
        }
    *abar = Gb[0][0] * dga[0] + Gb[1][1] * dga[1] + Gb[2][2] * dga[2];
    return true;
}

// Hencky stress tau = U diag(2 mu ln sg + lambda sum ln sg) U^T of the
// elastic F: adds (dtau/dF)^T taubar to Fbar; returns taubar : dtau/dE.
__device__ double hencky_adjoint(const float Ff[9], const float tb[9], double mu, double la, double dmu, double dla,
                                 float Fb[9]) {
    double U[3][3], sg[3], V[3][3];
    if (!dsvd3(Ff, U, sg, V) || !(sg[2] > 0.0)) return 0.0;
    const double ls[3] = {log(sg[0]), log(sg[1]), log(sg[2])};
    const double trl = ls[0] + ls[1] + ls[2];
    double T[3][3];   // U^T taubar U
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) v += U[k][i] * (double)tb[k * 3 + l] * U[l][j];
            T[i][j] = v;
        }
    double M[3][3];
    for (int i = 0; i < 3; ++i) {
        double v = 0.0;   // sum_j T_jj ds_j/dsg_i, ds_j/dsg_i = (2 mu delta_ij + lambda) / sg_i
        for (int j = 0; j < 3; ++j) v += T[j][j] * ((i == j ? 2.0 * mu : 0.0) + la) / sg[i];
        M[i][i] = v;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (i == j) continue;
            // (s_j - s_i) / (sg_j - sg_i) = 2 mu (ln sg_j - ln sg_i) / (sg_j - sg_i)
            const double c = 2.0 * mu * ddiff(ls[j], ls[i], sg[j], sg[i], 2.0 / (sg[i] + sg[j]));
            M[i][j] = c * sg[j] * (T[i][j] + T[j][i]) / (sg[i] + sg[j]);
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) v += U[a][i] * M[i][j] * V[b][j];
            Fb[a * 3 + b] += (float)v;
        }
    return 2.0 * (T[0][0] * ls[0] + T[1][1] * ls[1] + T[2][2] * ls[2]) * dmu + (T[0][0] + T[1][1] + T[2][2]) * trl * dla;
}

// ---- the series forms (the forward's path when ||F F^T - I||_F <= 1/16)
//
// The forward evaluates the Hencky strain as eps = ln(I + X) / 2, X = F F^T - I,
// by a fifth-order power series and the projected F as exp(Y) F_tr by a
// fourth-order one, both in Horner form.  Their adjoints below run the same
// Horner steps backwards in FP32: every step is a matrix product, so there is
// no divided difference of singular values to lose precision in.  Matrices
// are full 3x3, row-major.

constexpr float ADJ_SERIES_MAX2 = MPM_SERIES_MAX * MPM_SERIES_MAX;   // the forward's threshold, squared

__device__ __forceinline__ void mm3(const float A[9], const float B[9], float C[9]) {   // C = A B
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) C[i * 3 + j] = A[i * 3] * B[j] + A[i * 3 + 1] * B[3 + j] + A[i * 3 + 2] * B[6 + j];
}

__device__ __forceinline__ void mm3_add(const float A[9], const float B[9], float s, float C[9]) {   // C += s A B
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C[i * 3 + j] += s * (A[i * 3] * B[j] + A[i * 3 + 1] * B[3 + j] + A[i * 3 + 2] * B[6 + j]);
}

__device__ __forceinline__ void axpi3(const float A[9], float s, float d, float C[9]) {   // C = s A + d I
#pragma unroll
    for (int k = 0; k < 9; ++k) C[k] = s * A[k] + ((k % 4 == 0) ? d : 0.f);
}

// X = F F^T - I (diagonal as (F_ii - 1)(F_ii + 1) + the other two squares)
// and its squared Frobenius norm.
__device__ __forceinline__ float cg_minus_i(const float F[9], float X[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (i == j) {
                const int a = (i + 1) % 3, b = (i + 2) % 3;
                X[i * 4] = fmaf(F[i * 4] - 1.f, F[i * 4] + 1.f, F[i * 3 + a] * F[i * 3 + a] + F[i * 3 + b] * F[i * 3 + b]);
            } else {
                X[i * 3 + j] = F[i * 3] * F[j * 3] + F[i * 3 + 1] * F[j * 3 + 1] + F[i * 3 + 2] * F[j * 3 + 2];
            }
        }
    float n2 = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) n2 += X[k] * X[k];
    return n2;
}

// Forward: eps = q4 X / 2 with q1 = X/5 - I/4, q2 = q1 X + I/3,
// q3 = q2 X - I/2, q4 = q3 X + I (the intermediates are kept for the adjoint).
struct LogSeries {
    float q1[9], q2[9], q3[9], q4[9];
    __device__ __forceinline__ void eval(const float X[9], float eps[9]) {
        float t[9];
        axpi3(X, 0.2f, -0.25f, q1);
        mm3(q1, X, t);
        axpi3(t, 1.f, 1.f / 3.f, q2);
        mm3(q2, X, t);
        axpi3(t, 1.f, -0.5f, q3);
        mm3(q3, X, t);
        axpi3(t, 1.f, 1.f, q4);
        mm3(q4, X, t);
        axpi3(t, 0.5f, 0.f, eps);
    }
    // Xbar from epsbar (C = A B gives Abar = Cbar B^T, Bbar = A^T Cbar; all
    // forward matrices are symmetric)
    __device__ __forceinline__ void adjoint(const float X[9], const float eb[9], float Xb[9]) const {
        float b4[9], b3[9], b2[9], b1[9];
        mm3(eb, X, b4);
#pragma unroll
        for (int k = 0; k < 9; ++k) b4[k] *= 0.5f;
        mm3(q4, eb, Xb);
#pragma unroll
        for (int k = 0; k < 9; ++k) Xb[k] *= 0.5f;
        mm3(b4, X, b3);
        mm3_add(q3, b4, 1.f, Xb);
        mm3(b3, X, b2);
        mm3_add(q2, b3, 1.f, Xb);
        mm3(b2, X, b1);
        mm3_add(q1, b2, 1.f, Xb);
#pragma unroll
        for (int k = 0; k < 9; ++k) Xb[k] += 0.2f * b1[k];
    }
};

// Forward: E = I + Y e3, e3 = I + Y e2 / 2, e2 = I + Y e1 / 3, e1 = I + Y / 4.
struct ExpSeries {
    float e1[9], e2[9], e3[9];
    __device__ __forceinline__ void eval(const float Y[9], float E[9]) {
        float t[9];
        axpi3(Y, 0.25f, 1.f, e1);
        mm3(Y, e1, t);
        axpi3(t, 1.f / 3.f, 1.f, e2);
        mm3(Y, e2, t);
        axpi3(t, 0.5f, 1.f, e3);
        mm3(Y, e3, t);
        axpi3(t, 1.f, 1.f, E);
    }
    __device__ __forceinline__ void adjoint(const float Y[9], const float Eb[9], float Yb[9]) const {
        float b3[9], b2[9], b1[9];
        mm3(Eb, e3, Yb);
        mm3(Y, Eb, b3);
        mm3_add(b3, e2, 0.5f, Yb);
        mm3(Y, b3, b2);
#pragma unroll
        for (int k = 0; k < 9; ++k) b2[k] *= 0.5f;
        mm3_add(b2, e1, 1.f / 3.f, Yb);
        mm3(Y, b2, b1);
#pragma unroll
        for (int k = 0; k < 9; ++k) Yb[k] += 0.25f * (1.f / 3.f) * b1[k];
    }
};

// Fbar += (Xbar + Xbar^T) F, the adjoint of X = F F^T - I.
__device__ __forceinline__ void cg_adjoint(const float F[9], const float Xb[9], float Fb[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) v += (Xb[i * 3 + k] + Xb[k * 3 + i]) * F[k * 3 + j];
            Fb[i * 3 + j] += v;
        }
}

// The return map's adjoint in the series form: Fbar_tr and dL/dalpha from
// Fbar' (the same contract as dp_map_adjoint).  False outside the series
// range or for det F_tr <= 0.
__device__ bool dp_map_adjoint_series(const float Ftr[9], float alpha, float kappa, const float Fb[9], float Fb_tr[9],
                                      double* abar) {
    float X[9];
    if (!(cg_minus_i(Ftr, X) <= ADJ_SERIES_MAX2)) return false;
    const float J = Ftr[0] * (Ftr[4] * Ftr[8] - Ftr[5] * Ftr[7]) - Ftr[1] * (Ftr[3] * Ftr[8] - Ftr[5] * Ftr[6]) +
                    Ftr[2] * (Ftr[3] * Ftr[7] - Ftr[4] * Ftr[6]);
    if (!(J > 0.f)) return false;
    LogSeries ls;
    float e[9];
    ls.eval(X, e);
    const float tr = e[0] + e[4] + e[8];
    float dev[9];
    axpi3(e, 1.f, -tr / 3.f, dev);
    float nd2 = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) nd2 += dev[k] * dev[k];
    const float nd = sqrtf(nd2);
    const float dgam = nd + kappa * tr * alpha;
    *abar = 0.0;
    if (tr < 0.f && dgam <= 0.f) {   // inside the cone: F' = F_tr
#pragma unroll
        for (int k = 0; k < 9; ++k) Fb_tr[k] = Fb[k];
        return true;
    }
    const bool tip = tr >= 0.f;
    const float kk = tip ? 0.f : dgam / nd;
    float Y[9];
    if (tip) axpi3(e, -1.f, 0.f, Y);
    else axpi3(dev, -kk, 0.f, Y);
    ExpSeries es;
    float E[9];
    es.eval(Y, E);
    // F' = E F_tr: Fbar_tr = E^T Fbar' = E Fbar', Ebar = Fbar' F_tr^T
    mm3(E, Fb, Fb_tr);
    float Eb[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Eb[i * 3 + j] = Fb[i * 3] * Ftr[j * 3] + Fb[i * 3 + 1] * Ftr[j * 3 + 1] + Fb[i * 3 + 2] * Ftr[j * 3 + 2];
    float Yb[9];
    es.adjoint(Y, Eb, Yb);
    float eb[9];
    if (tip) {
        axpi3(Yb, -1.f, 0.f, eb);                    // Y = -eps
    } else {
        // Y = -k dev, k = 1 + kappa alpha tr / nd, nd = ||dev||, dev = eps - tr/3 I
        float kb = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) kb -= Yb[k] * dev[k];
        const float trb = kb * kappa * alpha / nd;
        const float ndb = -kb * kappa * alpha * tr / (nd * nd);
        *abar = (double)(kb * kappa * tr / nd);
        float devb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) devb[k] = -kk * Yb[k] + ndb * dev[k] / nd;
        const float trd = devb[0] + devb[4] + devb[8];
        axpi3(devb, 1.f, trb - trd / 3.f, eb);
    }
    float Xb[9];
    ls.adjoint(X, eb, Xb);
    cg_adjoint(Ftr, Xb, Fb_tr);
    return true;
}

// The Hencky stress adjoint in the series form (the same contract as
// hencky_adjoint); false outside the series range or for det F <= 0, where
// the caller takes the eigen form.
__device__ bool hencky_adjoint_series(const float F[9], const float tb[9], float mu, float la, double dmu, double dla,
                                      float Fb[9], double* e_part) {
    float X[9];
    if (!(cg_minus_i(F, X) <= ADJ_SERIES_MAX2)) return false;
    const float J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                    F[2] * (F[3] * F[7] - F[4] * F[6]);
    if (!(J > 0.f)) return false;
    LogSeries ls;
    float e[9];
    ls.eval(X, e);
    // tau = 2 mu eps + lambda tr(eps) I: epsbar = 2 mu taubar + lambda tr(taubar) I
    const float trt = tb[0] + tb[4] + tb[8];
    float eb[9];
    axpi3(tb, 2.f * mu, la * trt, eb);
    float Xb[9];
    ls.adjoint(X, eb, Xb);
    cg_adjoint(F, Xb, Fb);
    double te = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) te += (double)tb[k] * (double)e[k];
    *e_part = 2.0 * te * dmu + (double)trt * (double)(e[0] + e[4] + e[8]) * dla;
    return true;
}

// d alpha / d phi (phi in degrees) for alpha = sqrt(2/3) 2 sin phi / (3 - sin phi).
__device__ __forceinline__ double dalpha_dphi(double alpha) {
    const double k = 0.816496580927726 * 2.0;     // sqrt(2/3) * 2
    const double sp = 3.0 * alpha / (k + alpha);  // sin phi
    const double cp = sqrt(fmax(0.0, 1.0 - sp * sp));
    return k * 3.0 * cp / ((3.0 - sp) * (3.0 - sp)) * (3.141592653589793 / 180.0);
}

template <bool DENSE, int MAT>
__global__ void __launch_bounds__(128) k_adj_g2p(const float* __restrict__ ps, int64_t stride,
                                                 const uint32_t* __restrict__ perm, const uint32_t* __restrict__ skey,
                                                 int64_t n, const int* __restrict__ nbr, Params P,
                                                 const float4* __restrict__ gv, const float* __restrict__ adj_next,
                                                 float* __restrict__ adj_cur, float4* __restrict__ gvbar,
                                                 double kappa, double* __restrict__ dphi) {
    __shared__ double red[4];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double phi_part = 0.0;
    if (i < n) {
    const int64_t p = perm[i];
    const int64_t id = (int64_t)__float_as_uint(ps[pel(p, PID)]);
    int q[8];
    block_neighbours<DENSE>(P, nbr, (int)(skey[i] >> 6), q);
    float x[3], F[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = ps[pel(p, PX + k)];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = ps[pel(p, PF + k)];
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
    if (MAT == MPM_DRUCKER_PRAGER) {
        // F' is the return map of F_tr = (I + dt L) F: Fbar_tr = (dF'/dF_tr)^T Fbar'
        float Ftr[9], Fbt[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                float v = F[r * 3 + s];
#pragma unroll
                for (int k = 0; k < 3; ++k) v += P.dt * L[r * 3 + k] * F[k * 3 + s];
                Ftr[r * 3 + s] = v;
            }
        double abar = 0.0;
        const double alpha = (double)ps[pel(p, PPHI)];
        if (dp_map_adjoint_series(Ftr, (float)alpha, (float)kappa, Fb_n, Fbt, &abar) ||
            dp_map_adjoint(Ftr, alpha, kappa, Fb_n, Fbt, &abar)) {
#pragma unroll
            for (int k = 0; k < 9; ++k) Fb_n[k] = Fbt[k];
            phi_part = abar * dalpha_dphi(alpha);
        }
    }
    // Lbar = dt F_tr-bar F^T
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
    if (MAT == MPM_DRUCKER_PRAGER) {   // block sum of dL/dphi, one double atomic per block
        for (int o = 16; o > 0; o >>= 1) phi_part += __shfl_down_sync(0xffffffffu, phi_part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = phi_part;
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(dphi, red[0] + red[1] + red[2] + red[3]);
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

template <bool DENSE, int MAT>
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
        const int64_t id = (int64_t)__float_as_uint(ps[pel(p, PID)]);
        int q[8];
        block_neighbours<DENSE>(P, nbr, (int)(skey[i] >> 6), q);
        float x[3], v[3], C[9], F[9], t6[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            x[k] = ps[pel(p, PX + k)];
            v[k] = ps[pel(p, PV + k)];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            C[k] = ps[pel(p, PC + k)];
            F[k] = ps[pel(p, PF + k)];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) t6[k] = ps[pel(p, PT + k)];
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
        float* ac = adj_cur + id * ANF;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ac[AX + k] += xb[k];
            ac[AV + k] += vb[k];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) ac[AC + k] += Cb[k];
        if (MAT == MPM_DRUCKER_PRAGER) {
            // Hencky stress of the stored elastic F
            float Fbs[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) Fbs[k] = ac[AF + k];
            if (!hencky_adjoint_series(F, tb, P.mu, P.lambda, dmu_dE, dla_dE, Fbs, &e_part))
                e_part = hencky_adjoint(F, tb, (double)P.mu, (double)P.lambda, dmu_dE, dla_dE, Fbs);
#pragma unroll
            for (int k = 0; k < 9; ++k) ac[AF + k] = Fbs[k];
        } else {
            // Neo-Hookean: tau = mu (F F^T - I) + lambda ln J I,
            //   Fbar += mu (taubar + taubar^T) F + lambda tr(taubar) F^-T
            const float J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                            F[2] * (F[3] * F[7] - F[4] * F[6]);
            const float cof[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                                  F[2] * F[7] - F[1] * F[8], F[0] * F[8] - F[2] * F[6], F[1] * F[6] - F[0] * F[7],
                                  F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
            const float trb = tb[0] + tb[4] + tb[8];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    float sym = 0.f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) sym += (tb[r * 3 + k] + tb[k * 3 + r]) * F[k * 3 + s];
                    ac[AF + r * 3 + s] += P.mu * sym + P.lambda * trb * cof[r * 3 + s] / J;
                }
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
                           float4* gfbar, double* dE, double* dphi) {
    const float* ps = c->ps[c->cur];
    const uint32_t* perm = c->pval[c->sorted_sel];
    const uint32_t* skey = c->pkey[c->sorted_sel];
    const int64_t nodes = c->n_active * 64;
    cudaError_t e = cudaMemsetAsync(gvbar, 0, sizeof(float4) * nodes, c->st);
    if (e != cudaSuccess) return e;
    const unsigned g = blocks_for(c->n, 128);
    const double nu = c->cfg.nu;
    const double dmu = 1.0 / (2.0 * (1.0 + nu)), dla = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double kappa = (3.0 * (double)c->P.lambda + 2.0 * (double)c->P.mu) / (2.0 * (double)c->P.mu);
    const unsigned gg = (unsigned)std::min<int64_t>(blocks_for(nodes, 256), 148 * 16);
#define MPM_ADJ(D_, M_)                                                                                           \
    do {                                                                                                          \
        k_adj_g2p<D_, M_><<<g, 128, 0, c->st>>>(ps, c->pstride, perm, skey, c->n, c->nbr, c->P, c->gv, adj_next,  \
                                                adj_cur, gvbar, kappa, dphi);                                    \
        k_adj_grid<D_><<<gg, 256, 0, c->st>>>(c->live_cap, c->dstat, c->P, c->bcoord, c->gmv, c->gf, gvbar, gmbar, \
                                              gfbar);                                                             \
        k_adj_p2g<D_, M_><<<g, 128, 0, c->st>>>(ps, c->pstride, perm, skey, c->n, c->nbr, c->P, gmbar, gfbar,     \
                                                adj_cur, dmu, dla, dE);                                          \
    } while (0)
    const bool dp = c->P.material == MPM_DRUCKER_PRAGER;
    if (c->dense) {
        if (dp) MPM_ADJ(true, MPM_DRUCKER_PRAGER);
        else MPM_ADJ(true, MPM_NEOHOOKEAN);
    } else {
        if (dp) MPM_ADJ(false, MPM_DRUCKER_PRAGER);
        else MPM_ADJ(false, MPM_NEOHOOKEAN);
    }
#undef MPM_ADJ
    c->launches += 3;
    return cudaGetLastError();
}

}  // namespace mpm
