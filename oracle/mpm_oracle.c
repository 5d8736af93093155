/*
 * FP64 dense-grid CPU oracle for one explicit MPM step.  TEST INFRASTRUCTURE
 * ONLY (see mpm_oracle.h).  Plain, serial and deliberately unoptimised: every
 * sum is written the way the paper states it, over a dense grid covering the
 * whole potential domain.
 *
 * Readings taken where the paper is silent (each also listed in the design
 * notes of the repository):
 *   R1 support S(p): the full 3x3x3 stencil base + {0,1,2}^3 with
 *      base = floor(x/h - 1/2); nodes whose weight happens to be 0 stay in it.
 *   R2 compact order: blocks are scanned in ascending packed-key order of
 *      Eq. (key), i.e. i-major, k fastest; Phi(b) is the exclusive scan.
 *   R3 boundary conditions are applied to grid velocities after the update:
 *      floor (sticky / slip / Coulomb) on nodes with z_n <= floor_z, terrain
 *      level set (Coulomb with the terrain normal) on nodes with
 *      z_n <= H(x_n, y_n), then sticky walls on the outer wall_layers node
 *      layers of the box.
 *   R4 v_n = (mv)_n / m_n only where m_n > 0, else 0.
 *   R5 the stress in f_int is evaluated from F_p as stored at P2G time.
 *   R6 Neo-Hookean: tau = mu (F F^T - I) + lambda ln(J) I.
 *   R7 Drucker-Prager: return map in principal Hencky strain (Klar et al.
 *      2016): eps = ln(Sigma), alpha = sqrt(2/3) 2 sin(phi)/(3 - sin(phi)),
 *      dgamma = |dev eps| + (3 lambda + 2 mu)/(2 mu) tr(eps) alpha;
 *      tr eps >= 0 -> tip (Sigma = I); dgamma <= 0 -> unchanged;
 *      else eps -= dgamma dev(eps)/|dev eps|.  Hencky Kirchhoff stress
 *      tau = U diag(2 mu eps + lambda tr eps) U^T.
 *   R8 symplectic order: grid velocity first, then x_p += dt v_p^{n+1}.
 */
#include "mpm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ helpers */

static int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

static void box_dims(const orc_params* P, int64_t d[3]) {
    for (int a = 0; a < 3; ++a) d[a] = (int64_t)P->hi[a] - P->lo[a] + 1;
}

static int64_t node_index(const orc_params* P, const int32_t n[3]) {
    int64_t d[3];
    box_dims(P, d);
    for (int a = 0; a < 3; ++a)
        if (n[a] < P->lo[a] || n[a] > P->hi[a]) return -1;
    return (((int64_t)n[0] - P->lo[0]) * d[1] + ((int64_t)n[1] - P->lo[1])) * d[2] +
           ((int64_t)n[2] - P->lo[2]);
}

static void lame(const orc_params* P, double* mu, double* lambda) {
    *mu = P->E / (2.0 * (1.0 + P->nu));
    *lambda = P->E * P->nu / ((1.0 + P->nu) * (1.0 - 2.0 * P->nu));
}

static double particle_volume(const orc_params* P) { return P->h * P->h * P->h / P->ppc; }
static double particle_mass(const orc_params* P) { return P->rho * particle_volume(P); }

static void matmul(const double A[9], const double B[9], double C[9]) {
    double T[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
            T[3 * r + c] = s;
        }
    memcpy(C, T, sizeof T);
}

static void transpose(const double A[9], double T[9]) {
    double R[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[3 * c + r] = A[3 * r + c];
    memcpy(T, R, sizeof R);
}

static double det3(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

static int inverse3(const double A[9], double Ai[9]) {
    double d = det3(A);
    if (d == 0.0 || !isfinite(d)) return -1;
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / d;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / d;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / d;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / d;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / d;
    return 0;
}

/* ----------------------------------------------------- quadratic B-spline */

/* 1-D quadratic B-spline of the distance t = x/h - i (Steffen et al. 2008):
 * 3/4 - t^2 for |t| < 1/2, (3/2 - |t|)^2 / 2 for 1/2 <= |t| < 3/2, else 0;
 * dw is its derivative with respect to t. */
static void bspline(double t, double* w, double* dw) {
    double a = fabs(t);
    if (a < 0.5) {
        *w = 0.75 - t * t;
        *dw = -2.0 * t;
    } else if (a < 1.5) {
        double r = 1.5 - a;
        *w = 0.5 * r * r;
        *dw = (t > 0.0) ? -r : r;
    } else {
        *w = 0.0;
        *dw = 0.0;
    }
}

static void stencil_base(const orc_params* P, const double x[3], int32_t base[3]) {
    for (int a = 0; a < 3; ++a) base[a] = (int32_t)floor(x[a] / P->h - 0.5);
}

/* Sec. 4.1: N_n(x_p) = w(x/h - i) w(y/h - j) w(z/h - k) and
 * grad N_n = (w' w w, w w' w, w w w') / h, over the support of reading R1. */
void orc_weights(const orc_params* P, const double x[3], int32_t nodes[27 * 3],
                 double w[27], double gw[27 * 3]) {
    int32_t base[3];
    stencil_base(P, x, base);
    int q = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c, ++q) {
                int32_t n[3] = {base[0] + a, base[1] + b, base[2] + c};
                double wx, wy, wz, dx, dy, dz;
                bspline(x[0] / P->h - n[0], &wx, &dx);
                bspline(x[1] / P->h - n[1], &wy, &dy);
                bspline(x[2] / P->h - n[2], &wz, &dz);
                nodes[3 * q + 0] = n[0];
                nodes[3 * q + 1] = n[1];
                nodes[3 * q + 2] = n[2];
                w[q] = wx * wy * wz;
                gw[3 * q + 0] = dx * wy * wz / P->h;
                gw[3 * q + 1] = wx * dy * wz / P->h;
                gw[3 * q + 2] = wx * wy * dz / P->h;
            }
}

void orc_Dp(const orc_params* P, const double x[3], double D[9]) {
    int32_t nodes[81];
    double w[27], gw[81];
    orc_weights(P, x, nodes, w, gw);
    memset(D, 0, 9 * sizeof(double));
    for (int q = 0; q < 27; ++q) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = nodes[3 * q + a] * P->h - x[a];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) D[3 * r + c] += w[q] * d[r] * d[c];
    }
}

/* ------------------------------------------ active blocks: Alg. 2, 3, 4 */

int64_t orc_active_blocks(const orc_params* P, int64_t np, const double* x,
                          int32_t* out_b, int64_t cap) {
    const int64_t B = P->B;
    int64_t blo[3], nb[3];
    for (int a = 0; a < 3; ++a) {
        blo[a] = floordiv(P->lo[a], B);
        nb[a] = floordiv(P->hi[a], B) - blo[a] + 1;
    }
    const int64_t ncand = nb[0] * nb[1] * nb[2];
    unsigned char* chi = (unsigned char*)calloc((size_t)ncand, 1);
    int64_t* s = (int64_t*)malloc((size_t)ncand * sizeof(int64_t));
    if (!chi || !s) {
        free(chi);
        free(s);
        return -4;
    }
    /* Alg. 2: chi_b = 1 for b = n // B of every n in S(p). */
    for (int64_t p = 0; p < np; ++p) {
        int32_t base[3];
        stencil_base(P, &x[3 * p], base);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) {
                    int64_t n[3] = {base[0] + a, base[1] + b, base[2] + c};
                    int64_t q = 0;
                    for (int ax = 0; ax < 3; ++ax) {
                        if (n[ax] < P->lo[ax] || n[ax] > P->hi[ax]) {
                            free(chi);
                            free(s);
                            return -1;
                        }
                        q = q * nb[ax] + (floordiv(n[ax], B) - blo[ax]);
                    }
                    chi[q] = 1;
                }
    }
    /* Alg. 3 with one thread: s_q = number of active blocks before q, in the
     * flattened order q = (bi * nbj + bj) * nbk + bk (ascending packed key). */
    int64_t r = 0;
    for (int64_t q = 0; q < ncand; ++q) {
        s[q] = r;
        r += chi[q];
    }
    const int64_t nactive = r;
    if (nactive > cap) {
        free(chi);
        free(s);
        return -2;
    }
    /* Alg. 4: the compact block list at position s_q. */
    for (int64_t q = 0; q < ncand; ++q) {
        if (!chi[q]) continue;
        int64_t bk = q % nb[2], bj = (q / nb[2]) % nb[1], bi = q / (nb[1] * nb[2]);
        out_b[3 * s[q] + 0] = (int32_t)(bi + blo[0]);
        out_b[3 * s[q] + 1] = (int32_t)(bj + blo[1]);
        out_b[3 * s[q] + 2] = (int32_t)(bk + blo[2]);
    }
    free(chi);
    free(s);
    return nactive;
}

int64_t orc_block_index(const int32_t* blocks, int64_t nb, const int32_t b[3]) {
    for (int64_t q = 0; q < nb; ++q)
        if (blocks[3 * q] == b[0] && blocks[3 * q + 1] == b[1] && blocks[3 * q + 2] == b[2])
            return q;
    return -1;
}

/* ------------------------------------------------------------ 3x3 SVD */

/* One-sided (Hestenes) Jacobi: orthogonalise the columns of A by plane
 * rotations accumulated in V until every pair is orthogonal to machine
 * precision; then S = column norms, U = normalised columns. */
void orc_svd3(const double A[9], double U[9], double S[3], double V[9]) {
    double W[9];
    memcpy(W, A, sizeof W);
    double Vm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rotated = 0;
        for (int i = 0; i < 2; ++i)
            for (int j = i + 1; j < 3; ++j) {
                double al = 0, be = 0, ga = 0;
                for (int r = 0; r < 3; ++r) {
                    al += W[3 * r + i] * W[3 * r + i];
                    be += W[3 * r + j] * W[3 * r + j];
                    ga += W[3 * r + i] * W[3 * r + j];
                }
                if (fabs(ga) <= 1e-300 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                rotated = 1;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int r = 0; r < 3; ++r) {
                    double wi = W[3 * r + i], wj = W[3 * r + j];
                    W[3 * r + i] = c * wi - s * wj;
                    W[3 * r + j] = s * wi + c * wj;
                    double vi = Vm[3 * r + i], vj = Vm[3 * r + j];
                    Vm[3 * r + i] = c * vi - s * vj;
                    Vm[3 * r + j] = s * vi + c * vj;
                }
            }
        if (!rotated) break;
    }
    double sig[3];
    int ord[3] = {0, 1, 2};
    for (int c = 0; c < 3; ++c)
        sig[c] = sqrt(W[c] * W[c] + W[3 + c] * W[3 + c] + W[6 + c] * W[6 + c]);
    /* sort descending */
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (sig[ord[b]] > sig[ord[a]]) {
                int t = ord[a];
                ord[a] = ord[b];
                ord[b] = t;
            }
    for (int c = 0; c < 3; ++c) {
        int o = ord[c];
        S[c] = sig[o];
        for (int r = 0; r < 3; ++r) {
            V[3 * r + c] = Vm[3 * r + o];
            U[3 * r + c] = sig[o] > 0 ? W[3 * r + o] / sig[o] : 0.0;
        }
    }
    /* complete U for a zero singular value */
    if (S[2] <= 0.0) {
        U[2] = U[3] * U[7] - U[6] * U[4];
        U[5] = U[6] * U[1] - U[0] * U[7];
        U[8] = U[0] * U[4] - U[3] * U[1];
    }
    /* make V a rotation; then make U a rotation, moving the sign to S[2] */
    if (det3(V) < 0) {
        for (int r = 0; r < 3; ++r) {
            V[3 * r + 2] = -V[3 * r + 2];
            U[3 * r + 2] = -U[3 * r + 2];
        }
    }
    if (det3(U) < 0) {
        for (int r = 0; r < 3; ++r) U[3 * r + 2] = -U[3 * r + 2];
        S[2] = -S[2];
    }
}

/* -------------------------------------------------- constitutive models */

static double dp_alpha(double phi_deg) {
    double sp = sin(phi_deg * M_PI / 180.0);
    return sqrt(2.0 / 3.0) * 2.0 * sp / (3.0 - sp);
}

int orc_kirchhoff(const orc_params* P, const double F[9], double phi_deg, double tau[9]) {
    (void)phi_deg;
    double mu, la;
    lame(P, &mu, &la);
    if (P->material == ORC_NEOHOOKEAN) {
        double J = det3(F);
        if (!(J > 0.0)) return -3;
        double Ft[9], b[9];
        transpose(F, Ft);
        matmul(F, Ft, b);
        double lj = log(J);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                tau[3 * r + c] = mu * (b[3 * r + c] - (r == c ? 1.0 : 0.0)) + (r == c ? la * lj : 0.0);
        return 0;
    }
    /* Hencky: tau = U diag(2 mu eps_i + lambda sum eps) U^T */
    double U[9], S[3], V[9];
    orc_svd3(F, U, S, V);
    if (!(S[2] > 0.0)) return -3;
    double eps[3] = {log(S[0]), log(S[1]), log(S[2])};
    double tr = eps[0] + eps[1] + eps[2];
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = 2.0 * mu * eps[a] + la * tr;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += U[3 * r + a] * d[a] * U[3 * c + a];
            tau[3 * r + c] = s;
        }
    return 0;
}

int orc_dp_project(const orc_params* P, const double F[9], double phi_deg,
                   double Fout[9], int* case_out) {
    double mu, la;
    lame(P, &mu, &la);
    double U[9], S[3], V[9];
    orc_svd3(F, U, S, V);
    if (!(S[2] > 0.0)) return -3;
    double eps[3] = {log(S[0]), log(S[1]), log(S[2])};
    double tr = eps[0] + eps[1] + eps[2];
    double dev[3] = {eps[0] - tr / 3.0, eps[1] - tr / 3.0, eps[2] - tr / 3.0};
    double ndev = sqrt(dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]);
    double alpha = dp_alpha(phi_deg);
    double dgamma = ndev + (3.0 * la + 2.0 * mu) / (2.0 * mu) * tr * alpha;
    double H[3];
    int cs;
    if (tr >= 0.0) {
        H[0] = H[1] = H[2] = 0.0;
        cs = 1;
    } else if (dgamma <= 0.0) {
        H[0] = eps[0];
        H[1] = eps[1];
        H[2] = eps[2];
        cs = 0;
    } else {
        for (int a = 0; a < 3; ++a) H[a] = eps[a] - dgamma * dev[a] / ndev;
        cs = 2;
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += U[3 * r + a] * exp(H[a]) * V[3 * c + a];
            Fout[3 * r + c] = s;
        }
    if (case_out) *case_out = cs;
    return 0;
}

/* -------------------------------------------------------------- P2G */

/* One particle's contribution to its 27 stencil nodes, Sec. 4.1:
 *   m_n   += N m_p
 *   mv_n  += N m_p [v_p + C_p (x_n - x_p)]
 *   f_n   -= grad N sigma_p V_p,  sigma_p V_p = (tau/J)(J V0) = tau V0. */
static int p2g_particle(const orc_params* P, const double x[3], const double v[3],
                        const double C[9], const double F[9], double phi_deg,
                        int32_t nodes[81], double dm[27], double dmv[81], double df[81]) {
    double w[27], gw[81], tau[9];
    orc_weights(P, x, nodes, w, gw);
    if (orc_kirchhoff(P, F, phi_deg, tau) != 0) return -3;
    const double J = det3(F);
    const double Vp = J * particle_volume(P);
    double sigma[9];
    for (int a = 0; a < 9; ++a) sigma[a] = tau[a] / J;
    const double mp = particle_mass(P);
    for (int q = 0; q < 27; ++q) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = nodes[3 * q + a] * P->h - x[a];
        dm[q] = w[q] * mp;
        for (int r = 0; r < 3; ++r) {
            double cd = C[3 * r + 0] * d[0] + C[3 * r + 1] * d[1] + C[3 * r + 2] * d[2];
            dmv[3 * q + r] = w[q] * mp * (v[r] + cd);
            double sg = sigma[3 * r + 0] * gw[3 * q + 0] + sigma[3 * r + 1] * gw[3 * q + 1] +
                        sigma[3 * r + 2] * gw[3 * q + 2];
            df[3 * q + r] = -sg * Vp;
        }
    }
    return 0;
}

static double phi_of(const orc_params* P, const double* phi, int64_t p) {
    return phi ? phi[p] : P->phi_deg;
}

#ifdef _OPENMP
/* The all-core build (gcc -fopenmp; a timing baseline only, never the parity
 * reference): each thread scatters a contiguous share of the particles into
 * its own dense grid, and the grids are added node by node in thread order,
 * so a run is reproducible for a given thread count.  The serial build above
 * is the one the tests check against. */
static int p2g_threads(const orc_params* P, int64_t np, const double* x, const double* v,
                       const double* C, const double* F, const double* phi, int64_t nn,
                       double* m, double* mv, double* f) {
    /* at most 16 GB of per-thread grids */
    int nt = omp_get_max_threads();
    const double grid_bytes = (double)nn * 7 * sizeof(double);
    if (nt * grid_bytes > 16e9) nt = grid_bytes >= 16e9 ? 1 : (int)(16e9 / grid_bytes);
    double* g = (double*)calloc((size_t)nt * (size_t)nn * 7, sizeof(double));
    if (!g) return -4;
    int rc = 0;
#pragma omp parallel num_threads(nt) reduction(min : rc)
    {
        const int t = omp_get_thread_num(), nth = omp_get_num_threads();
        double* gm = g + (size_t)t * nn * 7;
        double* gmv = gm + nn;
        double* gf = gmv + 3 * nn;
        const int64_t p0 = np * t / nth, p1 = np * (t + 1) / nth;
        int err = 0;
        for (int64_t p = p0; p < p1 && err == 0; ++p) {
            int32_t nodes[81];
            double dm[27], dmv[81], df[81];
            err = p2g_particle(P, &x[3 * p], &v[3 * p], &C[9 * p], &F[9 * p], phi_of(P, phi, p),
                               nodes, dm, dmv, df);
            for (int q = 0; q < 27 && err == 0; ++q) {
                int64_t id = node_index(P, &nodes[3 * q]);
                if (id < 0) {
                    err = -1;
                    break;
                }
                gm[id] += dm[q];
                for (int a = 0; a < 3; ++a) {
                    gmv[3 * id + a] += dmv[3 * q + a];
                    gf[3 * id + a] += df[3 * q + a];
                }
            }
        }
        rc = err;
#pragma omp barrier
#pragma omp for schedule(static)
        for (int64_t id = 0; id < nn; ++id)
            for (int s = 0; s < nt; ++s) {
                const double* sm = g + (size_t)s * nn * 7;
                m[id] += sm[id];
                for (int a = 0; a < 3; ++a) {
                    mv[3 * id + a] += sm[nn + 3 * id + a];
                    f[3 * id + a] += sm[4 * nn + 3 * id + a];
                }
            }
    }
    free(g);
    return rc;
}
#endif

int orc_p2g(const orc_params* P, int64_t np, const double* x, const double* v,
            const double* C, const double* F, const double* phi,
            double* m, double* mv, double* f) {
    int64_t d[3];
    box_dims(P, d);
    const int64_t nn = d[0] * d[1] * d[2];
    memset(m, 0, (size_t)nn * sizeof(double));
    memset(mv, 0, (size_t)nn * 3 * sizeof(double));
    memset(f, 0, (size_t)nn * 3 * sizeof(double));
#ifdef _OPENMP
    if (omp_get_max_threads() > 1) return p2g_threads(P, np, x, v, C, F, phi, nn, m, mv, f);
#endif
    for (int64_t p = 0; p < np; ++p) {
        int32_t nodes[81];
        double dm[27], dmv[81], df[81];
        int rc = p2g_particle(P, &x[3 * p], &v[3 * p], &C[9 * p], &F[9 * p], phi_of(P, phi, p),
                              nodes, dm, dmv, df);
        if (rc) return rc;
        for (int q = 0; q < 27; ++q) {
            int64_t id = node_index(P, &nodes[3 * q]);
            if (id < 0) return -1;
            m[id] += dm[q];
            for (int a = 0; a < 3; ++a) {
                mv[3 * id + a] += dmv[3 * q + a];
                f[3 * id + a] += df[3 * q + a];
            }
        }
    }
    return 0;
}

int orc_p2g_abs(const orc_params* P, int64_t np, const double* x, const double* v,
                const double* C, const double* F, const double* phi,
                double* am, double* amv, double* af) {
    int64_t d[3];
    box_dims(P, d);
    const int64_t nn = d[0] * d[1] * d[2];
    memset(am, 0, (size_t)nn * sizeof(double));
    memset(amv, 0, (size_t)nn * 3 * sizeof(double));
    memset(af, 0, (size_t)nn * 3 * sizeof(double));
    double mu, la;
    lame(P, &mu, &la);
    for (int64_t p = 0; p < np; ++p) {
        int32_t nodes[81];
        double w[27], gw[81], tau[9];
        orc_weights(P, &x[3 * p], nodes, w, gw);
        if (orc_kirchhoff(P, &F[9 * p], phi_of(P, phi, p), tau) != 0) return -3;
        double tmax = 0.0;
        for (int a = 0; a < 9; ++a) tmax = fmax(tmax, fabs(tau[a]));
        const double mp = particle_mass(P);
        for (int q = 0; q < 27; ++q) {
            int64_t id = node_index(P, &nodes[3 * q]);
            if (id < 0) return -1;
            am[id] += w[q] * mp;
            double g1 = fabs(gw[3 * q]) + fabs(gw[3 * q + 1]) + fabs(gw[3 * q + 2]);
            for (int r = 0; r < 3; ++r) {
                double s = fabs(v[3 * p + r]);
                for (int c = 0; c < 3; ++c)
                    s += fabs(C[9 * p + 3 * r + c]) * fabs(nodes[3 * q + c] * P->h - x[3 * p + c]);
                amv[3 * id + r] += w[q] * mp * s;
                af[3 * id + r] += g1 * particle_volume(P) * (tmax + mu + la);
            }
        }
    }
    return 0;
}

int orc_p2g_nodes(const orc_params* P, int64_t np, const double* x, const double* v,
                  const double* C, const double* F, const double* phi,
                  int64_t nq, const int32_t* qn, double* m, double* mv, double* f, double* af) {
    memset(m, 0, (size_t)nq * sizeof(double));
    memset(mv, 0, (size_t)nq * 3 * sizeof(double));
    memset(f, 0, (size_t)nq * 3 * sizeof(double));
    if (af) memset(af, 0, (size_t)nq * sizeof(double));
    double mu, la;
    lame(P, &mu, &la);
    for (int64_t p = 0; p < np; ++p) {
        int32_t base[3];
        stencil_base(P, &x[3 * p], base);
        int touches = 0;
        for (int64_t k = 0; k < nq && !touches; ++k) {
            int in = 1;
            for (int a = 0; a < 3; ++a)
                if (qn[3 * k + a] < base[a] || qn[3 * k + a] > base[a] + 2) in = 0;
            touches = in;
        }
        if (!touches) continue;
        int32_t nodes[81];
        double dm[27], dmv[81], df[81];
        int rc = p2g_particle(P, &x[3 * p], &v[3 * p], &C[9 * p], &F[9 * p], phi_of(P, phi, p),
                              nodes, dm, dmv, df);
        if (rc) return rc;
        double tmax = 0.0, w[27], gw[81], tau[9];
        if (af) {
            int32_t nn[81];
            orc_weights(P, &x[3 * p], nn, w, gw);
            orc_kirchhoff(P, &F[9 * p], phi_of(P, phi, p), tau);
            for (int a = 0; a < 9; ++a) tmax = fmax(tmax, fabs(tau[a]));
        }
        for (int q = 0; q < 27; ++q)
            for (int64_t k = 0; k < nq; ++k) {
                if (nodes[3 * q] != qn[3 * k] || nodes[3 * q + 1] != qn[3 * k + 1] ||
                    nodes[3 * q + 2] != qn[3 * k + 2])
                    continue;
                m[k] += dm[q];
                for (int a = 0; a < 3; ++a) {
                    mv[3 * k + a] += dmv[3 * q + a];
                    f[3 * k + a] += df[3 * q + a];
                }
                if (af)
                    af[k] += (fabs(gw[3 * q]) + fabs(gw[3 * q + 1]) + fabs(gw[3 * q + 2])) * particle_volume(P) *
                             (tmax + mu + la);
            }
    }
    return 0;
}

/* ------------------------------------------------------- grid update */

/* Coulomb friction against a rigid boundary with outward normal nrm
 * (Stomakhin et al. 2013 form): only an approaching velocity (v.n < 0) is
 * changed; the normal part is removed and the tangential part is reduced by
 * mu |v.n|, or stopped when the reduction exceeds it. */
static void coulomb(double v[3], const double nrm[3], double mu) {
    double vn = v[0] * nrm[0] + v[1] * nrm[1] + v[2] * nrm[2];
    if (vn >= 0.0) return;
    double vt[3] = {v[0] - vn * nrm[0], v[1] - vn * nrm[1], v[2] - vn * nrm[2]};
    double nt = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
    if (nt + mu * vn <= 0.0) {
        v[0] = v[1] = v[2] = 0.0;
        return;
    }
    double s = (nt + mu * vn) / nt;
    for (int a = 0; a < 3; ++a) v[a] = vt[a] * s;
}

static double terrain_at(const orc_params* P, int64_t ti, int64_t tj) {
    if (ti < 0) ti = 0;
    if (tj < 0) tj = 0;
    if (ti >= P->terrain_nx) ti = P->terrain_nx - 1;
    if (tj >= P->terrain_ny) tj = P->terrain_ny - 1;
    return P->terrain[ti + (int64_t)P->terrain_nx * tj];
}

void orc_grid_node(const orc_params* P, const int32_t n[3], double m, const double mv[3],
                   const double f[3], double vo[3]) {
    if (m > 0.0) {
        for (int a = 0; a < 3; ++a) {
            double vn = mv[a] / m;                          /* v_n = (mv)_n / m_n */
            vo[a] = vn + P->dt / m * (f[a] + m * P->g[a]);   /* explicit Euler */
        }
    } else {
        vo[0] = vo[1] = vo[2] = 0.0;
    }
    const double z = n[2] * P->h;
    if (P->floor_kind != ORC_FLOOR_NONE && z <= P->floor_z) {
        const double up[3] = {0.0, 0.0, 1.0};
        if (P->floor_kind == ORC_FLOOR_STICKY) {
            vo[0] = vo[1] = vo[2] = 0.0;
        } else if (P->floor_kind == ORC_FLOOR_SLIP) {
            if (vo[2] < 0.0) vo[2] = 0.0;
        } else {
            coulomb(vo, up, P->floor_mu);
        }
    }
    if (P->terrain) {
        int64_t ti = (int64_t)n[0] - P->lo[0], tj = (int64_t)n[1] - P->lo[1];
        double H = terrain_at(P, ti, tj);
        if (z <= H) {
            /* outward normal of z = H(x, y) by central differences
             * (one-sided at the edges of the height map) */
            int64_t i0 = ti > 0 ? ti - 1 : ti, i1 = ti < P->terrain_nx - 1 ? ti + 1 : ti;
            int64_t j0 = tj > 0 ? tj - 1 : tj, j1 = tj < P->terrain_ny - 1 ? tj + 1 : tj;
            double hx = (terrain_at(P, i1, tj) - terrain_at(P, i0, tj)) / ((double)(i1 - i0) * P->h);
            double hy = (terrain_at(P, ti, j1) - terrain_at(P, ti, j0)) / ((double)(j1 - j0) * P->h);
            double nrm[3] = {-hx, -hy, 1.0};
            double l = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + 1.0);
            for (int a = 0; a < 3; ++a) nrm[a] /= l;
            coulomb(vo, nrm, P->terrain_mu);
        }
    }
    for (int a = 0; a < 3; ++a)
        if (n[a] - P->lo[a] < P->wall_layers || P->hi[a] - n[a] < P->wall_layers) {
            vo[0] = vo[1] = vo[2] = 0.0;
            break;
        }
}

void orc_grid_update(const orc_params* P, const double* m, const double* mv, const double* f,
                     double* vn) {
    int64_t d[3];
    box_dims(P, d);
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static)
#endif
    for (int64_t i = 0; i < d[0]; ++i)
        for (int64_t j = 0; j < d[1]; ++j)
            for (int64_t k = 0; k < d[2]; ++k) {
                int64_t id = (i * d[1] + j) * d[2] + k;
                int32_t n[3] = {(int32_t)(i + P->lo[0]), (int32_t)(j + P->lo[1]),
                                (int32_t)(k + P->lo[2])};
                orc_grid_node(P, n, m[id], &mv[3 * id], &f[3 * id], &vn[3 * id]);
            }
}

/* -------------------------------------------------------------- G2P */

/* Sec. 4.1: v_p = sum N v_n;  x_p += dt v_p;  C_p = (sum N v_n (x) (x_n - x_p)) D_p^-1;
 * F_p = (I + dt sum v_n (x) grad N) F_p;  then the constitutive update. */
int orc_g2p_one(const orc_params* P, const double vn27[81], double phi_deg, double x[3],
                double v[3], double C[9], double F[9]) {
    int32_t nodes[81];
    double w[27], gw[81];
    orc_weights(P, x, nodes, w, gw);
    double vp[3] = {0, 0, 0}, Bm[9] = {0}, L[9] = {0}, D[9] = {0};
    for (int q = 0; q < 27; ++q) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = nodes[3 * q + a] * P->h - x[a];
        for (int r = 0; r < 3; ++r) {
            vp[r] += w[q] * vn27[3 * q + r];
            for (int c = 0; c < 3; ++c) {
                Bm[3 * r + c] += w[q] * vn27[3 * q + r] * d[c];
                L[3 * r + c] += vn27[3 * q + r] * gw[3 * q + c];
                D[3 * r + c] += w[q] * d[r] * d[c];
            }
        }
    }
    double Di[9];
    if (inverse3(D, Di) != 0) return -3;
    double Cn[9];
    matmul(Bm, Di, Cn);
    double G[9];
    for (int a = 0; a < 9; ++a) G[a] = P->dt * L[a] + ((a % 4) == 0 ? 1.0 : 0.0);
    double Fn[9];
    matmul(G, F, Fn);
    for (int a = 0; a < 3; ++a) {
        v[a] = vp[a];
        x[a] += P->dt * vp[a];
    }
    memcpy(C, Cn, sizeof Cn);
    if (P->material == ORC_DRUCKER_PRAGER) {
        double Fp[9];
        if (orc_dp_project(P, Fn, phi_deg, Fp, NULL) != 0) return -3;
        memcpy(F, Fp, sizeof Fp);
    } else {
        memcpy(F, Fn, sizeof Fn);
    }
    for (int a = 0; a < 9; ++a)
        if (!isfinite(F[a]) || !isfinite(C[a])) return -3;
    return 0;
}

int orc_g2p(const orc_params* P, int64_t np, const double* vn, double* x, double* v,
            double* C, double* F, const double* phi) {
#ifdef _OPENMP
    if (omp_get_max_threads() > 1) {
        int rc = 0;
#pragma omp parallel for schedule(static) reduction(min : rc)
        for (int64_t p = 0; p < np; ++p) {
            int32_t nodes[81];
            double w[27], gw[81], v27[81];
            orc_weights(P, &x[3 * p], nodes, w, gw);
            int e = 0;
            for (int q = 0; q < 27 && !e; ++q) {
                int64_t id = node_index(P, &nodes[3 * q]);
                if (id < 0) e = -1;
                else
                    for (int a = 0; a < 3; ++a) v27[3 * q + a] = vn[3 * id + a];
            }
            if (!e) e = orc_g2p_one(P, v27, phi_of(P, phi, p), &x[3 * p], &v[3 * p], &C[9 * p], &F[9 * p]);
            if (e < rc) rc = e;
        }
        return rc;
    }
#endif
    for (int64_t p = 0; p < np; ++p) {
        int32_t nodes[81];
        double w[27], gw[81], v27[81];
        orc_weights(P, &x[3 * p], nodes, w, gw);
        for (int q = 0; q < 27; ++q) {
            int64_t id = node_index(P, &nodes[3 * q]);
            if (id < 0) return -1;
            for (int a = 0; a < 3; ++a) v27[3 * q + a] = vn[3 * id + a];
        }
        int rc = orc_g2p_one(P, v27, phi_of(P, phi, p), &x[3 * p], &v[3 * p], &C[9 * p], &F[9 * p]);
        if (rc) return rc;
    }
    return 0;
}

int orc_run(const orc_params* P, int64_t np, double* x, double* v, double* C, double* F,
            const double* phi, int32_t nsteps) {
    int64_t d[3];
    box_dims(P, d);
    const int64_t nn = d[0] * d[1] * d[2];
    double* m = (double*)malloc((size_t)nn * sizeof(double));
    double* mv = (double*)malloc((size_t)nn * 3 * sizeof(double));
    double* f = (double*)malloc((size_t)nn * 3 * sizeof(double));
    double* vn = (double*)malloc((size_t)nn * 3 * sizeof(double));
    int rc = (m && mv && f && vn) ? 0 : -4;
    for (int32_t s = 0; s < nsteps && rc == 0; ++s) {
        rc = orc_p2g(P, np, x, v, C, F, phi, m, mv, f);
        if (rc) break;
        orc_grid_update(P, m, mv, f, vn);
        rc = orc_g2p(P, np, vn, x, v, C, F, phi);
    }
    free(m);
    free(mv);
    free(f);
    free(vn);
    return rc;
}
