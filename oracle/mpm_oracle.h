/*
 * FP64 dense-grid CPU oracle for one explicit MPM step on a background grid.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library and never imports it.
 *
 * Every routine follows the paper (Zhao et al., "Unified sparse framework for
 * large-scale simulations using the material point method"):
 *   - Sec. 4.1 (MPM formulation): node tuple n=(i,j,k), x_n = h n, quadratic
 *     B-spline N_n and grad N_n, support S(p), active set A = U_p S(p), APIC
 *     P2G (mass, momentum), internal/external force, explicit Euler grid
 *     update, G2P (velocity, position, APIC C_p with D_p, deformation gradient).
 *   - Sec. 4.2, Alg. 2-4 (mark_active_blocks, parallel_scan with one thread,
 *     construct_compact_block_map): the active block set and its compact map
 *     Phi, with phi(n) = Phi(b(n)) B^3 + l(n) (Alg. 1 / Alg. 5).
 * Readings where the paper is silent (support = full 3x3x3 stencil, canonical
 * block order = ascending packed key, boundary conditions, Drucker-Prager
 * return map, Neo-Hookean stress) are listed in the repository's design notes
 * and restated beside each routine in mpm_oracle.c.
 *
 * Particle arrays are array-of-structs in double: x[np][3], v[np][3],
 * C[np][9] and F[np][9] (row-major 3x3), phi[np] in degrees (may be NULL).
 * Dense grid arrays cover the node box [lo, hi] (inclusive) with index
 *   ((i-lo0)*ny + (j-lo1))*nz + (k-lo2),  ny = hi1-lo1+1, nz = hi2-lo2+1,
 * scalar fields have one double per node, vector fields three.
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_NEOHOOKEAN = 0, ORC_DRUCKER_PRAGER = 1 };
enum { ORC_FLOOR_NONE = 0, ORC_FLOOR_STICKY = 1, ORC_FLOOR_SLIP = 2, ORC_FLOOR_COULOMB = 3 };

typedef struct {
    int32_t lo[3], hi[3];      /* potential grid node box, inclusive */
    double h;                  /* grid spacing */
    double dt;                 /* time step */
    double g[3];               /* body force per unit mass */
    int32_t B;                 /* block edge in nodes (1 or 4) */
    int32_t material;          /* ORC_NEOHOOKEAN or ORC_DRUCKER_PRAGER */
    double E, nu, rho;         /* Young's modulus, Poisson ratio, density */
    double phi_deg;            /* friction angle when no per-particle array */
    double ppc;                /* particles per cell: m_p = rho h^3/ppc, V0 = h^3/ppc */
    int32_t floor_kind;        /* ORC_FLOOR_* for nodes with z_n <= floor_z */
    double floor_z, floor_mu;
    const double* terrain;     /* heights at node columns (i-lo0) + nxt*(j-lo1), or NULL */
    int32_t terrain_nx, terrain_ny;
    double terrain_mu;
    int32_t wall_layers;       /* sticky node layers at each face of the box */
} orc_params;

/* Quadratic B-spline: N_n(x_p) and grad N_n(x_p) for the 27 stencil nodes
 * base + {0,1,2}^3 (base = floor(x/h - 1/2)); nodes[27][3]. */
void orc_weights(const orc_params* P, const double x[3], int32_t nodes[27 * 3],
                 double w[27], double gw[27 * 3]);

/* APIC D_p = sum_n N (x_n-x_p)(x_n-x_p)^T, written out as in Sec. 4.1. */
void orc_Dp(const orc_params* P, const double x[3], double D[9]);

/* Active blocks by dense mask + serial exclusive scan (Alg. 2-4, n_th = 1).
 * Writes the block tuples of the compact block list, in Phi order, to
 * out_b[cap][3].  Returns the number of active blocks, or -1 if a stencil
 * node leaves the box, or -2 if cap is too small. */
int64_t orc_active_blocks(const orc_params* P, int64_t np, const double* x,
                          int32_t* out_b, int64_t cap);

/* Phi(b) for one block tuple given the compact block list (binary-free
 * linear search, -1 if absent). */
int64_t orc_block_index(const int32_t* blocks, int64_t nb, const int32_t b[3]);

/* Kirchhoff stress tau = J sigma of the elastic model at F. */
int orc_kirchhoff(const orc_params* P, const double F[9], double phi_deg, double tau[9]);

/* Drucker-Prager return map in principal Hencky strain on an elastic trial F.
 * case_out: 0 inside the cone, 1 tip (tension), 2 projected to the cone. */
int orc_dp_project(const orc_params* P, const double F[9], double phi_deg,
                   double Fout[9], int* case_out);

/* SVD A = U diag(S) V^T by one-sided Jacobi, S descending, U and V rotations
 * (the sign of det A is carried by S[2]). */
void orc_svd3(const double A[9], double U[9], double S[3], double V[9]);

/* Dense P2G: m, mv = sum N m_p [v_p + C_p (x_n - x_p)], f = f_int (no gravity).
 * Arrays are zeroed first.  Returns 0, or -1 for a stencil outside the box,
 * -3 for an invalid stress state. */
int orc_p2g(const orc_params* P, int64_t np, const double* x, const double* v,
            const double* C, const double* F, const double* phi,
            double* m, double* mv, double* f);

/* Per-node absolute sums used to bound FP32 rounding in tests:
 * am = sum N m_p, amv = sum N m_p |v_p + C_p (x_n - x_p)| (per component),
 * af = sum |grad N|_1 V0 (max|tau_p| + mu + lambda) (per component, same value). */
int orc_p2g_abs(const orc_params* P, int64_t np, const double* x, const double* v,
                const double* C, const double* F, const double* phi,
                double* am, double* amv, double* af);

/* P2G sums at a list of query nodes only (for spot checks of large runs);
 * af (may be NULL) receives the force scale of orc_p2g_abs at those nodes. */
int orc_p2g_nodes(const orc_params* P, int64_t np, const double* x, const double* v,
                  const double* C, const double* F, const double* phi,
                  int64_t nq, const int32_t* qnodes, double* m, double* mv, double* f, double* af);

/* Grid update: v = mv/m + dt (f/m + g) for m > 0 else 0, then boundary
 * conditions.  vn has 3 doubles per node. */
void orc_grid_update(const orc_params* P, const double* m, const double* mv,
                     const double* f, double* vn);

/* Grid velocity after the update for a single node (used by spot checks). */
void orc_grid_node(const orc_params* P, const int32_t n[3], double m,
                   const double mv[3], const double f[3], double vout[3]);

/* G2P for one particle given v at its 27 stencil nodes (order of orc_weights).
 * Updates x, v, C, F in place; F is the projected elastic F for DP. */
int orc_g2p_one(const orc_params* P, const double vn27[27 * 3], double phi_deg,
                double x[3], double v[3], double C[9], double F[9]);

/* Dense G2P over all particles. */
int orc_g2p(const orc_params* P, int64_t np, const double* vn, double* x,
            double* v, double* C, double* F, const double* phi);

/* nsteps full steps (P2G, grid update, G2P) on a dense grid it allocates. */
int orc_run(const orc_params* P, int64_t np, double* x, double* v, double* C,
            double* F, const double* phi, int32_t nsteps);

#ifdef __cplusplus
}
#endif
#endif
