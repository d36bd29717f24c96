/*
 * Plain CPU FP64 oracle for the Total Lagrangian finite-element hot path.
 *
 * TEST INFRASTRUCTURE ONLY. This library exists so that tests, the smoke
 * check and the CPU baseline leg of the benchmark can compare the CUDA path
 * against a slow, obviously correct restatement of the paper. Nothing in the
 * product path may link, load or call it. It shares no code, header, table
 * or helper with the CUDA library.
 *
 * Every function follows the paper "A Total Lagrangian Finite Element
 * Framework for Multibody Dynamics: Part I - Formulation" (Zhou, Arivoli,
 * Negrut); the equation or section it restates is cited beside it.
 *
 * Conventions
 *   element types : 0 = T4, 1 = T10 (Appendix A.1), 2 = H8
 *   node arrays   : [n_nodes][3] row-major doubles
 *   connectivity  : [n_elem][nodes_per_elem] 0-based int32
 *   3x3 matrices  : row-major, M[a*3+b] = M_ab
 *   materials     : per element; model 0 = St. Venant-Kirchhoff (App. C.1.1),
 *                   1 = compressible neo-Hookean = Mooney-Rivlin with
 *                   mu01 = 0 (Sec. 3.2.2), with mu10 = mu/2, k = lam + 2 mu/3.
 *                   mu_v, lam_v: Kelvin-Voigt dissipation constants (Sec. 3.2.3).
 *   return value  : 0 on success, negative on bad arguments, positive = number
 *                   of quadrature points where the neo-Hookean law met J <= 0
 *                   (stress set to zero there).
 */
#ifndef TLFE_ORACLE_H
#define TLFE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t model;      /* 0 SVK, 1 neo-Hookean, 2 Mooney-Rivlin */
    double mu, lam;     /* Lame constants (small-strain shear and Lame lambda) */
    double mu_v, lam_v; /* Kelvin-Voigt constants */
    double rho;         /* reference density */
    double mu01;        /* Mooney-Rivlin mu01 (model 2); mu10 = mu/2 - mu01 */
} orc_material;

/* ---- parent elements (Appendix A) and quadrature (Section 6) ---------- */
int orc_nodes_per_elem(int type);
int orc_shape(int type, const double xi[3], double *s);
int orc_shape_grad(int type, const double xi[3], double *Hp);   /* [n][3] */
int orc_quad_rule(int type, int nq, double *pts, double *w);     /* pts [nq][3] */
int orc_exact_rule(int type, int order, double *pts, double *w); /* order^3 points */

/* ---- reference precompute, Eq. (H = Hp (U Hp)^-1), J_p = det(U Hp) ---- */
int orc_precompute(int type, int nq, int n_elem, const int32_t *conn,
                   const double *X, double *H, double *wJ, double *Jp_min);

/* ---- constitutive interface P(F, Fdot), Section 3 ---------------------- */
int orc_stress(const orc_material *m, const double F[9], const double Fdot[9], double P[9]);
int orc_strain_energy(const orc_material *m, const double F[9], double *psi);

/* ---- kinematics + internal force, Eq. (internal_force_universal) ------ */
/* kin_form 0: F = sum_i x_i h_i^T with x = X + u (the paper's literal form)
 * kin_form 1: F = I + sum_i u_i h_i^T (same quantity, using U H = I)
 * kin_form 2: F = I + sum_i (u_i - u_1) h_i^T (same, using sum_i h_i = 0);
 *             used by every other oracle routine.                          */
int orc_internal_force(int type, int nq, int n_elem, const int32_t *conn, int n_nodes,
                       const double *X, const double *u, const double *udot,
                       const orc_material *mat, int kin_form, double *f);

/* ---- tangent: closed-form blocks of App. C (and the derived KV blocks) -- */
/* y += a_M M v + a_K K_t v + a_C C v, element by element (transpose = 1 applies
 * K_t^T and C^T instead). sym_only = 1 drops the non-symmetric viscous stiffness
 * K^v from K_t. */
int orc_operator_apply(int type, int nq, int n_elem, const int32_t *conn, int n_nodes,
                       const double *X, const double *u, const double *udot,
                       const orc_material *mat, double a_M, double a_K, double a_C,
                       int transpose, int sym_only, const double *v, double *y);
int orc_element_matrices(int type, int nq, const int32_t *conn_e, const double *X,
                         const double *u, const double *udot, const orc_material *m,
                         double *Ke, double *Ce, double *Me);

/* same, with the viscous stiffness K^v left out of Ke (symmetric part) */
int orc_element_matrices_sym(int type, int nq, const int32_t *conn_e, const double *X,
                             const double *u, const double *udot, const orc_material *m,
                             double *Ke, double *Ce, double *Me);

/* ---- adjoint: g_u = K_t^T r, g_udot = C^T r, g_theta = d(f.r)/d(mu, lam) */
int orc_vjp(int type, int nq, int n_elem, const int32_t *conn, int n_nodes,
            const double *X, const double *u, const double *udot,
            const orc_material *mat, const double *r,
            double *g_u, double *g_udot, double *g_theta);

/* ---- mass and mass-distributed force field, Sec. 4.1 / 4.2 ------------- */
int orc_lumped_row_sums(int type, int n_elem, const int32_t *conn, int n_nodes,
                        const double *X, const orc_material *mat, double *m_row);
int orc_gravity(int type, int n_elem, const int32_t *conn, int n_nodes, const double *X,
                const orc_material *mat, const double g[3], double *f_ff);

/* ---- backward-Euler Newton step, Section 7 without constraints --------- */
/* ---- external loads (Sec. 4: pointwise loads, surface tractions) ------ */
int orc_point_loads(int type, int n_loads, const int32_t *conn, const int32_t *elem, const double *xi,
                    const double *force, double *f);
int orc_surface_traction(int type, int n_faces, const int32_t *conn, const double *X, const int32_t *elem,
                         const int32_t *fid, const double *t0, double *f);

typedef struct {
    int32_t newton_iters, cg_iters, status;
    double rel_residual;
} orc_report;

/* ---- bilateral constraints (Sec. 3 primitives) and the ALM step (Sec. 7) */
typedef struct {
    int32_t type;      /* 0 CD, 1 DIST, 2 DP1, 3 DP2 */
    int32_t elem[4];   /* element of points P, Q, R, T (block-local); < 0: ground point */
    double xi[4][3];   /* parent coordinates (ground points: world coordinates) */
    double d[3];       /* CD axis */
    double f;          /* prescribed value (DIST: the distance) */
} orc_constraint;

int orc_constraint_eval(int type, int n_cons, const orc_constraint *cons, const int32_t *conn, const double *X,
                        const double *u, double *c);
int orc_constraint_jt(int type, int n_cons, const orc_constraint *cons, const int32_t *conn, const double *X,
                      const double *u, const double *w, double *f);
int orc_constraint_j(int type, int n_cons, const orc_constraint *cons, const int32_t *conn, const double *X,
                     const double *u, const double *v, double *out);
int orc_newton_step_alm(int type, int nq, int n_elem, const int32_t *conn, int n_nodes, const double *X,
                        const orc_material *mat, const double *u_n, const double *v_n, double h,
                        const double gravity[3], const uint8_t *fixed, double newton_rtol, double cg_rtol,
                        int max_newton, int max_cg, int n_cons, const orc_constraint *cons, double rho,
                        double alm_tol, int max_outer, int row_norm, double *lam, double *v_out,
                        orc_report *rep, int *outer_iters, double *c_norm);
/* row weights of Eq. row_weights at the reference configuration */
int orc_constraint_row_weights(int type, int n_cons, const orc_constraint *cons, const int32_t *conn,
                               const double *X, double *w);

int orc_newton_step(int type, int nq, int n_elem, const int32_t *conn, int n_nodes,
                    const double *X, const orc_material *mat, const double *u_n,
                    const double *v_n, double h, const double gravity[3],
                    const uint8_t *fixed, double newton_rtol, double cg_rtol,
                    int max_newton, int max_cg, double *v_out, orc_report *rep);

/* ---- conflict colouring: greedy in descending splitmix64 priority ------ */
uint64_t orc_splitmix64(uint64_t x);
int orc_color_greedy(int n_elem, int npe, const int32_t *conn, int n_nodes,
                     uint64_t seed, int32_t *color);

#ifdef __cplusplus
}
#endif
#endif
