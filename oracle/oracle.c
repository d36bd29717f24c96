/*
 * Plain CPU FP64 oracle for the Total Lagrangian finite-element hot path.
 *
 * TEST INFRASTRUCTURE ONLY: called by tests, the smoke check and the CPU
 * baseline leg of the benchmark; never by the product path. It shares no code
 * with the CUDA library. Built with -ffp-contract=off so that every product
 * and sum is rounded once, in the order written.
 *
 * Sections / equations cited are those of the paper "A Total Lagrangian Finite
 * Element Framework for Multibody Dynamics: Part I - Formulation".
 *
 * Readings taken where the paper is silent (each also listed in the design
 * notes):
 *   - Neo-Hookean = Mooney-Rivlin with mu01 = 0 (Sec. 3.2.2); Lame (mu, lam)
 *     map to mu10 = mu/2 and k = lam + 2 mu / 3 (small-strain shear and bulk).
 *   - Quadrature constants are not tabulated in the paper (Sec. 6 only says
 *     they are tabulated once on the parent element): T4 centroid; T10 4-point
 *     (degree 2) and 5-point (degree 3, negative centroid weight) rules; H8
 *     2x2x2 Gauss-Legendre.
 *   - T4 and H8 are not in Appendix A: linear barycentric tetrahedron, and the
 *     trilinear brick with the Q27 node ordering (first index fastest).
 *   - J <= 0 at a neo-Hookean quadrature point: stress is set to zero there and
 *     the point is counted in the return value.
 *   - The Kelvin-Voigt tangent is promised but not printed (Sec. 4.3, App. C);
 *     the blocks below are derived from Eqs. (viscous2PKstress, viscous1PKstress).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small dense helpers                                                       */
/* ------------------------------------------------------------------------ */

static double det3(const double A[9])
{
    return A[0] * (A[4] * A[8] - A[5] * A[7])
         - A[1] * (A[3] * A[8] - A[5] * A[6])
         + A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* inverse by cofactors: A^{-1} = adj(A) / det(A) */
static void inv3(const double A[9], double det, double R[9])
{
    R[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    R[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    R[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    R[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    R[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    R[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    R[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    R[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    R[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

static void transpose3(const double A[9], double R[9])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) R[a * 3 + b] = A[b * 3 + a];
}

static void matmul3(const double A[9], const double B[9], double R[9])
{
    double T[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[a * 3 + k] * B[k * 3 + b];
            T[a * 3 + b] = s;
        }
    memcpy(R, T, sizeof(T));
}

static void matvec3(const double A[9], const double x[3], double y[3])
{
    for (int a = 0; a < 3; ++a) y[a] = A[a * 3] * x[0] + A[a * 3 + 1] * x[1] + A[a * 3 + 2] * x[2];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ------------------------------------------------------------------------ */
/* parent elements (Appendix A)                                              */
/* ------------------------------------------------------------------------ */

int orc_nodes_per_elem(int type)
{
    switch (type) {
    case 0: return 4;
    case 1: return 10;
    case 2: return 8;
    case 3: return 27;
    default: return -1;
    }
}

#define ORC_MAXN 27 /* nodes of the largest element (Q27) */
#define ORC_MAXQ 27 /* points of the largest volume rule (3x3x3 Gauss) */

/* 1-D quadratic Lagrange polynomials of the Q27 element on nodes -1, 0, 1
 * (App., "1D Lagrange Polynomials"): L0 = s(s-1)/2, L1 = 1 - s^2, L2 = s(s+1)/2 */
static double quad1(int a, double t) { return a == 0 ? 0.5 * t * (t - 1.0) : (a == 1 ? 1.0 - t * t : 0.5 * t * (t + 1.0)); }
static double dquad1(int a, double t) { return a == 0 ? t - 0.5 : (a == 1 ? -2.0 * t : t + 0.5); }

/* 1-D linear Lagrange factors on [-1, 1] used by the H8 tensor product */
static double lin1(int i, double t) { return i == 0 ? 0.5 * (1.0 - t) : 0.5 * (1.0 + t); }
static double dlin1(int i) { return i == 0 ? -0.5 : 0.5; }

int orc_shape(int type, const double xi[3], double *s)
{
    const double x = xi[0], y = xi[1], z = xi[2];
    if (type == 0) {
        /* barycentric L1..L4 of Appendix A.1: L1 = 1 - xi - eta - zeta */
        s[0] = 1.0 - x - y - z;
        s[1] = x;
        s[2] = y;
        s[3] = z;
        return 0;
    }
    if (type == 1) {
        /* Appendix A.1, shape-function vector s(xi, eta, zeta) */
        s[0] = 2 * y * y + 4 * x * y + 4 * y * z - 3 * y + 2 * x * x + 4 * x * z - 3 * x
             + 2 * z * z - 3 * z + 1;
        s[1] = 2 * x * x - x;
        s[2] = 2 * y * y - y;
        s[3] = 2 * z * z - z;
        s[4] = -4 * x * y - 4 * x * x - 4 * x * z + 4 * x;
        s[5] = 4 * x * y;
        s[6] = -4 * y * y - 4 * x * y - 4 * y * z + 4 * y;
        s[7] = -4 * y * z - 4 * x * z - 4 * z * z + 4 * z;
        s[8] = 4 * x * z;
        s[9] = 4 * y * z;
        return 0;
    }
    if (type == 2) {
        for (int k = 0; k < 2; ++k)
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i)
                    s[i + 2 * j + 4 * k] = lin1(i, x) * lin1(j, y) * lin1(k, z);
        return 0;
    }
    if (type == 3) {
        /* Q27: tensor products L_i(xi) L_j(eta) L_k(zeta), node i + 3 j + 9 k
         * at parent coordinates (i - 1, j - 1, k - 1) (App., Q27 node table) */
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i) s[i + 3 * j + 9 * k] = quad1(i, x) * quad1(j, y) * quad1(k, z);
        return 0;
    }
    return -1;
}

/* Hp[i*3 + k] = d s_i / d xi_k: the parent Jacobian of Appendix A (printed as
 * "H" for T10 there; it is the parent-coordinate table H^p of Section 6). */
int orc_shape_grad(int type, const double xi[3], double *Hp)
{
    const double x = xi[0], y = xi[1], z = xi[2];
    if (type == 0) {
        static const double g[12] = {-1, -1, -1, 1, 0, 0, 0, 1, 0, 0, 0, 1};
        memcpy(Hp, g, sizeof(g));
        return 0;
    }
    if (type == 1) {
        const double c = 4 * y + 4 * x + 4 * z - 3;
        double g[30] = {
            c, c, c,
            4 * x - 1, 0, 0,
            0, 4 * y - 1, 0,
            0, 0, 4 * z - 1,
            -4 * y - 8 * x - 4 * z + 4, -4 * x, -4 * x,
            4 * y, 4 * x, 0,
            -4 * y, -8 * y - 4 * x - 4 * z + 4, -4 * y,
            -4 * z, -4 * z, -4 * y - 4 * x - 8 * z + 4,
            4 * z, 0, 4 * x,
            0, 4 * z, 4 * y};
        memcpy(Hp, g, sizeof(g));
        return 0;
    }
    if (type == 2) {
        for (int k = 0; k < 2; ++k)
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i) {
                    const int n = i + 2 * j + 4 * k;
                    Hp[n * 3 + 0] = dlin1(i) * lin1(j, y) * lin1(k, z);
                    Hp[n * 3 + 1] = lin1(i, x) * dlin1(j) * lin1(k, z);
                    Hp[n * 3 + 2] = lin1(i, x) * lin1(j, y) * dlin1(k);
                }
        return 0;
    }
    if (type == 3) {
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i) {
                    const int n = i + 3 * j + 9 * k;
                    Hp[n * 3 + 0] = dquad1(i, x) * quad1(j, y) * quad1(k, z);
                    Hp[n * 3 + 1] = quad1(i, x) * dquad1(j, y) * quad1(k, z);
                    Hp[n * 3 + 2] = quad1(i, x) * quad1(j, y) * dquad1(k, z);
                }
        return 0;
    }
    return -1;
}

/* Quadrature on the parent element (Section 6, Eq. approximation-of-integral).
 * Tetrahedron rules are written in barycentric form; (xi, eta, zeta) =
 * (L2, L3, L4) per Appendix A.1. */
int orc_quad_rule(int type, int nq, double *pts, double *w)
{
    if (type == 0 || type == 1) {
        double L[5][4];
        if (nq == 1) {
            for (int k = 0; k < 4; ++k) L[0][k] = 0.25;
            w[0] = 1.0 / 6.0;
        } else if (nq == 4) {
            const double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
            for (int q = 0; q < 4; ++q) {
                for (int k = 0; k < 4; ++k) L[q][k] = (k == q) ? a : b;
                w[q] = 1.0 / 24.0;
            }
        } else if (nq == 5) {
            for (int k = 0; k < 4; ++k) L[0][k] = 0.25;
            w[0] = -2.0 / 15.0;
            for (int q = 1; q < 5; ++q) {
                for (int k = 0; k < 4; ++k) L[q][k] = (k == q - 1) ? 0.5 : 1.0 / 6.0;
                w[q] = 3.0 / 40.0;
            }
        } else {
            return -1;
        }
        for (int q = 0; q < nq; ++q) {
            pts[q * 3 + 0] = L[q][1];
            pts[q * 3 + 1] = L[q][2];
            pts[q * 3 + 2] = L[q][3];
        }
        return 0;
    }
    if (type == 2) {
        if (nq == 1) {
            pts[0] = pts[1] = pts[2] = 0.0;
            w[0] = 8.0;
            return 0;
        }
        if (nq == 8) {
            const double g = 1.0 / sqrt(3.0);
            for (int k = 0; k < 2; ++k)
                for (int j = 0; j < 2; ++j)
                    for (int i = 0; i < 2; ++i) {
                        const int q = i + 2 * j + 4 * k;
                        pts[q * 3 + 0] = i ? g : -g;
                        pts[q * 3 + 1] = j ? g : -g;
                        pts[q * 3 + 2] = k ? g : -g;
                        w[q] = 1.0;
                    }
            return 0;
        }
        return -1;
    }
    if (type == 3 && nq == 27) {
        /* 3 x 3 x 3 Gauss-Legendre: nodes 0, +-sqrt(3/5), weights 8/9, 5/9 */
        const double g = sqrt(0.6), x3[3] = {-g, 0.0, g}, w3[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i) {
                    const int q = i + 3 * j + 9 * k;
                    pts[q * 3 + 0] = x3[i];
                    pts[q * 3 + 1] = x3[j];
                    pts[q * 3 + 2] = x3[k];
                    w[q] = w3[i] * w3[j] * w3[k];
                }
        return 0;
    }
    return -1;
}

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on the Legendre
 * three-term recurrence (textbook construction). */
static void gauss_legendre(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double t = cos(pi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(t), p0 = P_{n-1}(t) */
            double dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 1; k < n; ++k) {
            double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* High-order rule for the mass and body-force integrals of Sec. 4.1-4.2:
 * tensor Gauss-Legendre on the brick; on the tetrahedron the collapsed
 * (Duffy) map xi = a, eta = (1-a) b, zeta = (1-a)(1-b) c of the unit cube,
 * Jacobian (1-a)^2 (1-b). order^3 points. */
int orc_exact_rule(int type, int order, double *pts, double *w)
{
    if (order < 1 || order > 12) return -1;
    double gx[12], gw[12];
    gauss_legendre(order, gx, gw);
    int q = 0;
    for (int k = 0; k < order; ++k)
        for (int j = 0; j < order; ++j)
            for (int i = 0; i < order; ++i, ++q) {
                if (type == 2 || type == 3) {
                    pts[q * 3 + 0] = gx[i];
                    pts[q * 3 + 1] = gx[j];
                    pts[q * 3 + 2] = gx[k];
                    w[q] = gw[i] * gw[j] * gw[k];
                } else if (type == 0 || type == 1) {
                    const double a = 0.5 * (gx[i] + 1.0), b = 0.5 * (gx[j] + 1.0),
                                 c = 0.5 * (gx[k] + 1.0);
                    pts[q * 3 + 0] = a;
                    pts[q * 3 + 1] = (1.0 - a) * b;
                    pts[q * 3 + 2] = (1.0 - a) * (1.0 - b) * c;
                    w[q] = 0.125 * gw[i] * gw[j] * gw[k] * (1.0 - a) * (1.0 - a) * (1.0 - b);
                } else {
                    return -1;
                }
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 6: reference precompute                                           */
/* ------------------------------------------------------------------------ */

/* dU/dxi = U Hp(xi) (3x3), with U = [u_1 .. u_n] the reference node matrix
 * (Sec. 6). Evaluated as sum_{i>1} (u_i - u_1) (dS_i/dxi)^T, equal because the
 * parent gradients sum to zero (sum_i s_i = 1, App. A); node coordinates far
 * from the origin then cost no digits. */
static void parent_jacobian(int n, const double *Xe, const double *Hp, double Jp[9])
{
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int i = 1; i < n; ++i) s += (Xe[i * 3 + a] - Xe[a]) * Hp[i * 3 + k];
            Jp[a * 3 + k] = s;
        }
}

static void gather(int n, const int32_t *ce, const double *A, double *Ae)
{
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) Ae[i * 3 + a] = A[(size_t)ce[i] * 3 + a];
}

/* H(u*) = Hp(xi*) [U Hp(xi*)]^{-1} and J_p = det(U Hp) (Eq. importantQuantities-
 * Parent2ReferenceJump); stored per element and quadrature point as
 * H[e][q][i][c] = (h_i)_c and wJ[e][q] = w_q J_p. */
int orc_precompute(int type, int nq, int n_elem, const int32_t *conn, const double *X,
                   double *H, double *wJ, double *Jp_min)
{
    const int n = orc_nodes_per_elem(type);
    double pts[ORC_MAXQ * 3], w[ORC_MAXQ];
    if (n < 0 || nq > ORC_MAXQ || orc_quad_rule(type, nq, pts, w)) return -1;
    int bad = 0;
    double jmin = INFINITY;
    double Xe[3 * ORC_MAXN], Hp[3 * ORC_MAXN], Jp[9], Ji[9];
    for (int e = 0; e < n_elem; ++e) {
        gather(n, conn + (size_t)e * n, X, Xe);
        for (int q = 0; q < nq; ++q) {
            orc_shape_grad(type, pts + q * 3, Hp);
            parent_jacobian(n, Xe, Hp, Jp);
            const double d = det3(Jp);
            if (d < jmin) jmin = d;
            double *He = H + ((size_t)e * nq + q) * n * 3;
            if (!(d > 0.0)) {
                ++bad;
                memset(He, 0, sizeof(double) * n * 3);
                wJ[(size_t)e * nq + q] = 0.0;
                continue;
            }
            inv3(Jp, d, Ji);
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += Hp[i * 3 + k] * Ji[k * 3 + c];
                    He[i * 3 + c] = s;
                }
            wJ[(size_t)e * nq + q] = w[q] * d;
        }
    }
    if (Jp_min) *Jp_min = jmin;
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Section 3: constitutive interface                                         */
/* ------------------------------------------------------------------------ */

/* Green-Lagrange rate Edot = 1/2 (Fdot^T F + F^T Fdot) and the Kelvin-Voigt
 * viscous second Piola-Kirchhoff stress S^v = 2 mu_v Edot + lam_v tr(Edot) I
 * (Eq. viscous2PKstress). */
static void viscous_S(const orc_material *m, const double F[9], const double Fd[9], double Sv[9])
{
    double Ed[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Fd[k * 3 + a] * F[k * 3 + b] + F[k * 3 + a] * Fd[k * 3 + b];
            Ed[a * 3 + b] = 0.5 * s;
        }
    const double tr = Ed[0] + Ed[4] + Ed[8];
    for (int a = 0; a < 9; ++a) Sv[a] = 2.0 * m->mu_v * Ed[a];
    Sv[0] += m->lam_v * tr;
    Sv[4] += m->lam_v * tr;
    Sv[8] += m->lam_v * tr;
}

static int has_viscous(const orc_material *m, const double *Fd)
{
    return Fd != NULL && (m->mu_v != 0.0 || m->lam_v != 0.0);
}

/* Mooney-Rivlin constants from the material record: the small-strain shear
 * modulus 2 (mu10 + mu01) equals mu and the bulk modulus is k = lam + 2 mu / 3;
 * neo-Hookean is the case mu01 = 0. */
static void mr_constants(const orc_material *m, double *mu10, double *mu01, double *k)
{
    *mu01 = m->model == 2 ? m->mu01 : 0.0;
    *mu10 = 0.5 * m->mu - *mu01;
    *k = m->lam + 2.0 * m->mu / 3.0;
}

/* I1 = tr C and I2 = 1/2 (I1^2 - tr(C C)) of C = F^T F */
static void invariants(const double F[9], double *I1, double *I2, double C[9])
{
    double Ft[9];
    transpose3(F, Ft);
    matmul3(Ft, F, C);
    double trC2 = 0.0;
    for (int a = 0; a < 9; ++a) trC2 += C[a] * C[a]; /* C symmetric: tr(C C) */
    *I1 = C[0] + C[4] + C[8];
    *I2 = 0.5 * (*I1 * *I1 - trC2);
}

/* P = P^e(F) + F S^v (Eq. total1PKstress). Elastic parts:
 *   SVK: P = lam (1/2 tr(F^T F) - 3/2) F + mu F F^T F - mu F  (App. C, expanded SVK P)
 *   MR : P = 2 mu10 J^{-2/3} (F - 1/3 I1 F^{-T})
 *          + 2 mu01 J^{-4/3} (I1 F - F C - 2/3 I2 F^{-T})
 *          + k (J - 1) J F^{-T}                      (App. C, Eq. mr_first_piola)
 *   NH : the same with mu01 = 0. */
int orc_stress(const orc_material *m, const double F[9], const double Fd[9], double P[9])
{
    int status = 0;
    if (m->model == 0) {
        double trC = 0.0;
        for (int a = 0; a < 9; ++a) trC += F[a] * F[a];
        double Ft[9], FFt[9], FFtF[9];
        transpose3(F, Ft);
        matmul3(F, Ft, FFt);
        matmul3(FFt, F, FFtF);
        const double c = m->lam * (0.5 * trC - 1.5);
        for (int a = 0; a < 9; ++a) P[a] = c * F[a] + m->mu * FFtF[a] - m->mu * F[a];
    } else if (m->model == 1 || m->model == 2) {
        const double J = det3(F);
        if (!(J > 0.0)) {
            for (int a = 0; a < 9; ++a) P[a] = 0.0;
            return 1;
        }
        double mu10, mu01, k;
        mr_constants(m, &mu10, &mu01, &k);
        double Fi[9], FiT[9], C[9], FC[9], I1, I2;
        inv3(F, J, Fi);
        transpose3(Fi, FiT);
        invariants(F, &I1, &I2, C);
        matmul3(F, C, FC);
        const double Jm23 = 1.0 / (cbrt(J) * cbrt(J));
        const double Jm43 = Jm23 * Jm23;
        for (int a = 0; a < 9; ++a)
            P[a] = 2.0 * mu10 * Jm23 * (F[a] - I1 / 3.0 * FiT[a]) +
                   2.0 * mu01 * Jm43 * (I1 * F[a] - FC[a] - 2.0 / 3.0 * I2 * FiT[a]) + k * (J - 1.0) * J * FiT[a];
    } else {
        return -1;
    }
    if (has_viscous(m, Fd)) {
        double Sv[9], Pv[9];
        viscous_S(m, F, Fd, Sv);
        matmul3(F, Sv, Pv);
        for (int a = 0; a < 9; ++a) P[a] += Pv[a];
    }
    return status;
}

/* Strain-energy densities: SVK psi(E) = lam/2 (tr E)^2 + mu tr(E^2) (Eq.
 * svk_strain_energy); MR: psi = mu10 (J^{-2/3} I1 - 3) + mu01 (J^{-4/3} I2 - 3)
 * + k/2 (J-1)^2 (Eq. mr_strain_energy; neo-Hookean: mu01 = 0). */
int orc_strain_energy(const orc_material *m, const double F[9], double *psi)
{
    if (m->model == 0) {
        double E[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += F[k * 3 + a] * F[k * 3 + b];
                E[a * 3 + b] = 0.5 * (s - (a == b ? 1.0 : 0.0));
            }
        const double tr = E[0] + E[4] + E[8];
        double trE2 = 0.0;
        for (int a = 0; a < 9; ++a) trE2 += E[a] * E[a]; /* E symmetric: tr(E E) */
        *psi = 0.5 * m->lam * tr * tr + m->mu * trE2;
        return 0;
    }
    if (m->model == 1 || m->model == 2) {
        const double J = det3(F);
        if (!(J > 0.0)) {
            *psi = NAN;
            return 1;
        }
        double C[9], I1, I2, mu10, mu01, k;
        invariants(F, &I1, &I2, C);
        mr_constants(m, &mu10, &mu01, &k);
        const double Jm23 = 1.0 / (cbrt(J) * cbrt(J));
        *psi = mu10 * (I1 * Jm23 - 3.0) + mu01 * (I2 * Jm23 * Jm23 - 3.0) + 0.5 * k * (J - 1.0) * (J - 1.0);
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Section 2.1 / Eq. (expression-F): kinematics at one quadrature point       */
/* ------------------------------------------------------------------------ */

/* He: [n][3] = h_i; Xe, ue: [n][3].
 * kin_form 0: F = sum_i x_i h_i^T, x = X + u (Eq. expression-F as printed);
 * kin_form 1: F = I + sum_i u_i h_i^T (U H = I, Sec. 6);
 * kin_form 2: F = I + sum_i (u_i - u_1) h_i^T (also sum_i h_i = 0, the
 *             gradient of the partition of unity sum_i s_i = 1). The three are
 *             equal in exact arithmetic; 2 rounds least when the element moves
 *             far from its reference position. */
static void deformation_gradient(int n, const double *He, const double *Xe, const double *ue,
                                 int kin_form, double F[9])
{
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            if (kin_form == 0) {
                for (int i = 0; i < n; ++i) s += (Xe[i * 3 + a] + ue[i * 3 + a]) * He[i * 3 + c];
                F[a * 3 + c] = s;
            } else if (kin_form == 1) {
                for (int i = 0; i < n; ++i) s += ue[i * 3 + a] * He[i * 3 + c];
                F[a * 3 + c] = (a == c ? 1.0 : 0.0) + s;
            } else {
                for (int i = 1; i < n; ++i) s += (ue[i * 3 + a] - ue[a]) * He[i * 3 + c];
                F[a * 3 + c] = (a == c ? 1.0 : 0.0) + s;
            }
        }
}

static void rate_gradient(int n, const double *He, const double *vde, double Fd[9])
{
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += vde[i * 3 + a] * He[i * 3 + c];
            Fd[a * 3 + c] = s;
        }
}

/* per-element reference data for one element (computed on the fly from X so
 * that the oracle never stores anything the CUDA side could share) */
typedef struct {
    int n, nq;
    double H[ORC_MAXQ * ORC_MAXN * 3];
    double wJ[ORC_MAXQ];
    int bad;
} elem_geom;

static int element_geometry(int type, int nq, const int32_t *ce, const double *X, elem_geom *g)
{
    g->n = orc_nodes_per_elem(type);
    g->nq = nq;
    double Jmin;
    g->bad = orc_precompute(type, nq, 1, ce, X, g->H, g->wJ, &Jmin);
    return g->bad;
}

/* f_i^int = int P(F) h_i dV_r ~ sum_q w_q J_p P_q h_i (Eqs. internal_force_universal
 * and approximation-of-integral), assembled in element order. */
int orc_internal_force(int type, int nq, int n_elem, const int32_t *conn, int n_nodes,
                       const double *X, const double *u, const double *udot,
                       const orc_material *mat, int kin_form, double *f)
{
    const int n = orc_nodes_per_elem(type);
    if (n < 0) return -1;
    (void)n_nodes;
    int bad = 0;
    double Xe[3 * ORC_MAXN], ue[3 * ORC_MAXN], vde[3 * ORC_MAXN], F[9], Fd[9], P[9];
    elem_geom g;
    for (int e = 0; e < n_elem; ++e) {
        const int32_t *ce = conn + (size_t)e * n;
        if (element_geometry(type, nq, ce, X, &g) < 0) return -1;
        gather(n, ce, X, Xe);
        gather(n, ce, u, ue);
        if (udot) gather(n, ce, udot, vde);
        double fe[3 * ORC_MAXN] = {0};
        for (int q = 0; q < nq; ++q) {
            const double *He = g.H + q * n * 3;
            deformation_gradient(n, He, Xe, ue, kin_form, F);
            if (udot) rate_gradient(n, He, vde, Fd);
            int st = orc_stress(mat + e, F, udot ? Fd : NULL, P);
            if (st < 0) return -1;
            bad += st;
            for (int i = 0; i < n; ++i) {
                double Ph[3];
                matvec3(P, He + i * 3, Ph);
                for (int a = 0; a < 3; ++a) fe[i * 3 + a] += g.wJ[q] * Ph[a];
            }
        }
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) f[(size_t)ce[i] * 3 + a] += fe[i * 3 + a];
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* App. C: tangent blocks                                                    */
/* ------------------------------------------------------------------------ */

static void outer_add(double K[9], double c, const double x[3], const double y[3])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) K[a * 3 + b] += c * x[a] * y[b];
}

static void eye_add(double K[9], double c)
{
    K[0] += c;
    K[4] += c;
    K[8] += c;
}

/* Elastic block dP-contribution K_ij at one quadrature point (without wJ):
 *   SVK: Eq. (svk_tangent)
 *   MR : Eq. (mr_tangent), dt1 - dt2 + dt3 - dt4 - dt5 + dt6
 *   NH : the same with mu01 = 0 (dt3 = dt4 = dt5 = 0). */
static int elastic_block(const orc_material *m, const double F[9], const double *hi,
                         const double *hj, double K[9])
{
    memset(K, 0, sizeof(double) * 9);
    double Fhi[3], Fhj[3];
    matvec3(F, hi, Fhi);
    matvec3(F, hj, Fhj);
    const double hij = dot3(hi, hj);
    if (m->model == 0) {
        double trC = 0.0;
        for (int a = 0; a < 9; ++a) trC += F[a] * F[a];
        const double trE = 0.5 * trC - 1.5;
        double Ft[9], FFt[9];
        transpose3(F, Ft);
        matmul3(F, Ft, FFt);
        outer_add(K, m->lam, Fhi, Fhj);
        eye_add(K, m->lam * trE * hij);
        eye_add(K, m->mu * dot3(Fhj, Fhi));
        outer_add(K, m->mu, Fhj, Fhi);
        for (int a = 0; a < 9; ++a) K[a] += m->mu * hij * FFt[a];
        eye_add(K, -m->mu * hij);
        return 0;
    }
    if (m->model == 1 || m->model == 2) {
        const double J = det3(F);
        if (!(J > 0.0)) return 1;
        double mu10, mu01, k;
        mr_constants(m, &mu10, &mu01, &k);
        double Fi[9], FiT[9], C[9], I1, I2;
        inv3(F, J, Fi);
        transpose3(Fi, FiT);
        invariants(F, &I1, &I2, C);
        const double Jm23 = 1.0 / (cbrt(J) * cbrt(J));
        double Gi[3], Gj[3]; /* F^{-T} h_i, F^{-T} h_j */
        matvec3(FiT, hi, Gi);
        matvec3(FiT, hj, Gj);
        /* dt1 = 2 mu10 J^{-2/3} [ (h_j.h_i) I - 2/3 (F h_i)(F^{-T} h_j)^T ] */
        const double c1 = 2.0 * mu10 * Jm23;
        eye_add(K, c1 * hij);
        outer_add(K, -c1 * 2.0 / 3.0, Fhi, Gj);
        /* - dt2, dt2 = 2 mu10/3 J^{-2/3} [ (F^{-T}h_i)(2 F h_j)^T
         *               - 2/3 I1 (F^{-T}h_i)(F^{-T}h_j)^T - I1 (F^{-T}h_j)(F^{-T}h_i)^T ] */
        const double c2 = 2.0 * mu10 / 3.0 * Jm23;
        outer_add(K, -c2 * 2.0, Gi, Fhj);
        outer_add(K, c2 * 2.0 / 3.0 * I1, Gi, Gj);
        outer_add(K, c2 * I1, Gj, Gi);
        /* dt6 = k J [ (2J - 1)(F^{-T}h_i)(F^{-T}h_j)^T - (J - 1)(F^{-T}h_j)(F^{-T}h_i)^T ] */
        outer_add(K, k * J * (2.0 * J - 1.0), Gi, Gj);
        outer_add(K, -k * J * (J - 1.0), Gj, Gi);
        if (mu01 != 0.0) {
            const double Jm43 = Jm23 * Jm23;
            double Ft[9], FFt[9], FFtFhi[3], Bj[3];
            transpose3(F, Ft);
            matmul3(F, Ft, FFt);
            matvec3(FFt, Fhi, FFtFhi);
            /* dt3 = 2 mu01 J^{-4/3} [ I1 (h_j.h_i) I + (F h_i)(2 F h_j)^T - 4/3 I1 (F h_i)(F^{-T} h_j)^T ] */
            const double c3 = 2.0 * mu01 * Jm43;
            eye_add(K, c3 * I1 * hij);
            outer_add(K, c3 * 2.0, Fhi, Fhj);
            outer_add(K, -c3 * 4.0 / 3.0 * I1, Fhi, Gj);
            /* - dt4, dt4 = 2 mu01 J^{-4/3} [ (F h_j).(F h_i) I + (F h_j)(F h_i)^T + (h_j.h_i) F F^T
             *               - 4/3 F F^T (F h_i)(F^{-T} h_j)^T ] */
            eye_add(K, -c3 * dot3(Fhj, Fhi));
            outer_add(K, -c3, Fhj, Fhi);
            for (int a = 0; a < 9; ++a) K[a] -= c3 * hij * FFt[a];
            outer_add(K, c3 * 4.0 / 3.0, FFtFhi, Gj);
            /* - dt5, dt5 = 4 mu01/3 J^{-4/3} [ (F^{-T}h_i)( 2 (F h_j)^T (I1 I - F F^T) - 4/3 I2 (F^{-T}h_j)^T )
             *               - I2 (F^{-T}h_j)(F^{-T}h_i)^T ] */
            const double c5 = 4.0 * mu01 / 3.0 * Jm43;
            for (int b = 0; b < 3; ++b) { /* B_j = (I1 I - F F^T)^T (F h_j) = (I1 I - F F^T)(F h_j) */
                Bj[b] = I1 * Fhj[b];
                for (int c = 0; c < 3; ++c) Bj[b] -= FFt[c * 3 + b] * Fhj[c];
            }
            outer_add(K, -c5 * 2.0, Gi, Bj);
            outer_add(K, c5 * 4.0 / 3.0 * I2, Gi, Gj);
            outer_add(K, c5 * I2, Gj, Gi);
        }
        return 0;
    }
    return -1;
}

/* Kelvin-Voigt blocks, derived from P^v = F S^v with S^v(Edot),
 * Edot = 1/2 (Fdot^T F + F^T Fdot):
 *   C_ij   = d f_i / d xdot_j
 *          = mu_v (F h_j)(F h_i)^T + mu_v (h_i.h_j) F F^T + lam_v (F h_i)(F h_j)^T
 *   K^v_ij = d f^v_i / d x_j (xdot fixed)
 *          = (h_j^T S^v h_i) I + mu_v (h_i.h_j) F Fdot^T + mu_v (F h_j)(Fdot h_i)^T
 *            + lam_v (F h_i)(Fdot h_j)^T                                        */
static void viscous_blocks(const orc_material *m, const double F[9], const double Fd[9],
                           const double *hi, const double *hj, double Cb[9], double Kv[9])
{
    double Fhi[3], Fhj[3], Fdhi[3], Fdhj[3], Ft[9], FFt[9], Fdt[9], FFdt[9], Sv[9], Svhi[3];
    matvec3(F, hi, Fhi);
    matvec3(F, hj, Fhj);
    matvec3(Fd, hi, Fdhi);
    matvec3(Fd, hj, Fdhj);
    transpose3(F, Ft);
    matmul3(F, Ft, FFt);
    transpose3(Fd, Fdt);
    matmul3(F, Fdt, FFdt);
    const double hij = dot3(hi, hj);
    memset(Cb, 0, sizeof(double) * 9);
    outer_add(Cb, m->mu_v, Fhj, Fhi);
    for (int a = 0; a < 9; ++a) Cb[a] += m->mu_v * hij * FFt[a];
    outer_add(Cb, m->lam_v, Fhi, Fhj);

    viscous_S(m, F, Fd, Sv);
    matvec3(Sv, hi, Svhi);
    memset(Kv, 0, sizeof(double) * 9);
    eye_add(Kv, dot3(hj, Svhi));
    for (int a = 0; a < 9; ++a) Kv[a] += m->mu_v * hij * FFdt[a];
    outer_add(Kv, m->mu_v, Fhj, Fdhi);
    outer_add(Kv, m->lam_v, Fhi, Fdhj);
}

/* consistent mass m_ij = rho int s_i s_j dV_r (Eq. virtual_work_inertia_discrete)
 * and v_i = int s_i dV_r (Eq. virtual_work_force_field_uniform), by the
 * high-order rule of orc_exact_rule (exact for the polynomial integrands of the
 * affine T4/T10 and trilinear H8 maps). */
static int element_mass(int type, const int32_t *ce, const double *X, double rho, double *Me,
                        double *vol_s)
{
    const int n = orc_nodes_per_elem(type);
    const int order = 5;
    double pts[125 * 3], w[125], Xe[3 * ORC_MAXN], Hp[3 * ORC_MAXN], Jp[9], s[ORC_MAXN];
    if (orc_exact_rule(type, order, pts, w)) return -1;
    gather(n, ce, X, Xe);
    if (Me) memset(Me, 0, sizeof(double) * n * n);
    if (vol_s) memset(vol_s, 0, sizeof(double) * n);
    for (int q = 0; q < order * order * order; ++q) {
        orc_shape(type, pts + q * 3, s);
        orc_shape_grad(type, pts + q * 3, Hp);
        parent_jacobian(n, Xe, Hp, Jp);
        const double dv = w[q] * det3(Jp);
        for (int i = 0; i < n; ++i) {
            if (vol_s) vol_s[i] += s[i] * dv;
            if (Me)
                for (int j = 0; j < n; ++j) Me[i * n + j] += rho * s[i] * s[j] * dv;
        }
    }
    return 0;
}

/* Element matrices (3n x 3n, row 3i+a, column 3j+b):
 *   Ke = sum_q wJ [K^e_ij + K^v_ij], Ce = sum_q wJ C_ij, Me = m_ij I_3. */
static int element_matrices_sel(int type, int nq, const int32_t *ce, const double *X,
                                const double *u, const double *udot, const orc_material *m,
                                int sym_only, double *Ke, double *Ce, double *Me)
{
    const int n = orc_nodes_per_elem(type);
    const int N = 3 * n;
    elem_geom g;
    if (element_geometry(type, nq, ce, X, &g) < 0) return -1;
    double Xe[3 * ORC_MAXN], ue[3 * ORC_MAXN], vde[3 * ORC_MAXN], F[9], Fd[9];
    gather(n, ce, X, Xe);
    gather(n, ce, u, ue);
    const int visc = udot != NULL && (m->mu_v != 0.0 || m->lam_v != 0.0);
    if (udot) gather(n, ce, udot, vde);
    if (Ke) memset(Ke, 0, sizeof(double) * N * N);
    if (Ce) memset(Ce, 0, sizeof(double) * N * N);
    int bad = 0;
    for (int q = 0; q < nq; ++q) {
        const double *He = g.H + q * n * 3;
        deformation_gradient(n, He, Xe, ue, 2, F);
        if (udot) rate_gradient(n, He, vde, Fd);
        else memset(Fd, 0, sizeof(Fd));
        const double wq = g.wJ[q];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double Kb[9], Cb[9], Kv[9];
                if (Ke) {
                    int st = elastic_block(m, F, He + i * 3, He + j * 3, Kb);
                    if (st < 0) return -1;
                    if (st > 0) {
                        if (i == 0 && j == 0) ++bad;
                        continue;
                    }
                }
                if (m->mu_v != 0.0 || m->lam_v != 0.0) {
                    /* C needs only F; K^v also needs Fdot */
                    viscous_blocks(m, F, Fd, He + i * 3, He + j * 3, Cb, Kv);
                } else {
                    memset(Cb, 0, sizeof(Cb));
                    memset(Kv, 0, sizeof(Kv));
                }
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        const size_t idx = (size_t)(3 * i + a) * N + 3 * j + b;
                        if (Ke) Ke[idx] += wq * (Kb[a * 3 + b] + ((visc && !sym_only) ? Kv[a * 3 + b] : 0.0));
                        if (Ce) Ce[idx] += wq * Cb[a * 3 + b];
                    }
            }
    }
    if (Me) {
        double m_ij[100];
        if (element_mass(type, ce, X, m->rho, m_ij, NULL)) return -1;
        memset(Me, 0, sizeof(double) * N * N);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int a = 0; a < 3; ++a) Me[(size_t)(3 * i + a) * N + 3 * j + a] = m_ij[i * n + j];
    }
    return bad;
}

int orc_element_matrices(int type, int nq, const int32_t *conn_e, const double *X,
                         const double *u, const double *udot, const orc_material *m,
                         double *Ke, double *Ce, double *Me)
{
    return element_matrices_sel(type, nq, conn_e, X, u, udot, m, 0, Ke, Ce, Me);
}

int orc_element_matrices_sym(int type, int nq, const int32_t *conn_e, const double *X,
                             const double *u, const double *udot, const orc_material *m,
                             double *Ke, double *Ce, double *Me)
{
    return element_matrices_sel(type, nq, conn_e, X, u, udot, m, 1, Ke, Ce, Me);
}

int orc_operator_apply(int type, int nq, int n_elem, const int32_t *conn, int n_nodes,
                       const double *X, const double *u, const double *udot,
                       const orc_material *mat, double a_M, double a_K, double a_C,
                       int transpose, int sym_only, const double *v, double *y)
{
    const int n = orc_nodes_per_elem(type);
    if (n < 0) return -1;
    (void)n_nodes;
    const int N = 3 * n;
    double *Ke = malloc(sizeof(double) * N * N);
    double *Ce = malloc(sizeof(double) * N * N);
    double *Me = malloc(sizeof(double) * N * N);
    if (!Ke || !Ce || !Me) {
        free(Ke);
        free(Ce);
        free(Me);
        return -2;
    }
    int bad = 0;
    double ve[3 * ORC_MAXN];
    for (int e = 0; e < n_elem; ++e) {
        const int32_t *ce = conn + (size_t)e * n;
        int st = element_matrices_sel(type, nq, ce, X, u, udot, mat + e, sym_only,
                                      a_K != 0.0 ? Ke : NULL, a_C != 0.0 ? Ce : NULL,
                                      a_M != 0.0 ? Me : NULL);
        if (st < 0) {
            bad = -1;
            break;
        }
        bad += st;
        gather(n, ce, v, ve);
        for (int r = 0; r < N; ++r) {
            double s = 0.0;
            for (int c = 0; c < N; ++c) {
                const size_t idx = transpose ? (size_t)c * N + r : (size_t)r * N + c;
                double A = 0.0;
                if (a_K != 0.0) A += a_K * Ke[idx];
                if (a_C != 0.0) A += a_C * Ce[idx];
                if (a_M != 0.0) A += a_M * Me[idx];
                s += A * ve[c];
            }
            y[(size_t)ce[r / 3] * 3 + r % 3] += s;
        }
    }
    free(Ke);
    free(Ce);
    free(Me);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* adjoint                                                                   */
/* ------------------------------------------------------------------------ */

/* dP/dmu and dP/dlam of the elastic laws at fixed F:
 *   SVK (P = lam trE F + 2 mu F E): dP/dlam = trE F, dP/dmu = 2 F E.
 *   NH  (P = mu J^{-2/3}(F - I1/3 F^{-T}) + (lam + 2mu/3)(J-1) J F^{-T}):
 *       dP/dmu  = J^{-2/3}(F - I1/3 F^{-T}) + 2/3 (J-1) J F^{-T},
 *       dP/dlam = (J-1) J F^{-T}.
 *   MR  (mu10 = mu/2 - mu01, mu01 fixed): the same as NH. */
static int stress_param_derivs(const orc_material *m, const double F[9], double dPdmu[9],
                               double dPdlam[9])
{
    if (m->model == 0) {
        double E[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += F[k * 3 + a] * F[k * 3 + b];
                E[a * 3 + b] = 0.5 * (s - (a == b ? 1.0 : 0.0));
            }
        const double trE = E[0] + E[4] + E[8];
        double FE[9];
        matmul3(F, E, FE);
        for (int a = 0; a < 9; ++a) {
            dPdlam[a] = trE * F[a];
            dPdmu[a] = 2.0 * FE[a];
        }
        return 0;
    }
    if (m->model == 1 || m->model == 2) {
        /* MR: mu10 = mu/2 - mu01 with mu01 held fixed, so the mu01 term does not
         * depend on (mu, lam) and the derivatives equal the neo-Hookean ones */
        const double J = det3(F);
        if (!(J > 0.0)) {
            memset(dPdmu, 0, sizeof(double) * 9);
            memset(dPdlam, 0, sizeof(double) * 9);
            return 1;
        }
        double Fi[9], FiT[9];
        inv3(F, J, Fi);
        transpose3(Fi, FiT);
        double I1 = 0.0;
        for (int a = 0; a < 9; ++a) I1 += F[a] * F[a];
        const double Jm23 = 1.0 / (cbrt(J) * cbrt(J));
        for (int a = 0; a < 9; ++a) {
            dPdmu[a] = Jm23 * (F[a] - I1 / 3.0 * FiT[a]) + 2.0 / 3.0 * (J - 1.0) * J * FiT[a];
            dPdlam[a] = (J - 1.0) * J * FiT[a];
        }
        return 0;
    }
    return -1;
}

/* vector-Jacobian products of f_int against a cotangent r:
 *   g_u = K_t^T r and g_udot = C^T r from the assembled closed-form blocks,
 *   g_theta[e] = (r . df/dmu_e, r . df/dlam_e) = sum_q wJ sum_i r_i^T (dP/dtheta) h_i. */
int orc_vjp(int type, int nq, int n_elem, const int32_t *conn, int n_nodes,
            const double *X, const double *u, const double *udot,
            const orc_material *mat, const double *r,
            double *g_u, double *g_udot, double *g_theta)
{
    int bad = 0;
    if (g_u) {
        int st = orc_operator_apply(type, nq, n_elem, conn, n_nodes, X, u, udot, mat, 0.0, 1.0,
                                    0.0, 1, 0, r, g_u);
        if (st < 0) return st;
        bad += st;
    }
    if (g_udot) {
        int st = orc_operator_apply(type, nq, n_elem, conn, n_nodes, X, u, udot, mat, 0.0, 0.0,
                                    1.0, 1, 0, r, g_udot);
        if (st < 0) return st;
    }
    if (g_theta) {
        const int n = orc_nodes_per_elem(type);
        double Xe[3 * ORC_MAXN], ue[3 * ORC_MAXN], re[3 * ORC_MAXN], F[9], dmu[9], dlam[9];
        elem_geom g;
        for (int e = 0; e < n_elem; ++e) {
            const int32_t *ce = conn + (size_t)e * n;
            if (element_geometry(type, nq, ce, X, &g) < 0) return -1;
            gather(n, ce, X, Xe);
            gather(n, ce, u, ue);
            gather(n, ce, r, re);
            double gm = 0.0, gl = 0.0;
            for (int q = 0; q < nq; ++q) {
                const double *He = g.H + q * n * 3;
                deformation_gradient(n, He, Xe, ue, 2, F);
                if (stress_param_derivs(mat + e, F, dmu, dlam) < 0) return -1;
                for (int i = 0; i < n; ++i) {
                    double a[3], b[3];
                    matvec3(dmu, He + i * 3, a);
                    matvec3(dlam, He + i * 3, b);
                    gm += g.wJ[q] * dot3(re + i * 3, a);
                    gl += g.wJ[q] * dot3(re + i * 3, b);
                }
            }
            g_theta[(size_t)e * 2 + 0] = gm;
            g_theta[(size_t)e * 2 + 1] = gl;
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1-4.2: mass row sums and the uniform force field                    */
/* ------------------------------------------------------------------------ */

int orc_lumped_row_sums(int type, int n_elem, const int32_t *conn, int n_nodes,
                        const double *X, const orc_material *mat, double *m_row)
{
    const int n = orc_nodes_per_elem(type);
    if (n < 0) return -1;
    (void)n_nodes;
    double Me[100];
    for (int e = 0; e < n_elem; ++e) {
        const int32_t *ce = conn + (size_t)e * n;
        if (element_mass(type, ce, X, mat[e].rho, Me, NULL)) return -1;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += Me[i * n + j];
            m_row[ce[i]] += s;
        }
    }
    return 0;
}

/* f^ff_i = rho v_i b0, v_i = int s_i dV_r (Eq. virtual_work_force_field_uniform) */
int orc_gravity(int type, int n_elem, const int32_t *conn, int n_nodes, const double *X,
                const orc_material *mat, const double g[3], double *f_ff)
{
    const int n = orc_nodes_per_elem(type);
    if (n < 0) return -1;
    (void)n_nodes;
    double vs[ORC_MAXN];
    for (int e = 0; e < n_elem; ++e) {
        const int32_t *ce = conn + (size_t)e * n;
        if (element_mass(type, ce, X, 1.0, NULL, vs)) return -1;
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) f_ff[(size_t)ce[i] * 3 + a] += mat[e].rho * vs[i] * g[a];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4 (Pointwise External Force Loads, Surface Traction Loads)           */
/* ------------------------------------------------------------------------ */

/* f_iP = s_i(xi_P) f_P (Eq. virtual_work_point_force_discrete), assembled:
 * load k acts at parent point xi[k] of element elem[k] (0-based within this
 * connectivity) with force[k]. Adds into f. */
int orc_point_loads(int type, int n_loads, const int32_t *conn, const int32_t *elem, const double *xi,
                    const double *force, double *f)
{
    const int n = orc_nodes_per_elem(type);
    if (n < 0) return -1;
    double s[ORC_MAXN];
    for (int k = 0; k < n_loads; ++k) {
        if (orc_shape(type, xi + 3 * k, s)) return -1;
        const int32_t *ce = conn + (size_t)elem[k] * n;
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) f[(size_t)ce[i] * 3 + a] += s[i] * force[3 * k + a];
    }
    return 0;
}

/* Face `face` of the parent element as a map (a, b) -> xi with its tangents
 * dxi/da, dxi/db:
 *   tetrahedra: face k lies opposite barycentric vertex k (L_k = 0); with the
 *     other vertices p < q < r, L_p = 1 - a - b, L_q = a, L_r = b on the unit
 *     triangle; xi = (L_2, L_3, L_4) in the 1-based numbering of App. A.1;
 *   bricks: face 2 d + s is xi_d = (s ? +1 : -1); (a, b) are the other two
 *     parent coordinates in increasing order, on [-1, 1]^2. */
static int face_map(int type, int face, double a, double b, double xi[3], double ta[3], double tb[3])
{
    if (type == 0 || type == 1) {
        if (face < 0 || face > 3) return -1;
        int v[3], m = 0;
        for (int j = 0; j < 4; ++j)
            if (j != face) v[m++] = j;
        double L[4] = {0, 0, 0, 0}, La[4] = {0, 0, 0, 0}, Lb[4] = {0, 0, 0, 0};
        L[v[0]] = 1.0 - a - b;
        L[v[1]] = a;
        L[v[2]] = b;
        La[v[0]] = -1.0;
        La[v[1]] = 1.0;
        Lb[v[0]] = -1.0;
        Lb[v[2]] = 1.0;
        for (int c = 0; c < 3; ++c) {
            xi[c] = L[c + 1];
            ta[c] = La[c + 1];
            tb[c] = Lb[c + 1];
        }
        return 0;
    }
    if (type == 2 || type == 3) {
        if (face < 0 || face > 5) return -1;
        const int d = face / 2, sgn = face % 2;
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        for (int c = 0; c < 3; ++c) ta[c] = tb[c] = 0.0;
        xi[d] = sgn ? 1.0 : -1.0;
        xi[d1] = a;
        xi[d2] = b;
        ta[d1] = 1.0;
        tb[d2] = 1.0;
        return 0;
    }
    return -1;
}

/* Face rule: tetrahedron faces 4 x 4 collapsed Gauss-Legendre on the unit
 * triangle ((a, b) = (u, (1 - u) v), weight (1 - u)); brick faces (H8, Q27)
 * 3 x 3 Gauss-Legendre, exact for the biquadratic face shape functions of a
 * flat face. Returns the number of points. */
static int face_rule(int type, double *pa, double *pb, double *pw)
{
    double gx[4], gw[4];
    if (type == 0 || type == 1) {
        gauss_legendre(4, gx, gw);
        int q = 0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j, ++q) {
                const double u = 0.5 * (gx[i] + 1.0), v = 0.5 * (gx[j] + 1.0);
                pa[q] = u;
                pb[q] = (1.0 - u) * v;
                pw[q] = 0.25 * gw[i] * gw[j] * (1.0 - u);
            }
        return 16;
    }
    gauss_legendre(3, gx, gw);
    int q = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j, ++q) {
            pa[q] = gx[i];
            pb[q] = gx[j];
            pw[q] = gw[i] * gw[j];
        }
    return 9;
}

/* f_i^tr = int_{Gamma_t0} s_i t0 dA0 (Eq. virtual_work_traction_discrete) for a
 * nominal traction t0 constant over each loaded face, by boundary quadrature
 * on the reference configuration: dA0 = |dX/da x dX/db| da db with
 * X(a, b) = sum_i X_i s_i(xi(a, b)). Face k is face fid[k] of element
 * elem[k]; adds into f. */
int orc_surface_traction(int type, int n_faces, const int32_t *conn, const double *X, const int32_t *elem,
                         const int32_t *fid, const double *t0, double *f)
{
    const int n = orc_nodes_per_elem(type);
    if (n < 0) return -1;
    double pa[16], pb[16], pw[16], s[ORC_MAXN], Hp[3 * ORC_MAXN];
    const int nq = face_rule(type, pa, pb, pw);
    for (int k = 0; k < n_faces; ++k) {
        const int32_t *ce = conn + (size_t)elem[k] * n;
        for (int q = 0; q < nq; ++q) {
            double xi[3], ta[3], tb[3];
            if (face_map(type, fid[k], pa[q], pb[q], xi, ta, tb)) return -1;
            orc_shape(type, xi, s);
            orc_shape_grad(type, xi, Hp);
            double Xa[3] = {0, 0, 0}, Xb[3] = {0, 0, 0};
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) {
                    const double xic = X[(size_t)ce[i] * 3 + c];
                    for (int d = 0; d < 3; ++d) {
                        Xa[c] += xic * Hp[i * 3 + d] * ta[d];
                        Xb[c] += xic * Hp[i * 3 + d] * tb[d];
                    }
                }
            const double nx = Xa[1] * Xb[2] - Xa[2] * Xb[1], ny = Xa[2] * Xb[0] - Xa[0] * Xb[2],
                         nz = Xa[0] * Xb[1] - Xa[1] * Xb[0];
            const double dA = sqrt(nx * nx + ny * ny + nz * nz) * pw[q];
            for (int i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) f[(size_t)ce[i] * 3 + a] += s[i] * t0[3 * k + a] * dA;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Bilateral constraints (Sec. 3.x primitives DP1, DP2, DIST, CD)            */
/* ------------------------------------------------------------------------ */

/* Position r of constraint point p: sum_i s_i(xi_p) (X_i + u_i) of element
 * elem[p] (point evaluation through the shape functions); elem[p] < 0 is a
 * fixed ground point at world coordinates xi_p. */
static void con_point(int type, const orc_constraint *k, int p, const int32_t *conn, const double *X,
                      const double *u, double r[3])
{
    if (k->elem[p] < 0) {
        for (int a = 0; a < 3; ++a) r[a] = k->xi[p][a];
        return;
    }
    const int n = orc_nodes_per_elem(type);
    double s[ORC_MAXN];
    orc_shape(type, k->xi[p], s);
    const int32_t *ce = conn + (size_t)k->elem[p] * n;
    for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        for (int i = 0; i < n; ++i) v += s[i] * (X[(size_t)ce[i] * 3 + a] + (u ? u[(size_t)ce[i] * 3 + a] : 0.0));
        r[a] = v;
    }
}

static int con_npoints(int ctype) { return (ctype == 2 || ctype == 3) ? 4 : 2; }

/* c and dc/dr_p of one constraint:
 *   CD  : c = d.(r_Q - r_P) - f;            dc/dr_P = -d, dc/dr_Q = +d
 *   DIST: c = 1/2 (a.a - f^2), a = r_Q - r_P; dc/dr_P = -a, dc/dr_Q = +a
 *   DP1, DP2: c = a.b - f, a = r_Q - r_P, b = r_T - r_R;
 *         dc/dr_P = -b, dc/dr_Q = +b, dc/dr_R = -a, dc/dr_T = +a
 * (Eqs. cd_constraint, dist_constraint, dp1_constraint, dp2_constraint and their blocks). */
static int con_eval(int type, const orc_constraint *k, const int32_t *conn, const double *X, const double *u,
                    double *c, double gp[4][3])
{
    double r[4][3];
    const int np = con_npoints(k->type);
    for (int p = 0; p < np; ++p) con_point(type, k, p, conn, X, u, r[p]);
    double a[3], b[3];
    for (int q = 0; q < 3; ++q) a[q] = r[1][q] - r[0][q];
    memset(gp, 0, sizeof(double) * 12);
    if (k->type == 0) {
        *c = dot3(k->d, a) - k->f;
        for (int q = 0; q < 3; ++q) {
            gp[0][q] = -k->d[q];
            gp[1][q] = k->d[q];
        }
    } else if (k->type == 1) {
        *c = 0.5 * (dot3(a, a) - k->f * k->f);
        for (int q = 0; q < 3; ++q) {
            gp[0][q] = -a[q];
            gp[1][q] = a[q];
        }
    } else if (k->type == 2 || k->type == 3) {
        for (int q = 0; q < 3; ++q) b[q] = r[3][q] - r[2][q];
        *c = dot3(a, b) - k->f;
        for (int q = 0; q < 3; ++q) {
            gp[0][q] = -b[q];
            gp[1][q] = b[q];
            gp[2][q] = -a[q];
            gp[3][q] = a[q];
        }
    } else {
        return -1;
    }
    return 0;
}

/* c(q) for every constraint, q = X + u */
int orc_constraint_eval(int type, int n_cons, const orc_constraint *cons, const int32_t *conn, const double *X,
                        const double *u, double *c)
{
    double gp[4][3];
    for (int k = 0; k < n_cons; ++k)
        if (con_eval(type, cons + k, conn, X, u, c + k, gp)) return -1;
    return 0;
}

/* f += C_q^T w: for each constraint k and point p on an element, node i of
 * that element receives w_k s_i(xi_p) dc_k/dr_p (the element blocks above,
 * applied without forming C_q) */
int orc_constraint_jt(int type, int n_cons, const orc_constraint *cons, const int32_t *conn, const double *X,
                      const double *u, const double *w, double *f)
{
    const int n = orc_nodes_per_elem(type);
    double gp[4][3], c, s[ORC_MAXN];
    for (int k = 0; k < n_cons; ++k) {
        const orc_constraint *ck = cons + k;
        if (con_eval(type, ck, conn, X, u, &c, gp)) return -1;
        for (int p = 0; p < con_npoints(ck->type); ++p) {
            if (ck->elem[p] < 0) continue;
            orc_shape(type, ck->xi[p], s);
            const int32_t *ce = conn + (size_t)ck->elem[p] * n;
            for (int i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) f[(size_t)ce[i] * 3 + a] += w[k] * s[i] * gp[p][a];
        }
    }
    return 0;
}

/* Row weights of the constraint set (Eq. row_weights), constant, from the
 * reference configuration q = X: a DP1 row gets w = 1 / sqrt(|a0|^2 + |b0|^2)
 * with its directions a0 = r_Q - r_P and b0 = r_T - r_R there; CD rows (and
 * the DIST and DP2 rows, which the equation does not scale) get 1. A DP1 row
 * whose reference directions both vanish keeps 1. */
int orc_constraint_row_weights(int type, int n_cons, const orc_constraint *cons, const int32_t *conn,
                               const double *X, double *w)
{
    for (int k = 0; k < n_cons; ++k) {
        w[k] = 1.0;
        if (cons[k].type != 2) continue;
        double r[4][3], a0[3], b0[3];
        for (int p = 0; p < 4; ++p) con_point(type, cons + k, p, conn, X, NULL, r[p]);
        for (int q = 0; q < 3; ++q) {
            a0[q] = r[1][q] - r[0][q];
            b0[q] = r[3][q] - r[2][q];
        }
        const double s2 = dot3(a0, a0) + dot3(b0, b0);
        if (s2 > 0.0) w[k] = 1.0 / sqrt(s2);
    }
    return 0;
}

/* out = C_q v */
int orc_constraint_j(int type, int n_cons, const orc_constraint *cons, const int32_t *conn, const double *X,
                     const double *u, const double *v, double *out)
{
    const int n = orc_nodes_per_elem(type);
    double gp[4][3], c, s[ORC_MAXN];
    for (int k = 0; k < n_cons; ++k) {
        const orc_constraint *ck = cons + k;
        if (con_eval(type, ck, conn, X, u, &c, gp)) return -1;
        double acc = 0.0;
        for (int p = 0; p < con_npoints(ck->type); ++p) {
            if (ck->elem[p] < 0) continue;
            orc_shape(type, ck->xi[p], s);
            const int32_t *ce = conn + (size_t)ck->elem[p] * n;
            for (int i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) acc += gp[p][a] * s[i] * v[(size_t)ce[i] * 3 + a];
        }
        out[k] = acc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 7: backward-Euler step (augmented-Lagrangian constraints optional) */
/* ------------------------------------------------------------------------ */

typedef struct {
    int type, nq, n_elem, n, n_nodes;
    const int32_t *conn;
    const double *X;
    const orc_material *mat;
    const uint8_t *fixed;
    double *A; /* element matrices [n_elem][3n][3n] of M/h + h K^e + C */
    /* augmented-Lagrangian constraints (Sec. 7): none when n_cons = 0 */
    int n_cons;
    const orc_constraint *cons;
    const double *lam;
    const double *wrow; /* [n_cons] row weights w_k (Eq. row_weights), or NULL for all ones */
    double rho, h;
    const double *uq;  /* q(v) - X at which C_q is evaluated */
    double *cw;        /* [n_cons] scratch */
} step_ctx;

static double row_w(const step_ctx *c, int k) { return c->wrow ? c->wrow[k] : 1.0; }

static void project(const step_ctx *c, double *x)
{
    if (!c->fixed) return;
    for (int i = 0; i < c->n_nodes; ++i)
        if (c->fixed[i]) x[i * 3] = x[i * 3 + 1] = x[i * 3 + 2] = 0.0;
}

static double norm2(const double *x, size_t N)
{
    double s = 0.0;
    for (size_t i = 0; i < N; ++i) s += x[i] * x[i];
    return sqrt(s);
}

/* g(v) = 1/h M (v - v_n) + f_int(q(v), v) - f_ff + h C^_q^T (lam + rho c^)
 * with q(v) = q_n + h v (Eqs. step_map_velocity_level and residual, f_ext = 0)
 * and the row-normalised constraints c^ = W c, C^_q = W C_q (Eq. rev_normalized);
 * clamped DOFs are projected out. */
static int residual(const step_ctx *c, const double *u_n, const double *v_n, const double *v,
                    double h, const double *f_ff, double *u_tmp, double *dv, double *g)
{
    const size_t N = (size_t)c->n_nodes * 3;
    for (size_t k = 0; k < N; ++k) {
        u_tmp[k] = u_n[k] + h * v[k];
        dv[k] = v[k] - v_n[k];
        g[k] = -f_ff[k];
    }
    int st = orc_operator_apply(c->type, c->nq, c->n_elem, c->conn, c->n_nodes, c->X, u_tmp,
                                NULL, c->mat, 1.0 / h, 0.0, 0.0, 0, 1, dv, g);
    if (st < 0) return st;
    int st2 = orc_internal_force(c->type, c->nq, c->n_elem, c->conn, c->n_nodes, c->X, u_tmp, v,
                                 c->mat, 2, g);
    if (st2 < 0) return st2;
    if (c->n_cons > 0) {
        if (orc_constraint_eval(c->type, c->n_cons, c->cons, c->conn, c->X, u_tmp, c->cw)) return -1;
        for (int k = 0; k < c->n_cons; ++k) c->cw[k] = h * row_w(c, k) * (c->lam[k] + c->rho * row_w(c, k) * c->cw[k]);
        if (orc_constraint_jt(c->type, c->n_cons, c->cons, c->conn, c->X, u_tmp, c->cw, g)) return -1;
    }
    project(c, g);
    return st + st2;
}

static void apply_A(const step_ctx *c, const double *x, double *y)
{
    const int N = 3 * c->n;
    memset(y, 0, sizeof(double) * c->n_nodes * 3);
    for (int e = 0; e < c->n_elem; ++e) {
        const int32_t *ce = c->conn + (size_t)e * c->n;
        const double *Ae = c->A + (size_t)e * N * N;
        for (int r = 0; r < N; ++r) {
            double s = 0.0;
            for (int q = 0; q < N; ++q) s += Ae[(size_t)r * N + q] * x[(size_t)ce[q / 3] * 3 + q % 3];
            y[(size_t)ce[r / 3] * 3 + r % 3] += s;
        }
    }
    if (c->n_cons > 0) {
        /* Gauss-Newton constraint term h^2 rho C^_q^T C^_q (the curvature terms
         * h^2 sum eta_k grad^2 c_k are left out, App. B.2) */
        orc_constraint_j(c->type, c->n_cons, c->cons, c->conn, c->X, c->uq, x, c->cw);
        for (int k = 0; k < c->n_cons; ++k) c->cw[k] *= c->h * c->h * c->rho * row_w(c, k) * row_w(c, k);
        orc_constraint_jt(c->type, c->n_cons, c->cons, c->conn, c->X, c->uq, c->cw, y);
    }
    project(c, y);
}

/* Inexact Newton on g(v) = 0 at fixed multipliers. Each iteration solves
 * (M/h + h K^e + C [+ h^2 rho C_q^T C_q]) dv = -g with Jacobi-preconditioned
 * CG (the symmetric, Gauss-Newton part of dg/dv), then v += dv. Stops when
 * ||g|| <= rtol g_ref, g_ref = ||g|| at the start (or *g_ref_io when it is
 * positive on entry; it returns the reference used). v_out holds the start. */
static int newton_core(int type, int nq, int n_elem, const int32_t *conn, int n_nodes, const double *X,
                       const orc_material *mat, const double *u_n, const double *v_n, double h,
                       const double gravity[3], const uint8_t *fixed, double newton_rtol, double cg_rtol,
                       int max_newton, int max_cg, int n_cons, const orc_constraint *cons, const double *lam,
                       const double *wrow, double rho, double *g_ref_io, double *v_out, orc_report *rep)
{
    const int n = orc_nodes_per_elem(type);
    if (n < 0 || h <= 0.0) return -1;
    const int NE = 3 * n;
    const size_t N = (size_t)n_nodes * 3;
    step_ctx c = {type, nq, n_elem, n, n_nodes, conn, X, mat, fixed, NULL, n_cons, cons, lam, wrow, rho, h, NULL, NULL};
    double *cw = malloc(sizeof(double) * (n_cons > 0 ? n_cons : 1));
    c.cw = cw;
    c.A = malloc(sizeof(double) * (size_t)n_elem * NE * NE);
    double *f_ff = calloc(N, sizeof(double)), *g = malloc(N * sizeof(double)),
           *ut = malloc(N * sizeof(double)), *dv = malloc(N * sizeof(double)),
           *D = malloc(N * sizeof(double)), *r = malloc(N * sizeof(double)),
           *z = malloc(N * sizeof(double)), *p = malloc(N * sizeof(double)),
           *Ap = malloc(N * sizeof(double)), *x = malloc(N * sizeof(double));
    double *Ke = malloc(sizeof(double) * NE * NE), *Ce = malloc(sizeof(double) * NE * NE),
           *Me = malloc(sizeof(double) * NE * NE);
    int ret = 0;
    rep->newton_iters = 0;
    rep->cg_iters = 0;
    rep->status = 0;
    rep->rel_residual = 0.0;
    if (!c.A || !f_ff || !g || !ut || !dv || !D || !r || !z || !p || !Ap || !x || !Ke || !Ce || !Me) {
        ret = -2;
        goto done;
    }
    orc_gravity(type, n_elem, conn, n_nodes, X, mat, gravity, f_ff);
    project(&c, v_out);
    c.uq = ut;
    if (residual(&c, u_n, v_n, v_out, h, f_ff, ut, dv, g) < 0) {
        ret = -1;
        goto done;
    }
    double g0 = norm2(g, N);
    if (g_ref_io) {
        if (*g_ref_io > 0.0) g0 = *g_ref_io;
        else *g_ref_io = g0;
    }
    double gn = norm2(g, N);
    int it = 0;
    while (g0 > 0.0 && gn > newton_rtol * g0 && it < max_newton) {
        /* assemble element matrices of the symmetric Newton operator at v */
        for (size_t k = 0; k < N; ++k) ut[k] = u_n[k] + h * v_out[k];
        memset(D, 0, N * sizeof(double));
        for (int e = 0; e < n_elem; ++e) {
            const int32_t *ce = conn + (size_t)e * n;
            int st = element_matrices_sel(type, nq, ce, X, ut, v_out, mat + e, 1, Ke, Ce, Me);
            if (st < 0) {
                ret = -1;
                goto done;
            }
            double *Ae = c.A + (size_t)e * NE * NE;
            for (int k = 0; k < NE * NE; ++k) Ae[k] = Me[k] / h + h * Ke[k] + Ce[k];
            for (int q = 0; q < NE; ++q) D[(size_t)ce[q / 3] * 3 + q % 3] += Ae[(size_t)q * NE + q];
        }
        if (n_cons > 0) {
            /* diagonal of h^2 rho C^_q^T C^_q: sum over constraint points of (w_k s_i dc/dr_p)^2 */
            double gp[4][3], cv, sh[ORC_MAXN];
            for (int k = 0; k < n_cons; ++k) {
                con_eval(type, cons + k, conn, X, ut, &cv, gp);
                const double wk2 = row_w(&c, k) * row_w(&c, k);
                for (int pp = 0; pp < con_npoints(cons[k].type); ++pp) {
                    if (cons[k].elem[pp] < 0) continue;
                    orc_shape(type, cons[k].xi[pp], sh);
                    const int32_t *ce = conn + (size_t)cons[k].elem[pp] * n;
                    for (int i = 0; i < n; ++i)
                        for (int a = 0; a < 3; ++a)
                            D[(size_t)ce[i] * 3 + a] += h * h * rho * wk2 * sh[i] * sh[i] * gp[pp][a] * gp[pp][a];
                }
            }
        }
        /* Jacobi-PCG on A x = -g */
        for (size_t k = 0; k < N; ++k) {
            x[k] = 0.0;
            r[k] = -g[k];
        }
        project(&c, r);
        const double r0 = norm2(r, N);
        for (size_t k = 0; k < N; ++k) z[k] = (D[k] != 0.0) ? r[k] / D[k] : 0.0;
        project(&c, z);
        memcpy(p, z, N * sizeof(double));
        double rz = 0.0;
        for (size_t k = 0; k < N; ++k) rz += r[k] * z[k];
        int k_cg = 0;
        while (norm2(r, N) > cg_rtol * r0 && k_cg < max_cg) {
            apply_A(&c, p, Ap);
            double pAp = 0.0;
            for (size_t k = 0; k < N; ++k) pAp += p[k] * Ap[k];
            const double alpha = rz / pAp;
            for (size_t k = 0; k < N; ++k) {
                x[k] += alpha * p[k];
                r[k] -= alpha * Ap[k];
            }
            for (size_t k = 0; k < N; ++k) z[k] = (D[k] != 0.0) ? r[k] / D[k] : 0.0;
            project(&c, z);
            double rz1 = 0.0;
            for (size_t k = 0; k < N; ++k) rz1 += r[k] * z[k];
            const double beta = rz1 / rz;
            rz = rz1;
            for (size_t k = 0; k < N; ++k) p[k] = z[k] + beta * p[k];
            ++k_cg;
        }
        rep->cg_iters += k_cg;
        for (size_t k = 0; k < N; ++k) v_out[k] += x[k];
        project(&c, v_out);
        if (residual(&c, u_n, v_n, v_out, h, f_ff, ut, dv, g) < 0) {
            ret = -1;
            goto done;
        }
        gn = norm2(g, N);
        ++it;
    }
    rep->newton_iters = it;
    rep->rel_residual = g0 > 0.0 ? gn / g0 : 0.0;
    rep->status = (g0 > 0.0 && gn > newton_rtol * g0) ? 5 : 0;
done:
    free(cw);
    free(c.A);
    free(f_ff);
    free(g);
    free(ut);
    free(dv);
    free(D);
    free(r);
    free(z);
    free(p);
    free(Ap);
    free(x);
    free(Ke);
    free(Ce);
    free(Me);
    return ret;
}

int orc_newton_step(int type, int nq, int n_elem, const int32_t *conn, int n_nodes,
                    const double *X, const orc_material *mat, const double *u_n,
                    const double *v_n, double h, const double gravity[3],
                    const uint8_t *fixed, double newton_rtol, double cg_rtol,
                    int max_newton, int max_cg, double *v_out, orc_report *rep)
{
    memcpy(v_out, v_n, (size_t)n_nodes * 3 * sizeof(double));
    return newton_core(type, nq, n_elem, conn, n_nodes, X, mat, u_n, v_n, h, gravity, fixed, newton_rtol, cg_rtol,
                       max_newton, max_cg, 0, NULL, NULL, NULL, 0.0, NULL, v_out, rep);
}

/* Augmented-Lagrangian step (Sec. 7, Eq. alm_multiplier_update): alternate the
 * inner Newton solve of g(v, lam) = 0 with lam += rho c^(q(v)) until
 * ||c^(q(v))||_2 <= alm_tol or max_outer updates; lam is updated in place.
 * With row_norm, c^ = W c holds the row-normalised constraints of Eqs.
 * row_weights and rev_normalized (lam are their multipliers); without it,
 * W = I. Reports the outer iterations and ||c^||. */
int orc_newton_step_alm(int type, int nq, int n_elem, const int32_t *conn, int n_nodes, const double *X,
                        const orc_material *mat, const double *u_n, const double *v_n, double h,
                        const double gravity[3], const uint8_t *fixed, double newton_rtol, double cg_rtol,
                        int max_newton, int max_cg, int n_cons, const orc_constraint *cons, double rho,
                        double alm_tol, int max_outer, int row_norm, double *lam, double *v_out, orc_report *rep,
                        int *outer_iters, double *c_norm)
{
    const size_t N = (size_t)n_nodes * 3;
    double *uq = malloc(N * sizeof(double)), *cv = malloc(sizeof(double) * (n_cons > 0 ? n_cons : 1)),
           *wr = malloc(sizeof(double) * (n_cons > 0 ? n_cons : 1));
    if (!uq || !cv || !wr) {
        free(uq);
        free(cv);
        free(wr);
        return -2;
    }
    for (int j = 0; j < n_cons; ++j) wr[j] = 1.0;
    if (row_norm) orc_constraint_row_weights(type, n_cons, cons, conn, X, wr);
    memcpy(v_out, v_n, N * sizeof(double));
    int ret = 0, k = 0;
    double g_ref = 0.0; /* inner solves stop relative to the first residual of the step */
    orc_report r1;
    rep->newton_iters = rep->cg_iters = 0;
    for (;;) {
        ret = newton_core(type, nq, n_elem, conn, n_nodes, X, mat, u_n, v_n, h, gravity, fixed, newton_rtol,
                          cg_rtol, max_newton, max_cg, n_cons, cons, lam, wr, rho, &g_ref, v_out, &r1);
        if (ret < 0) break;
        rep->newton_iters += r1.newton_iters;
        rep->cg_iters += r1.cg_iters;
        rep->status = r1.status;
        rep->rel_residual = r1.rel_residual;
        for (size_t q = 0; q < N; ++q) uq[q] = u_n[q] + h * v_out[q];
        orc_constraint_eval(type, n_cons, cons, conn, X, uq, cv);
        for (int j = 0; j < n_cons; ++j) cv[j] *= wr[j];
        *c_norm = norm2(cv, (size_t)n_cons);
        if (*c_norm <= alm_tol || k >= max_outer) break;
        for (int j = 0; j < n_cons; ++j) lam[j] += rho * cv[j];
        ++k;
    }
    *outer_iters = k;
    if (ret >= 0 && *c_norm > alm_tol) rep->status = 5;
    free(uq);
    free(cv);
    free(wr);
    return ret;
}

/* ------------------------------------------------------------------------ */
/* conflict colouring                                                         */
/* ------------------------------------------------------------------------ */

/* splitmix64 finaliser (Steele, Lea and Flood 2014), applied to x + golden gamma */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static const uint64_t *g_prio;
static int cmp_prio_desc(const void *a, const void *b)
{
    const uint64_t pa = g_prio[*(const int32_t *)a], pb = g_prio[*(const int32_t *)b];
    return pa < pb ? 1 : (pa > pb ? -1 : 0);
}

/* Two elements conflict iff they share a node. Elements are visited in
 * descending priority p(e) = splitmix64(e xor seed); each takes the smallest
 * colour not held by an already coloured conflicting element. */
int orc_color_greedy(int n_elem, int npe, const int32_t *conn, int n_nodes, uint64_t seed,
                     int32_t *color)
{
    uint64_t *prio = malloc(sizeof(uint64_t) * (size_t)n_elem);
    int32_t *order = malloc(sizeof(int32_t) * (size_t)n_elem);
    int32_t *deg = calloc((size_t)n_nodes + 1, sizeof(int32_t));
    if (!prio || !order || !deg) return -2;
    for (int e = 0; e < n_elem; ++e) {
        prio[e] = orc_splitmix64((uint64_t)e ^ seed);
        order[e] = e;
        color[e] = -1;
        for (int i = 0; i < npe; ++i) deg[conn[(size_t)e * npe + i] + 1]++;
    }
    for (int k = 0; k < n_nodes; ++k) deg[k + 1] += deg[k];
    int32_t *inc = malloc(sizeof(int32_t) * (size_t)n_elem * npe);
    int32_t *fill = calloc((size_t)n_nodes, sizeof(int32_t));
    for (int e = 0; e < n_elem; ++e)
        for (int i = 0; i < npe; ++i) {
            const int nd = conn[(size_t)e * npe + i];
            inc[deg[nd] + fill[nd]++] = e;
        }
    g_prio = prio;
    qsort(order, (size_t)n_elem, sizeof(int32_t), cmp_prio_desc);
    int cap = 4096, ncol = 0;
    int32_t *stamp = malloc(sizeof(int32_t) * cap);
    for (int k = 0; k < cap; ++k) stamp[k] = -1;
    for (int t = 0; t < n_elem; ++t) {
        const int e = order[t];
        for (int i = 0; i < npe; ++i) {
            const int nd = conn[(size_t)e * npe + i];
            for (int k = deg[nd]; k < deg[nd + 1]; ++k) {
                const int c = color[inc[k]];
                if (c >= 0 && c < cap) stamp[c] = e;
            }
        }
        int c = 0;
        while (c < cap && stamp[c] == e) ++c;
        color[e] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(stamp);
    free(prio);
    free(order);
    free(deg);
    free(inc);
    free(fill);
    return ncol;
}
