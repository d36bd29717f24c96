// Device-side element and constitutive math of the TL-FEA hot path.
//
// Everything works in the displacement form of the kinematics: with the
// nodal unknowns x_i = X_i + u_i and U H = I (Sec. 6, H = Hp (U Hp)^{-1}),
// the deformation gradient F = sum_i x_i h_i^T (Sec. 2.1) equals I + G with
// G = sum_i u_i h_i^T. Strain-like quantities are formed from G directly so
// that FP32 keeps its relative accuracy at small strain:
//   E     = (G + G^T + G^T G) / 2
//   b - I = G + G^T + G G^T
//   J - 1 = tr G + I2(G) + det G     (expansion of det(I + G))
// The Mooney-Rivlin stress of App. C (Eq. mr_first_piola; neo-Hookean is
// mu01 = 0) is used in the algebraically equal form
//   P = [ 2 mu10 J^{-5/3} D + 2 mu01 J^{-7/3} dev(I1 b - b^2) + k (J - 1) I ] cof(F)
// with cof(F) = J F^{-T}, D = dev(b - I) and, writing b = I + beta,
//   dev(I1 b - b^2) = (1 + tr(beta)/3) D - dev(D D)
// (I1 F - F C = (I1 b - b^2) F^{-T} and F = b F^{-T}), which needs no division
// by J in the volumetric term and no cancellation of the identity in the
// isochoric ones.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tlfe {

enum { ET_T4 = 0, ET_T10 = 1, ET_H8 = 2, ET_Q27 = 3 };
enum { MODEL_SVK = 0, MODEL_NH = 1, MODEL_MR = 2 };

template <int ET> struct Elem;
template <> struct Elem<ET_T4> { static constexpr int NPE = 4; };
template <> struct Elem<ET_T10> { static constexpr int NPE = 10; };
template <> struct Elem<ET_H8> { static constexpr int NPE = 8; };
template <> struct Elem<ET_Q27> { static constexpr int NPE = 27; };

__host__ __device__ inline int nodes_per_elem(int et)
{
    return et == ET_T4 ? 4 : (et == ET_T10 ? 10 : (et == ET_H8 ? 8 : (et == ET_Q27 ? 27 : -1)));
}

// Material record as the kernels see it (Lame constants, Kelvin-Voigt
// constants, density, Mooney-Rivlin mu01 with mu10 = mu/2 - mu01; mu01 = 0
// unless model == MODEL_MR) in the arithmetic type R.
template <typename R> struct Mat {
    int model;
    R mu, lam, mu_v, lam_v, rho, mu01;
};

// ---------------------------------------------------------------------------
// 3x3 helpers on row-major register arrays
// ---------------------------------------------------------------------------

template <typename R> __device__ __forceinline__ R tr3(const R A[9]) { return A[0] + A[4] + A[8]; }

// cofactor matrix cof(F) (rows = cross products of the other two rows); equals J F^{-T}
template <typename R> __device__ __forceinline__ void cof3(const R F[9], R C[9])
{
    C[0] = F[4] * F[8] - F[5] * F[7];
    C[1] = F[5] * F[6] - F[3] * F[8];
    C[2] = F[3] * F[7] - F[4] * F[6];
    C[3] = F[7] * F[2] - F[8] * F[1];
    C[4] = F[8] * F[0] - F[6] * F[2];
    C[5] = F[6] * F[1] - F[7] * F[0];
    C[6] = F[1] * F[5] - F[2] * F[4];
    C[7] = F[2] * F[3] - F[0] * F[5];
    C[8] = F[0] * F[4] - F[1] * F[3];
}

// directional derivative of cof at F along dF (cof is quadratic in F)
template <typename R> __device__ __forceinline__ void dcof3(const R F[9], const R D[9], R C[9])
{
    C[0] = D[4] * F[8] + F[4] * D[8] - D[5] * F[7] - F[5] * D[7];
    C[1] = D[5] * F[6] + F[5] * D[6] - D[3] * F[8] - F[3] * D[8];
    C[2] = D[3] * F[7] + F[3] * D[7] - D[4] * F[6] - F[4] * D[6];
    C[3] = D[7] * F[2] + F[7] * D[2] - D[8] * F[1] - F[8] * D[1];
    C[4] = D[8] * F[0] + F[8] * D[0] - D[6] * F[2] - F[6] * D[2];
    C[5] = D[6] * F[1] + F[6] * D[1] - D[7] * F[0] - F[7] * D[0];
    C[6] = D[1] * F[5] + F[1] * D[5] - D[2] * F[4] - F[2] * D[4];
    C[7] = D[2] * F[3] + F[2] * D[3] - D[0] * F[5] - F[0] * D[5];
    C[8] = D[0] * F[4] + F[0] * D[4] - D[1] * F[3] - F[1] * D[3];
}

// R = A B
template <typename R> __device__ __forceinline__ void mm3(const R A[9], const R B[9], R C[9])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            C[a * 3 + b] = A[a * 3] * B[b] + A[a * 3 + 1] * B[3 + b] + A[a * 3 + 2] * B[6 + b];
}

// C += A B
template <typename R> __device__ __forceinline__ void mm3_acc(const R A[9], const R B[9], R C[9])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            C[a * 3 + b] += A[a * 3] * B[b] + A[a * 3 + 1] * B[3 + b] + A[a * 3 + 2] * B[6 + b];
}

// FP32 products with rows 0 and 1 paired in packed FP32x2 operations (one
// instruction for two lanes of work; the same operations in the same order
// as the scalar form)
__device__ __forceinline__ void mm3(const float A[9], const float B[9], float C[9])
{
    const float2 a0 = make_float2(A[0], A[3]), a1 = make_float2(A[1], A[4]), a2 = make_float2(A[2], A[5]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float2 q = __fmul2_rn(a0, make_float2(B[b], B[b]));
        q = __ffma2_rn(a1, make_float2(B[3 + b], B[3 + b]), q);
        q = __ffma2_rn(a2, make_float2(B[6 + b], B[6 + b]), q);
        C[b] = q.x;
        C[3 + b] = q.y;
        C[6 + b] = fmaf(A[8], B[6 + b], fmaf(A[7], B[3 + b], A[6] * B[b]));
    }
}
__device__ __forceinline__ void mm3_acc(const float A[9], const float B[9], float C[9])
{
    const float2 a0 = make_float2(A[0], A[3]), a1 = make_float2(A[1], A[4]), a2 = make_float2(A[2], A[5]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float2 q = __fmul2_rn(a0, make_float2(B[b], B[b]));
        q = __ffma2_rn(a1, make_float2(B[3 + b], B[3 + b]), q);
        q = __ffma2_rn(a2, make_float2(B[6 + b], B[6 + b]), q);
        const float2 c = __fadd2_rn(make_float2(C[b], C[3 + b]), q);
        C[b] = c.x;
        C[3 + b] = c.y;
        C[6 + b] += fmaf(A[8], B[6 + b], fmaf(A[7], B[3 + b], A[6] * B[b]));
    }
}

// sym(A^T B) = (A^T B + B^T A) / 2
template <typename R> __device__ __forceinline__ void symAtB(const R A[9], const R B[9], R S[9])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
            R s = A[a] * B[b] + A[3 + a] * B[3 + b] + A[6 + a] * B[6 + b] + B[a] * A[b] +
                  B[3 + a] * A[3 + b] + B[6 + a] * A[6 + b];
            S[a * 3 + b] = R(0.5) * s;
            S[b * 3 + a] = R(0.5) * s;
        }
}

// ---------------------------------------------------------------------------
// Constitutive state at one quadrature point
// ---------------------------------------------------------------------------

// Per-point quantities kept between the stress and its derivatives.
template <typename R> struct QP {
    R F[9];    // I + G
    R G[9];    // sum u_i h_i^T
    R Fd[9];   // sum udot_i h_i^T (valid when visc)
    R S[9];    // SVK: elastic 2nd PK stress; MR / NH: A with P = A cof(F)
    R Sv[9];   // viscous 2nd PK stress
    R Cf[9];   // NH: cof(F)
    R dev[9];  // MR / NH: D = dev(b - I)
    R Jm1, J, Jm53, rJ;  // J - 1, J, J^{-5/3}, 1/J
    R bt;      // MR: tr(b - I) / 3
    bool ok;
};

template <typename R> __device__ __forceinline__ R rcbrt_(R x);
template <> __device__ __forceinline__ float rcbrt_<float>(float x) { return rcbrtf(x); }
template <> __device__ __forceinline__ double rcbrt_<double>(double x) { return rcbrt(x); }

// Elastic + viscous stress. visc: whether Fd is meaningful and the material damped.
// Returns P. Sets q.ok = false (and P = viscous part only) when the
// neo-Hookean law meets J <= 0.
template <typename R>
__device__ __forceinline__ void stress(const Mat<R> &m, QP<R> &q, bool visc, R P[9])
{
    const R *G = q.G;
#pragma unroll
    for (int k = 0; k < 9; ++k) q.F[k] = G[k] + ((k % 4 == 0) ? R(1) : R(0));
    q.ok = true;
    if (visc) {
        // Edot = sym(Fd^T F); S^v = 2 mu_v Edot + lam_v tr(Edot) I  (Sec. 3.2.3)
        R Ed[9];
        symAtB(q.Fd, q.F, Ed);
        const R t = tr3(Ed);
#pragma unroll
        for (int k = 0; k < 9; ++k) q.Sv[k] = R(2) * m.mu_v * Ed[k];
        q.Sv[0] += m.lam_v * t;
        q.Sv[4] += m.lam_v * t;
        q.Sv[8] += m.lam_v * t;
    }
    if (m.model == MODEL_SVK) {
        // E = (G + G^T + G^T G)/2, S = lam tr(E) I + 2 mu E, P = F S  (App. C SVK)
        R E[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) {
                R s = G[a * 3 + b] + G[b * 3 + a] + G[a] * G[b] + G[3 + a] * G[3 + b] + G[6 + a] * G[6 + b];
                E[a * 3 + b] = R(0.5) * s;
                E[b * 3 + a] = R(0.5) * s;
            }
        const R t = tr3(E);
#pragma unroll
        for (int k = 0; k < 9; ++k) q.S[k] = R(2) * m.mu * E[k];
        q.S[0] += m.lam * t;
        q.S[4] += m.lam * t;
        q.S[8] += m.lam * t;
        if (visc) {
            R St[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) St[k] = q.S[k] + q.Sv[k];
            mm3(q.F, St, P);
        } else {
            mm3(q.F, q.S, P);
        }
        return;
    }
    // neo-Hookean: mu10 = mu/2, k = lam + 2 mu / 3
    const R third = R(1.0 / 3.0);
    const R kb = m.lam + R(2) * third * m.mu;
    const R I2 = G[0] * G[4] + G[4] * G[8] + G[0] * G[8] - G[1] * G[3] - G[5] * G[7] - G[2] * G[6];
    const R dG = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                 G[2] * (G[3] * G[7] - G[4] * G[6]);
    q.Jm1 = tr3(G) + I2 + dG;
    q.J = R(1) + q.Jm1;
    if (!(q.J > R(0))) {
        q.ok = false;
#pragma unroll
        for (int k = 0; k < 9; ++k) P[k] = R(0);
        if (visc) mm3(q.F, q.Sv, P);
        return;
    }
    const R r = rcbrt_<R>(q.J);
    const R r2 = r * r;
    const R r3 = r2 * r;  // 1/J
    q.Jm53 = r3 * r2;
    q.rJ = r3;
    // b - I = G + G^T + G G^T
    R bt = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
            R s = G[a * 3 + b] + G[b * 3 + a] + G[a * 3] * G[b * 3] + G[a * 3 + 1] * G[b * 3 + 1] +
                  G[a * 3 + 2] * G[b * 3 + 2];
            q.dev[a * 3 + b] = s;
            q.dev[b * 3 + a] = s;
        }
    bt = tr3(q.dev) * third;
    q.bt = bt;
    q.dev[0] -= bt;
    q.dev[4] -= bt;
    q.dev[8] -= bt;
    const R c1 = (m.mu - R(2) * m.mu01) * q.Jm53;  // 2 mu10 J^{-5/3}
#pragma unroll
    for (int k = 0; k < 9; ++k) q.S[k] = c1 * q.dev[k];
    if (m.model == MODEL_MR) {
        // + 2 mu01 J^{-7/3} [ (1 + tr(beta)/3) D - dev(D D) ]
        const R c2 = R(2) * m.mu01 * q.Jm53 * q.Jm53 * q.J;
        R DD[9];
        mm3(q.dev, q.dev, DD);
        const R t = tr3(DD) * third;
#pragma unroll
        for (int k = 0; k < 9; ++k) q.S[k] += c2 * ((R(1) + bt) * q.dev[k] - DD[k]);
        q.S[0] += c2 * t;
        q.S[4] += c2 * t;
        q.S[8] += c2 * t;
    }
    q.S[0] += kb * q.Jm1;
    q.S[4] += kb * q.Jm1;
    q.S[8] += kb * q.Jm1;
    cof3(q.F, q.Cf);
    mm3(q.S, q.Cf, P);
    if (visc) mm3_acc(q.F, q.Sv, P);
}

// Directional derivative of P along (dF, dFd):
//   dP = D_F P^e[dF] + (position-side viscous terms, if visc_pos)
//        + D_Fd P^v[dFd]  (if has_dFd)
// cK scales everything depending on dF, cC everything depending on dFd.
// sym_only drops the viscous stiffness K^v (the non-symmetric part).
template <typename R>
__device__ __forceinline__ void dstress(const Mat<R> &m, const QP<R> &q, bool visc, const R dF[9],
                                        R cK, R cC, bool sym_only, R dP[9])
{
#pragma unroll
    for (int k = 0; k < 9; ++k) dP[k] = R(0);
    if (cK != R(0)) {
        if (m.model == MODEL_SVK) {
            // dE = sym(F^T dF); dS = lam tr(dE) I + 2 mu dE; dP = dF S + F dS
            R dE[9], dS[9];
            symAtB(q.F, dF, dE);
            const R t = tr3(dE);
#pragma unroll
            for (int k = 0; k < 9; ++k) dS[k] = R(2) * m.mu * dE[k];
            dS[0] += m.lam * t;
            dS[4] += m.lam * t;
            dS[8] += m.lam * t;
            mm3_acc(dF, q.S, dP);
            mm3_acc(q.F, dS, dP);
        } else if (q.ok) {
            const R third = R(1.0 / 3.0);
            const R kb = m.lam + R(2) * third * m.mu;
            // dJ = cof(F) : dF
            R dJ = R(0);
#pragma unroll
            for (int k = 0; k < 9; ++k) dJ += q.Cf[k] * dF[k];
            // d(b - I) = dF + dF^T + dF G^T + G dF^T
            R db[9];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = a; b < 3; ++b) {
                    R s = dF[a * 3 + b] + dF[b * 3 + a] + dF[a * 3] * q.G[b * 3] +
                          dF[a * 3 + 1] * q.G[b * 3 + 1] + dF[a * 3 + 2] * q.G[b * 3 + 2] +
                          q.G[a * 3] * dF[b * 3] + q.G[a * 3 + 1] * dF[b * 3 + 1] +
                          q.G[a * 3 + 2] * dF[b * 3 + 2];
                    db[a * 3 + b] = s;
                    db[b * 3 + a] = s;
                }
            const R dbt = tr3(db) * third;
            db[0] -= dbt;
            db[4] -= dbt;
            db[8] -= dbt;
            const R dJm53 = R(-5.0 / 3.0) * q.Jm53 * dJ * q.rJ;
            const R mu2 = m.mu - R(2) * m.mu01;  // 2 mu10
            R dA[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) dA[k] = mu2 * (dJm53 * q.dev[k] + q.Jm53 * db[k]);
            if (m.model == MODEL_MR) {
                // d{ c2 [ (1 + bt) D - dev(D D) ] }, c2 = 2 mu01 J^{-7/3}
                const R c2 = R(2) * m.mu01 * q.Jm53 * q.Jm53 * q.J;
                const R dc2 = R(-7.0 / 3.0) * c2 * dJ * q.rJ;
                R DD[9], dDD[9];
                mm3(q.dev, q.dev, DD);
                mm3(db, q.dev, dDD);
                mm3_acc(q.dev, db, dDD);
                const R t = tr3(DD) * third, dt = tr3(dDD) * third;
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    dA[k] += dc2 * ((R(1) + q.bt) * q.dev[k] - DD[k]) +
                             c2 * (dbt * q.dev[k] + (R(1) + q.bt) * db[k] - dDD[k]);
                const R iso = dc2 * t + c2 * dt;
                dA[0] += iso;
                dA[4] += iso;
                dA[8] += iso;
            }
            dA[0] += kb * dJ;
            dA[4] += kb * dJ;
            dA[8] += kb * dJ;
            R dC[9];
            dcof3(q.F, dF, dC);
            mm3_acc(dA, q.Cf, dP);
            mm3_acc(q.S, dC, dP);
        }
        if (visc && !sym_only) {
            mm3_acc(dF, q.Sv, dP);  // q.S holds the elastic part only, for both laws
            // F dS^v with dEdot = sym(Fd^T dF)
            R dE[9], dS[9];
            symAtB(q.Fd, dF, dE);
            const R t = tr3(dE);
#pragma unroll
            for (int k = 0; k < 9; ++k) dS[k] = R(2) * m.mu_v * dE[k];
            dS[0] += m.lam_v * t;
            dS[4] += m.lam_v * t;
            dS[8] += m.lam_v * t;
            mm3_acc(q.F, dS, dP);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) dP[k] *= cK;
    }
    if (cC != R(0) && (m.mu_v != R(0) || m.lam_v != R(0))) {
        // velocity direction: dEdot = sym(F^T dFd), dP = F dS^v
        R dE[9], dS[9], T[9];
        symAtB(q.F, dF, dE);
        const R t = tr3(dE);
#pragma unroll
        for (int k = 0; k < 9; ++k) dS[k] = R(2) * m.mu_v * dE[k];
        dS[0] += m.lam_v * t;
        dS[4] += m.lam_v * t;
        dS[8] += m.lam_v * t;
        mm3(q.F, dS, T);
#pragma unroll
        for (int k = 0; k < 9; ++k) dP[k] += cC * T[k];
    }
}

// Adjoint of the stress map at one point against a cotangent Gh (=sum r_i h_i^T):
//   gF  = (dP/dF)^T [Gh]  (elastic part self-adjoint; viscous part explicit)
//   gFd = (dP/dFd)^T [Gh]
//   gmu = dP/dmu : Gh, glam = dP/dlam : Gh
template <typename R>
__device__ __forceinline__ void astress(const Mat<R> &m, const QP<R> &q, bool visc, const R Gh[9],
                                        R gF[9], R gFd[9], R &gmu, R &glam)
{
    dstress<R>(m, q, false, Gh, R(1), R(0), true, gF);
#pragma unroll
    for (int k = 0; k < 9; ++k) gFd[k] = R(0);
    if (visc) {
        // L = (F S^v) : Gh.  Sbar = sym(F^T Gh), Ebar = 2 mu_v Sbar + lam_v tr(Sbar) I
        // dL/dF = Gh S^v + Fd Ebar,  dL/dFd = F Ebar
        R Sb[9], Eb[9];
        symAtB(q.F, Gh, Sb);
        const R t = tr3(Sb);
#pragma unroll
        for (int k = 0; k < 9; ++k) Eb[k] = R(2) * m.mu_v * Sb[k];
        Eb[0] += m.lam_v * t;
        Eb[4] += m.lam_v * t;
        Eb[8] += m.lam_v * t;
        mm3_acc(Gh, q.Sv, gF);
        mm3_acc(q.Fd, Eb, gF);
        mm3(q.F, Eb, gFd);
    }
    gmu = R(0);
    glam = R(0);
    if (m.model == MODEL_SVK) {
        // dP/dlam = tr(E) F, dP/dmu = 2 F E ; E recovered from S = lam trE I + 2 mu E
        // is ill-posed when mu = 0, so recompute E from G.
        R E[9];
        const R *G = q.G;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                E[a * 3 + b] = R(0.5) * (G[a * 3 + b] + G[b * 3 + a] + G[a] * G[b] + G[3 + a] * G[3 + b] +
                                         G[6 + a] * G[6 + b]);
        R FE[9];
        mm3(q.F, E, FE);
        const R t = tr3(E);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            gmu += R(2) * FE[k] * Gh[k];
            glam += t * q.F[k] * Gh[k];
        }
    } else if (q.ok) {
        // P = [(mu - 2 mu01) J^{-5/3} D + 2 mu01 J^{-7/3} D2 + (lam + 2mu/3)(J-1) I] cof with
        // mu01 held fixed: dP/dmu = [J^{-5/3} D + 2/3 (J-1) I] cof, dP/dlam = (J-1) cof
        R Bm[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Bm[k] = q.Jm53 * q.dev[k];
        Bm[0] += R(2.0 / 3.0) * q.Jm1;
        Bm[4] += R(2.0 / 3.0) * q.Jm1;
        Bm[8] += R(2.0 / 3.0) * q.Jm1;
        R Pm[9];
        mm3(Bm, q.Cf, Pm);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            gmu += Pm[k] * Gh[k];
            glam += q.Jm1 * q.Cf[k] * Gh[k];
        }
    }
}

}  // namespace tlfe
