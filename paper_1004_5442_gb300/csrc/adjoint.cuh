// adjoint.cuh - reverse mode of one cell of the fused step (model.cuh).
//
// With f^{n+1} = f + Adv(f) + dt Omega(f), lam = dL/df^{n+1} and
// mu = M^-T lam:
//   dL/df^n     = lam + Adv^T(lam) - M^T (I - JE)^T S mu     (per cell)
//   dL/dsigma_k += -mu_k (m_k - m^eq_k),  k = 5..16,  sigma_k = s_k dt
// where JE = d fhat^eq / d fhat is non-zero only in the columns of
// (rho, jx, jy, e) and rows 1..4 of (I - JE) vanish.  Adv^T is the same
// Lax-Wendroff stencil with the two neighbour weights exchanged (c -> -c).
//
// In the group-combination basis the forward increment is
//   dt Omega_i = sum_k (coef of Delta_k for the group of i) * (sign of i in
//   the butterfly of that k) * Delta_k,
// so mu_k = -sum_g coef_g,k * butterfly_g,k(lam): the forward constants and
// butterflies serve the transpose too.  d fhat^eq / d(rho, j, e) is applied
// as a reverse sweep through the Appendix formulas (adj_equilibrium).
#pragma once
#include "model.cuh"

namespace mrt {

#ifdef __CUDACC__

// Reverse sweep of the equilibria: given nu_5..nu_16, returns the gradient
// of sum_k nu_k fhat^eq_k(rho, jx, jy, e) with respect to (rho, jx, jy, e).
template <class T>
__device__ __forceinline__ void adj_equilibrium(T rho, T jx, T jy, T e, const Coef<T>& k, const T nu[12],
                                                T& a_rho, T& a_jx, T& a_jy, T& a_e) {
    // forward intermediates (as in cell_update)
    const T rinv = (T)1 / rho;
    const T ux = jx * rinv, uy = jy * rinv;
    const T kx = jx * ux, ky = jy * uy;
    const T j2r = kx + ky;
    const T P = (e - j2r) * k.inv_b;
    const T Tt = P * rinv;
    const T twoP = P + P;
    const T q5 = twoP + j2r;
    const T q6 = kx - ky;
    const T e2P = e + twoP;
    const T h10 = twoP + q5;
    const T u2 = ux * ux + uy * uy;
    const T A14 = k.c14a * P + k.c14b * j2r;
    const T g15 = k.c15 * P + j2r;
    const T n5 = nu[0], n6 = nu[1], n7 = nu[2], n8 = nu[3], n9 = nu[4], n10 = nu[5];
    const T n11 = nu[6], n12 = nu[7], n13 = nu[8], n14 = nu[9], n15 = nu[10], n16 = nu[11];
    // q15 = g15 ux uy, q16 = g15 (ux^2 - uy^2)
    const T a_g15 = n15 * (ux * uy) + n16 * (ux * ux - uy * uy);
    T a_ux = n15 * g15 * uy + n16 * g15 * (ux + ux);
    T a_uy = n15 * g15 * ux - n16 * g15 * (uy + uy);
    // q14 = Tt A14 + j2r u2
    const T a_Tt = n14 * A14;
    T a_P = n14 * Tt * k.c14a;
    T a_j2r = n14 * (Tt * k.c14b + u2);
    const T a_u2 = n14 * j2r;
    // g15 = c15 P + j2r
    a_P += k.c15 * a_g15;
    a_j2r += a_g15;
    // u2 = ux^2 + uy^2
    a_ux += (ux + ux) * a_u2;
    a_uy += (uy + uy) * a_u2;
    // q13 = (q6 - 2P) uy, q12 = (2P + q6) ux
    T a_q6 = n13 * uy + n12 * ux;
    T a_twoP = n12 * ux - n13 * uy;
    a_uy += n13 * (q6 - twoP);
    a_ux += n12 * (twoP + q6);
    // q10 = h10 ux, q11 = h10 uy, h10 = 2P + q5
    const T a_h10 = n10 * ux + n11 * uy;
    a_ux += n10 * h10;
    a_uy += n11 * h10;
    a_twoP += a_h10;
    const T a_q5 = n5 + a_h10;
    // q8 = e2P ux, q9 = e2P uy, e2P = e + 2P
    const T a_e2P = n8 * ux + n9 * uy;
    a_ux += n8 * e2P;
    a_uy += n9 * e2P;
    T ae = a_e2P;
    a_twoP += a_e2P;
    // q7 = jx uy
    T ajx = n7 * uy;
    a_uy += n7 * jx;
    // q6 = kx - ky
    a_q6 += n6;
    T a_kx = a_q6, a_ky = -a_q6;
    // q5 = 2P + j2r
    a_twoP += a_q5;
    a_j2r += a_q5;
    a_P += a_twoP + a_twoP;
    // Tt = P rinv
    a_P += a_Tt * rinv;
    T a_rinv = a_Tt * P;
    // P = (e - j2r)/b
    ae += a_P * k.inv_b;
    a_j2r -= a_P * k.inv_b;
    // j2r = kx + ky, kx = jx ux, ky = jy uy
    a_kx += a_j2r;
    a_ky += a_j2r;
    ajx += a_kx * ux;
    a_ux += a_kx * jx;
    T ajy = a_ky * uy;
    a_uy += a_ky * jy;
    // ux = jx rinv, uy = jy rinv
    ajx += a_ux * rinv;
    a_rinv += a_ux * jx;
    ajy += a_uy * rinv;
    a_rinv += a_uy * jy;
    a_rho = -a_rinv * rinv * rinv;
    a_jx = ajx;
    a_jy = ajy;
    a_e = ae;
}

// Butterfly of one group of four values (axis: Dx = v0-v2, Dy = v1-v3,
// Q = (v0+v2)-(v1+v3); diagonal: Dx = (v0-v2)-(v1-v3), Dy = (v0-v2)+(v1-v3),
// X = (v0+v2)-(v1+v3)).
template <class T>
__device__ __forceinline__ void butterfly(int g, const T* v, T& S, T& Dx, T& Dy, T& QX) {
    const T s02 = v[0] + v[2], s13 = v[1] + v[3];
    const T d02 = v[0] - v[2], d13 = v[1] - v[3];
    S = s02 + s13;
    QX = s02 - s13;
    if (g < 2) { Dx = d02; Dy = d13; }
    else { Dx = d02 - d13; Dy = d02 + d13; }
}

// |c_x c_y| / 4 of diagonal group g (2 or 3); 0 on the axis groups.
template <class T>
__device__ __forceinline__ T k_xy(const Coef<T>& k, int g) {
    return g >= 2 ? k.kxy[g - 2] : (T)0;
}

// Forward Lax-Wendroff weight that plane i puts on its neighbour at pos
// (the weight multiplies (f_pos - f_centre)).
template <class T>
__device__ __forceinline__ T lw_weight(const Coef<T>& k, int i, int pos) {
    const int g = i >> 2, m = i & 3;
    const T p = k.lwp[g], q = k.lwq[g];
    int sx, sy;  // direction signs of the velocity
    if (g < 2) { sx = m == 0 ? 1 : m == 2 ? -1 : 0; sy = m == 1 ? 1 : m == 3 ? -1 : 0; }
    else { sx = (m == 0 || m == 3) ? 1 : -1; sy = (m == 0 || m == 1) ? 1 : -1; }
    switch (pos) {
        case XM: return sx == 0 ? (T)0 : (sx > 0 ? p : q);
        case XP: return sx == 0 ? (T)0 : (sx > 0 ? q : p);
        case YM: return sy == 0 ? (T)0 : (sy > 0 ? p : q);
        default: return sy == 0 ? (T)0 : (sy > 0 ? q : p);
    }
}

// One cell of the reverse step.  LF(i, pos) reads lam = dL/df^{n+1} on the
// stencil (ghost values of fixed axes are zero), f[] is f^n at the cell.
// Writes lam_out = dL/df^n at the cell and adds -mu_k (m_k - m^eq_k) to
// gsig[k-5].  XT: the unsplit operator; its mixed term is symmetric (the
// weight on f(x+a, y+b) is c_x c_y a b / 4 = the weight on f(x-a, y-b)), so
// its transpose is the same term applied to lam.
template <class T, bool XT = false, class LFetch>
__device__ __forceinline__ void cell_adjoint(const LFetch& LF, const T f[NV], const Coef<T>& k, T lam_out[NV],
                                             T gsig[12]) {
    // ---- forward moments and equilibria of f^n ----------------------------
    T S[4], Dx[4], Dy[4], QX[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) butterfly<T>(g, f + 4 * g, S[g], Dx[g], Dy[g], QX[g]);
    const T m1 = (S[0] + S[1]) + (S[2] + S[3]);
    T m[12];  // m_5 .. m_16
    T mw[4];  // rho, jx, jy, e
    {
        const T m5 = (T)kV(0) * S[0] + (T)kV(1) * S[1] + (T)kV(2) * S[2] + (T)kV(3) * S[3];
        const T m4 = (T)6.25 * S[0] + m5;
        m[0] = m5;
        m[9] = (T)(kV(0) * kW(0)) * S[0] + (T)(kV(1) * kW(1)) * S[1] + (T)(kV(2) * kW(2)) * S[2] +
               (T)(kV(3) * kW(3)) * S[3];
        const T m2 = (T)kU(0) * Dx[0] + (T)kU(1) * Dx[1] + (T)kU(2) * Dx[2] + (T)kU(3) * Dx[3];
        m[7] = (T)(kU(1) * kV(1)) * Dx[1] + Dx[0];                                        // m12
        m[5] = (T)(kU(3) * kV(3)) * Dx[3] + ((T)(kU(2) * kV(2)) * Dx[2] + m[7]);          // m10
        m[3] = (T)6.25 * Dx[0] + m[5];                                                    // m8
        const T m3 = (T)kU(0) * Dy[0] + (T)kU(1) * Dy[1] + (T)kU(2) * Dy[2] + (T)kU(3) * Dy[3];
        const T n13 = (T)(kU(1) * kV(1)) * Dy[1] + Dy[0];
        m[8] = -n13;                                                                      // m13
        m[6] = (T)(kU(3) * kV(3)) * Dy[3] + ((T)(kU(2) * kV(2)) * Dy[2] + n13);           // m11
        m[4] = (T)6.25 * Dy[0] + m[6];                                                    // m9
        m[1] = (T)kV(1) * QX[1] + QX[0];                                                  // m6
        m[11] = (T)(kV(1) * kW(1)) * QX[1] + (T)(kV(0) * kW(0)) * QX[0];                  // m16
        m[2] = (T)(0.5 * kV(3)) * QX[3] + (T)(0.5 * kV(2)) * QX[2];                       // m7
        m[10] = (T)(0.5 * kV(3) * kW(3)) * QX[3] + (T)(0.5 * kV(2) * kW(2)) * QX[2];      // m15
        mw[0] = m1; mw[1] = m2; mw[2] = m3; mw[3] = m4;
    }
    T q[12];
    {
        const T rho = mw[0], jx = mw[1], jy = mw[2], e = mw[3];
        const T rinv = (T)1 / rho;
        const T ux = jx * rinv, uy = jy * rinv;
        const T kx = jx * ux, ky = jy * uy;
        const T j2r = kx + ky;
        const T P = (e - j2r) * k.inv_b;
        const T Tt = P * rinv;
        const T twoP = P + P;
        q[0] = twoP + j2r;
        q[1] = kx - ky;
        q[2] = jx * uy;
        const T e2P = e + twoP;
        q[3] = e2P * ux; q[4] = e2P * uy;
        const T h10 = twoP + q[0];
        q[5] = h10 * ux; q[6] = h10 * uy;
        q[7] = (twoP + q[1]) * ux;
        q[8] = (q[1] - twoP) * uy;
        const T u2 = ux * ux + uy * uy;
        q[9] = Tt * (k.c14a * P + k.c14b * j2r) + j2r * u2;
        const T g15 = k.c15 * P + j2r;
        q[10] = g15 * (ux * uy);
        q[11] = g15 * (ux * ux - uy * uy);
    }

    // ---- mu = M^-T lam (only k = 5..16 are needed) -------------------------
    T lc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) lc[i] = LF(i, C);
    T LS[4], LX[4], LY[4], LQ[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) butterfly<T>(g, lc + 4 * g, LS[g], LX[g], LY[g], LQ[g]);
    T mu[12];
    mu[0] = -(k.kS[0][0] * LS[0] + k.kS[1][0] * LS[1] + k.kS[2][0] * LS[2] + k.kS[3][0] * LS[3]);   // m5
    mu[9] = -(k.kS[0][1] * LS[0] + k.kS[1][1] * LS[1] + k.kS[2][1] * LS[2] + k.kS[3][1] * LS[3]);   // m14
    mu[3] = -(k.kD[0][0] * LX[0] + k.kD[1][0] * LX[1] + k.kD[2][0] * LX[2] + k.kD[3][0] * LX[3]);   // m8
    mu[5] = -(k.kD[0][1] * LX[0] + k.kD[1][1] * LX[1] + k.kD[2][1] * LX[2] + k.kD[3][1] * LX[3]);   // m10
    mu[7] = -(k.kD[0][2] * LX[0] + k.kD[1][2] * LX[1] + k.kD[2][2] * LX[2] + k.kD[3][2] * LX[3]);   // m12
    mu[4] = -(k.kD[0][0] * LY[0] + k.kD[1][0] * LY[1] + k.kD[2][0] * LY[2] + k.kD[3][0] * LY[3]);   // m9
    mu[6] = -(k.kD[0][1] * LY[0] + k.kD[1][1] * LY[1] + k.kD[2][1] * LY[2] + k.kD[3][1] * LY[3]);   // m11
    mu[8] = (k.kD[0][2] * LY[0] + k.kD[1][2] * LY[1] + k.kD[2][2] * LY[2] + k.kD[3][2] * LY[3]);    // m13
    mu[1] = -(k.kQ[0][0] * LQ[0] + k.kQ[1][0] * LQ[1]);                                             // m6
    mu[11] = -(k.kQ[0][1] * LQ[0] + k.kQ[1][1] * LQ[1]);                                            // m16
    mu[2] = -(k.kX[0][0] * LQ[2] + k.kX[1][0] * LQ[3]);                                             // m7
    mu[10] = -(k.kX[0][1] * LQ[2] + k.kX[1][1] * LQ[3]);                                            // m15

    // ---- rate gradients and nu = S mu -------------------------------------
    T nu[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        gsig[j] += -mu[j] * (m[j] - q[j]);
        nu[j] = k.sig[j] * mu[j];
    }
    T a_rho, a_jx, a_jy, a_e;
    adj_equilibrium<T>(mw[0], mw[1], mw[2], mw[3], k, nu, a_rho, a_jx, a_jy, a_e);
    // w = (I - JE)^T nu: w_1..4 = -(a_rho, a_jx, a_jy, a_e), w_5..16 = nu
    const T w1 = -a_rho, w2 = -a_jx, w3 = -a_jy, w4 = -a_e;

    // ---- M^T w: blocks transposed, then the butterfly transposed -----------
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const T u = (T)kU(g), V = (T)kV(g), Wg = (T)kW(g);
        const T bS = w1 + Wg * w4 + V * nu[0] + (T)(kV(g) * kW(g)) * nu[9];
        T bX = u * w2 + (T)(kU(g) * kW(g)) * nu[3] + (T)(kU(g) * kV(g)) * nu[5];
        T bY = u * w3 + (T)(kU(g) * kW(g)) * nu[4] + (T)(kU(g) * kV(g)) * nu[6];
        T c[4];
        if (g < 2) {
            bX += (T)(kU(g) * kV(g)) * nu[7];
            bY -= (T)(kU(g) * kV(g)) * nu[8];
            const T bQ = V * nu[1] + (T)(kV(g) * kW(g)) * nu[11];
            c[0] = bS + bX + bQ;
            c[1] = bS + bY - bQ;
            c[2] = bS - bX + bQ;
            c[3] = bS - bY - bQ;
        } else {
            const T bXY = (T)(0.5 * kV(g)) * nu[2] + (T)(0.5 * kV(g) * kW(g)) * nu[10];
            c[0] = bS + bX + bY + bXY;
            c[1] = bS - bX + bY - bXY;
            c[2] = bS - bX - bY + bXY;
            c[3] = bS + bX - bY - bXY;
        }
        // ---- transposed advection + identity, minus M^T w ----------------
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) {
            const int i = 4 * g + mm;
            const T lcen = lc[i];
            T t = -c[mm];
            // transpose: the weight on f(x-1) in the forward reads lam(x+1) here
            const T wxm = lw_weight<T>(k, i, XM), wxp = lw_weight<T>(k, i, XP);
            const T wym = lw_weight<T>(k, i, YM), wyp = lw_weight<T>(k, i, YP);
            if (g < 2) {
                if (mm == 0 || mm == 2) t += wxm * (LF(i, XP) - lcen) + wxp * (LF(i, XM) - lcen);
                else t += wym * (LF(i, YP) - lcen) + wyp * (LF(i, YM) - lcen);
            } else {
                t += wxm * (LF(i, XP) - lcen) + wxp * (LF(i, XM) - lcen);
                t += wym * (LF(i, YP) - lcen) + wyp * (LF(i, YM) - lcen);
                if constexpr (XT) {
                    // c_x c_y > 0 for (+,+) and (-,-), < 0 for (-,+) and (+,-)
                    const T wxy = (mm == 0 || mm == 2) ? k.kxy[g - 2] : -k.kxy[g - 2];
                    t += wxy * ((LF(i, XPYP) - LF(i, XPYM)) - (LF(i, XMYP) - LF(i, XMYM)));
                }
            }
            lam_out[i] = lcen + t;
        }
    }
}

#endif  // __CUDACC__

}  // namespace mrt
