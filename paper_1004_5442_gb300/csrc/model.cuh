// model.cuh - the D2V16 MRT-FDLB model as the GPU kernels apply it.
//
// The 16 velocities form four groups of four (Sect. "Construction of
// energy-conserving MRT LB model", velocity table):
//   g = 0: speed 1 on the axes, eta^2 = 25/4;  g = 1: speed 6 on the axes;
//   g = 2: sqrt(2)(+-1,+-1);                    g = 3: (3/sqrt(2))(+-1,+-1).
// Members of an axis group: +x, +y, -x, -y; of a diagonal group:
// (+,+), (-,+), (-,-), (+,-).  Per group the four values are combined into
//   S = f0+f1+f2+f3, Dx, Dy, and Q (axis: (f0+f2)-(f1+f3)) or
//   X (diagonal: (f0+f2)-(f1+f3)),
// and every Appendix moment row m_k is a combination of one kind of these
// over the groups (the rows split by their symmetry under the square's
// rotations and reflections):
//   (m1, m4, m5, m14)  from S_0..S_3      4x4 block A
//   (m2, m8, m10, m12) from Dx_0..Dx_3    4x4 block B
//   (m3, m9, m11, m13) from Dy_0..Dy_3    B with the m13 row negated
//   (m6, m16)          from Q_0, Q_1      2x2 block C1
//   (m7, m15)          from X_2, X_3      2x2 block C2
// so M f costs 32 adds plus 56 multiply-adds instead of 256, and M^-1 is
// the inverse of these blocks followed by the inverse butterflies.  The
// blocks are built and inverted on the host in FP64 (mrt_model_build) and
// passed to the kernels as FP32 or FP64 constants.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mrt {

constexpr int NV = 16;

// Per-group constants: component magnitude u (speed on an axis, or the
// common |v_x| = |v_y| of a diagonal), V = |v|^2 and W = |v|^2 + eta^2.
__host__ __device__ constexpr double kU(int g) {
    return g == 0 ? 1.0 : g == 1 ? 6.0 : g == 2 ? 1.4142135623730951 : 2.1213203435596424;
}
__host__ __device__ constexpr double kV(int g) { return g == 0 ? 1.0 : g == 1 ? 36.0 : g == 2 ? 4.0 : 9.0; }
__host__ __device__ constexpr double kW(int g) { return g == 0 ? 7.25 : g == 1 ? 36.0 : g == 2 ? 4.0 : 9.0; }

// Plane of the velocity mirrored across a wall normal to x (axis 0) or to y
// (axis 1).  Inside a group of four the order is (1,0),(0,1),(-1,0),(0,-1)
// for the axis groups and (1,1),(-1,1),(-1,-1),(1,-1) for the diagonal ones.
__host__ __device__ constexpr int mirror_plane(int i, int axis) {
    const int g = i >> 2, k = i & 3;
    if (g < 2) return 4 * g + (axis == 0 ? (k == 0 ? 2 : k == 2 ? 0 : k) : (k == 1 ? 3 : k == 3 ? 1 : k));
    return 4 * g + (axis == 0 ? (k ^ 1) : (3 - k));
}

// FP64 only: the inverse-block constants with each moment's sigma_k folded
// in (so the relaxation costs one subtraction per moment instead of two
// operations), and the centre weights of the Lax-Wendroff update written as
// a0 f + p f_up + q f_down (+ the diagonal groups' second axis), so that
// one multiply-add takes each neighbour.  FP64 runs on a pipe that retires
// two lanes per clock per SM, which bounds the FP64 step; the FP32 step is
// bound by HBM and keeps the difference form, which leaves a uniform state
// exactly unchanged.  Empty for FP32, so the per-instance constant table of
// the batched kernel keeps its size.
template <class T>
struct CoefFold {};
template <>
struct CoefFold<double> {
    double kSs[4][2];  // kS[g][j] * (sigma_5, sigma_14)
    double kDx[4][3];  // kD[g][j] * (sigma_8, sigma_10, sigma_12)
    double kDy[4][3];  // kD[g][j] * (sigma_9, sigma_11, sigma_13)
    double kQs[2][2];  // kQ[g][j] * (sigma_6, sigma_16)
    double kXs[2][2];  // kX[g][j] * (sigma_7, sigma_15)
    double lw0[4];     // centre weight: 1 - c^2 (axis groups), 1 - 2 c^2 (diagonal groups)
};

// Everything a step kernel needs besides the state.
template <class T>
struct Coef : CoefFold<T> {
    // Collision increment dt*Omega in the combined basis, already scaled by
    // the inverse butterflies' 1/4 or 1/2 and by -1:
    T kS[4][2];   // S_g    <- (Delta_5, Delta_14)
    T kD[4][3];   // Dx_g   <- (Delta_8, Delta_10, Delta_12); Dy_g <- (Delta_9, Delta_11, -Delta_13)
    T kQ[2][2];   // Q_g    <- (Delta_6, Delta_16), g = 0, 1
    T kX[2][2];   // X_g    <- (Delta_7, Delta_15), g = 2, 3
    T sig[12];    // sigma_k = s_k dt for k = 5..16
    // Lax-Wendroff weights per group with c = u_g dt/dx:
    // p = (c^2 + c)/2 on the upwind neighbour, q = (c^2 - c)/2 on the other.
    T lwp[4], lwq[4];
    // Mixed term of the unsplit two-dimensional operator on the diagonal
    // groups 2, 3: |c_x c_y| / 4 = (u_g dt/dx)^2 / 4.
    T kxy[2];
    T inv_b;      // 1/b
    T c14a;       // 2 (b + 2)
    T c14b;       // 6 + b
    T c15;        // b + 4
};

// Host-side, FP64: builds the blocks from (u, V, W), inverts them and fills
// the FP64 constants; returns 0 on success.  dx, dt, b and s[16] as given.
int mrt_model_build(double dx, double dt, double b, const double s[16], Coef<double>* out);

// Full (unscaled) block inverses, used by the initialisation kernel to map
// equilibrium moments to f.  Ainv[g][k]: k over (m1, m4, m5, m14);
// Binv[g][k]: k over (m2, m8, m10, m12); C1inv / C2inv over (m6, m16) / (m7, m15).
struct InitCoef {
    double Ainv[4][4];
    double Binv[4][4];
    double C1inv[2][2];
    double C2inv[2][2];
    double b;
};
int mrt_init_coef_build(double b, InitCoef* out);

template <class Dst, class Src>
inline void coef_cast(const Coef<Src>& a, Coef<Dst>* o) {
    for (int g = 0; g < 4; ++g) {
        for (int j = 0; j < 2; ++j) o->kS[g][j] = (Dst)a.kS[g][j];
        for (int j = 0; j < 3; ++j) o->kD[g][j] = (Dst)a.kD[g][j];
        o->lwp[g] = (Dst)a.lwp[g];
        o->lwq[g] = (Dst)a.lwq[g];
    }
    for (int g = 0; g < 2; ++g) {
        for (int j = 0; j < 2; ++j) {
            o->kQ[g][j] = (Dst)a.kQ[g][j];
            o->kX[g][j] = (Dst)a.kX[g][j];
        }
        o->kxy[g] = (Dst)a.kxy[g];
    }
    for (int k = 0; k < 12; ++k) o->sig[k] = (Dst)a.sig[k];
    o->inv_b = (Dst)a.inv_b;
    o->c14a = (Dst)a.c14a;
    o->c14b = (Dst)a.c14b;
    o->c15 = (Dst)a.c15;
}

#ifdef __CUDACC__

// Stencil positions handed to a fetch functor; the four diagonal
// neighbours are read only by the unsplit operator (XT).
enum Pos { C = 0, XM = 1, XP = 2, YM = 3, YP = 4, XPYP = 5, XPYM = 6, XMYP = 7, XMYM = 8 };

// Conserved moments (rho, jx, jy, e) of a 16-vector, from the group sums.
template <class T>
__device__ __forceinline__ void conserved_moments(const T f[NV], T& rho, T& jx, T& jy, T& e) {
    T S[4], Dx[4], Dy[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const T* q = f + 4 * g;
        const T d02 = q[0] - q[2], d13 = q[1] - q[3];
        S[g] = (q[0] + q[2]) + (q[1] + q[3]);
        if (g < 2) { Dx[g] = d02; Dy[g] = d13; }
        else { Dx[g] = d02 - d13; Dy[g] = d02 + d13; }
    }
    rho = (S[0] + S[1]) + (S[2] + S[3]);
    jx = (T)kU(0) * Dx[0] + (T)kU(1) * Dx[1] + (T)kU(2) * Dx[2] + (T)kU(3) * Dx[3];
    jy = (T)kU(0) * Dy[0] + (T)kU(1) * Dy[1] + (T)kU(2) * Dy[2] + (T)kU(3) * Dy[3];
    e = (T)kW(0) * S[0] + (T)kW(1) * S[1] + (T)kW(2) * S[2] + (T)kW(3) * S[3];
}

template <class T>
__device__ __forceinline__ T recip(T x) { return (T)1 / x; }
template <>
__device__ __forceinline__ float recip<float>(float x) { return __fdividef(1.0f, x); }

// One cell of one time step (Eq. 3, forward Euler + Lax-Wendroff):
// reads the stencil through F(i, pos), writes f^{n+1} to out and returns
// the cell's input rho and P for the health check.
//
// The Lax-Wendroff terms are accumulated as multiply-adds of neighbour
// differences onto the collision increment, so a uniform state is left
// exactly unchanged by the advection in any precision.
//
// XT: the unsplit two-dimensional Lax-Wendroff operator, which adds to each
// diagonal velocity the mixed term (c_x c_y / 4)(f(x+1,y+1) - f(x+1,y-1)
// - f(x-1,y+1) + f(x-1,y-1)) of the second-order Taylor expansion in time
// (c_x c_y > 0 for (+,+) and (-,-), < 0 for (-,+) and (+,-)).
template <class T, bool XT = false, class Fetch>
__device__ __forceinline__ void cell_update(const Fetch& F, const Coef<T>& k, T out[NV],
                                            T& rho_in, T& P_in) {
    T f[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) f[i] = F(i, C);

    // ---- forward transform: butterflies, then the five blocks ----------
    T S[4], Dx[4], Dy[4], QX[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const T* q = f + 4 * g;
        const T s02 = q[0] + q[2], s13 = q[1] + q[3];
        const T d02 = q[0] - q[2], d13 = q[1] - q[3];
        S[g] = s02 + s13;
        QX[g] = s02 - s13;
        if (g < 2) { Dx[g] = d02; Dy[g] = d13; }
        else { Dx[g] = d02 - d13; Dy[g] = d02 + d13; }
    }
    // eta^2 = 25/4 on group 0 only, so W_g = V_g except W_0 = V_0 + 25/4.
    constexpr double E2 = 6.25;
    const T m1 = (S[0] + S[1]) + (S[2] + S[3]);
    const T m5 = (T)kV(0) * S[0] + (T)kV(1) * S[1] + (T)kV(2) * S[2] + (T)kV(3) * S[3];
    const T m4 = (T)E2 * S[0] + m5;
    const T m14 = (T)(kV(0) * kW(0)) * S[0] + (T)(kV(1) * kW(1)) * S[1]
                + (T)(kV(2) * kW(2)) * S[2] + (T)(kV(3) * kW(3)) * S[3];
    const T m2 = (T)kU(0) * Dx[0] + (T)kU(1) * Dx[1] + (T)kU(2) * Dx[2] + (T)kU(3) * Dx[3];
    const T m12 = (T)(kU(1) * kV(1)) * Dx[1] + Dx[0];                 // u^3 on the axis groups
    const T m10 = (T)(kU(3) * kV(3)) * Dx[3] + ((T)(kU(2) * kV(2)) * Dx[2] + m12);
    const T m8 = (T)E2 * Dx[0] + m10;
    const T m3 = (T)kU(0) * Dy[0] + (T)kU(1) * Dy[1] + (T)kU(2) * Dy[2] + (T)kU(3) * Dy[3];
    const T n13 = (T)(kU(1) * kV(1)) * Dy[1] + Dy[0];                 // -m13
    const T m11 = (T)(kU(3) * kV(3)) * Dy[3] + ((T)(kU(2) * kV(2)) * Dy[2] + n13);
    const T m9 = (T)E2 * Dy[0] + m11;
    const T m6 = (T)kV(1) * QX[1] + QX[0];
    const T m16 = (T)(kV(1) * kW(1)) * QX[1] + (T)(kV(0) * kW(0)) * QX[0];
    const T m7 = (T)(0.5 * kV(3)) * QX[3] + (T)(0.5 * kV(2)) * QX[2];
    const T m15 = (T)(0.5 * kV(3) * kW(3)) * QX[3] + (T)(0.5 * kV(2) * kW(2)) * QX[2];

    // ---- equilibrium moments (Appendix), P = (e - j^2/rho)/b, R = 1 ------
    const T rho = m1, jx = m2, jy = m3, e = m4;
    const T rinv = recip<T>(rho);
    const T ux = jx * rinv, uy = jy * rinv;
    const T kx = jx * ux, ky = jy * uy;
    const T j2r = kx + ky;                       // j^2 / rho
    const T P = (e - j2r) * k.inv_b;
    const T Tt = P * rinv;
    const T twoP = P + P;
    const T q5 = twoP + j2r;
    const T q6 = kx - ky;                        // (jx^2 - jy^2)/rho
    const T q7 = jx * uy;
    const T e2P = e + twoP;
    const T q8 = e2P * ux, q9 = e2P * uy;
    const T h10 = twoP + q5;                     // 4P + j^2/rho
    const T q10 = h10 * ux, q11 = h10 * uy;
    const T q12 = (twoP + q6) * ux;
    const T nq13 = (twoP - q6) * uy;             // -q13
    const T u2 = ux * ux + uy * uy;
    const T q14 = Tt * (k.c14a * P + k.c14b * j2r) + j2r * u2;
    const T g15 = k.c15 * P + j2r;
    const T q15 = g15 * (ux * uy);
    const T q16 = g15 * (ux * ux - uy * uy);
    rho_in = rho;
    P_in = P;

    // ---- relaxation Delta_k = sigma_k (m_k - m^eq_k), k = 5..16 ---------
    // (FP64: the residuals m_k - m^eq_k alone; sigma_k is in the constants)
    constexpr bool kFold = sizeof(T) == 8;
    auto relax = [&](int j, T r) -> T {
        if constexpr (kFold) return r; else return k.sig[j] * r;
    };
    const T d5 = relax(0, m5 - q5), d6 = relax(1, m6 - q6), d7 = relax(2, m7 - q7);
    const T d8 = relax(3, m8 - q8), d9 = relax(4, m9 - q9);
    const T d10 = relax(5, m10 - q10), d11 = relax(6, m11 - q11);
    const T d12 = relax(7, m12 - q12), nd13 = relax(8, n13 - nq13);   // -Delta_13
    const T d14 = relax(9, m14 - q14), d15 = relax(10, m15 - q15);
    const T d16 = relax(11, m16 - q16);

    // ---- inverse blocks (scaled), inverse butterflies, then advection ----
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        T cS, cX, cY;
        if constexpr (kFold) {
            cS = k.kSs[g][0] * d5 + k.kSs[g][1] * d14;
            cX = k.kDx[g][0] * d8 + k.kDx[g][1] * d10 + k.kDx[g][2] * d12;
            cY = k.kDy[g][0] * d9 + k.kDy[g][1] * d11 + k.kDy[g][2] * nd13;
        } else {
            cS = k.kS[g][0] * d5 + k.kS[g][1] * d14;
            cX = k.kD[g][0] * d8 + k.kD[g][1] * d10 + k.kD[g][2] * d12;
            cY = k.kD[g][0] * d9 + k.kD[g][1] * d11 + k.kD[g][2] * nd13;
        }
        const T p = k.lwp[g], qq = k.lwq[g];
        const int i0 = 4 * g;
        if constexpr (kFold) {
          if (g < 2) {
            // FP64: out = a0 f + p f_up + q f_down + collision, one
            // multiply-add per neighbour (+x: p on x-1, q on x+1; -x mirrored;
            // +y / -y likewise along y)
            const T cQ = k.kQs[g][0] * d6 + k.kQs[g][1] * d16;
            const T sp = cS + cQ, sm = cS - cQ;
            const T a0 = k.lw0[g];
            out[i0 + 0] = a0 * f[i0 + 0] + (p * F(i0 + 0, XM) + (qq * F(i0 + 0, XP) + (sp + cX)));
            out[i0 + 2] = a0 * f[i0 + 2] + (p * F(i0 + 2, XP) + (qq * F(i0 + 2, XM) + (sp - cX)));
            out[i0 + 1] = a0 * f[i0 + 1] + (p * F(i0 + 1, YM) + (qq * F(i0 + 1, YP) + (sm + cY)));
            out[i0 + 3] = a0 * f[i0 + 3] + (p * F(i0 + 3, YP) + (qq * F(i0 + 3, YM) + (sm - cY)));
          } else {
            // FP64 diagonal groups: a0 = 1 - 2 c^2; the mixed term of the
            // unsplit operator enters as four more multiply-adds
            const T cXY = k.kXs[g - 2][0] * d7 + k.kXs[g - 2][1] * d15;
            const T t1 = cS + cXY, t2 = cS - cXY, s1 = cX + cY, s2 = cX - cY;
            const T a0 = k.lw0[g];
            auto mixed = [&](int i, T w, T acc) -> T {
                if constexpr (XT)
                    return w * F(i, XPYP) + (-w * F(i, XPYM) + (-w * F(i, XMYP) + (w * F(i, XMYM) + acc)));
                else
                    return acc;
            };
            const T w = XT ? k.kxy[g - 2] : (T)0;
            {   // (+,+): p on x-1, y-1; q on x+1, y+1
                const T c0 = mixed(i0 + 0, w, t1 + s1);
                out[i0 + 0] = a0 * f[i0 + 0] + (p * (F(i0 + 0, XM) + F(i0 + 0, YM)) +
                                                 (qq * (F(i0 + 0, XP) + F(i0 + 0, YP)) + c0));
            }
            {   // (-,+): p on x+1, y-1; q on x-1, y+1
                const T c1 = mixed(i0 + 1, -w, t2 - s2);
                out[i0 + 1] = a0 * f[i0 + 1] + (p * (F(i0 + 1, XP) + F(i0 + 1, YM)) +
                                                 (qq * (F(i0 + 1, XM) + F(i0 + 1, YP)) + c1));
            }
            {   // (-,-): p on x+1, y+1; q on x-1, y-1
                const T c2 = mixed(i0 + 2, w, t1 - s1);
                out[i0 + 2] = a0 * f[i0 + 2] + (p * (F(i0 + 2, XP) + F(i0 + 2, YP)) +
                                                 (qq * (F(i0 + 2, XM) + F(i0 + 2, YM)) + c2));
            }
            {   // (+,-): p on x-1, y+1; q on x+1, y-1
                const T c3 = mixed(i0 + 3, -w, t2 + s2);
                out[i0 + 3] = a0 * f[i0 + 3] + (p * (F(i0 + 3, XM) + F(i0 + 3, YP)) +
                                                 (qq * (F(i0 + 3, XP) + F(i0 + 3, YM)) + c3));
            }
          }
        } else {
          if (g < 2) {
            const T cQ = k.kQ[g][0] * d6 + k.kQ[g][1] * d16;
            const T sp = cS + cQ, sm = cS - cQ;
            // +x: p on x-1, q on x+1; -x mirrored; +y / -y likewise along y
            {
                const T fc = f[i0 + 0];
                T t = qq * (F(i0 + 0, XP) - fc) + (sp + cX);
                out[i0 + 0] = fc + (p * (F(i0 + 0, XM) - fc) + t);
            }
            {
                const T fc = f[i0 + 2];
                T t = p * (F(i0 + 2, XP) - fc) + (sp - cX);
                out[i0 + 2] = fc + (qq * (F(i0 + 2, XM) - fc) + t);
            }
            {
                const T fc = f[i0 + 1];
                T t = qq * (F(i0 + 1, YP) - fc) + (sm + cY);
                out[i0 + 1] = fc + (p * (F(i0 + 1, YM) - fc) + t);
            }
            {
                const T fc = f[i0 + 3];
                T t = p * (F(i0 + 3, YP) - fc) + (sm - cY);
                out[i0 + 3] = fc + (qq * (F(i0 + 3, YM) - fc) + t);
            }
        } else {
            const T cXY = k.kX[g - 2][0] * d7 + k.kX[g - 2][1] * d15;
            const T t1 = cS + cXY, t2 = cS - cXY, s1 = cX + cY, s2 = cX - cY;
            // XT: mixed terms, (f++ - f+-) - (f-+ - f--) scaled by |c_x c_y|/4
            // and signed by c_x c_y; exactly 0 on a uniform state
            T e0 = 0, e1 = 0, e2 = 0, e3 = 0;
            auto with_mixed = [](T v, T e) -> T {
                if constexpr (XT) return v + e; else return v;
            };
            if constexpr (XT) {
                const T w = k.kxy[g - 2];
                auto mixed = [&](int i) { return (F(i, XPYP) - F(i, XPYM)) - (F(i, XMYP) - F(i, XMYM)); };
                e0 = w * mixed(i0 + 0);
                e1 = -(w * mixed(i0 + 1));
                e2 = w * mixed(i0 + 2);
                e3 = -(w * mixed(i0 + 3));
            }
            // |c_x| = |c_y| on a diagonal: pair the x and y neighbours that
            // carry the same weight, (a + b - 2 f) is exact for a uniform state
            {   // (+,+): p on x-1, y-1; q on x+1, y+1
                const T fc = f[i0 + 0];
                const T a = (F(i0 + 0, XM) + F(i0 + 0, YM)) - (fc + fc);
                const T b = (F(i0 + 0, XP) + F(i0 + 0, YP)) - (fc + fc);
                out[i0 + 0] = fc + (p * a + (qq * b + with_mixed((t1 + s1), e0)));
            }
            {   // (-,+): q on x-1, p on x+1; p on y-1, q on y+1
                const T fc = f[i0 + 1];
                const T a = (F(i0 + 1, XP) + F(i0 + 1, YM)) - (fc + fc);
                const T b = (F(i0 + 1, XM) + F(i0 + 1, YP)) - (fc + fc);
                out[i0 + 1] = fc + (p * a + (qq * b + with_mixed((t2 - s2), e1)));
            }
            {   // (-,-): q on x-1, y-1; p on x+1, y+1
                const T fc = f[i0 + 2];
                const T a = (F(i0 + 2, XP) + F(i0 + 2, YP)) - (fc + fc);
                const T b = (F(i0 + 2, XM) + F(i0 + 2, YM)) - (fc + fc);
                out[i0 + 2] = fc + (p * a + (qq * b + with_mixed((t1 - s1), e2)));
            }
            {   // (+,-): p on x-1, q on x+1; q on y-1, p on y+1
                const T fc = f[i0 + 3];
                const T a = (F(i0 + 3, XM) + F(i0 + 3, YP)) - (fc + fc);
                const T b = (F(i0 + 3, XP) + F(i0 + 3, YM)) - (fc + fc);
                out[i0 + 3] = fc + (p * a + (qq * b + with_mixed((t2 + s2), e3)));
            }
          }
        }
    }
}

#endif  // __CUDACC__

}  // namespace mrt
