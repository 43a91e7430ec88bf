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

// The cell update is written in phases, so that one thread can run all of
// them for a cell (cell_update) or four threads can share a cell, one per
// velocity group (the split kernel), with bit-identical arithmetic.

// Phase 1, per group g: the butterflies of its four values (the order inside
// a group is (+x, +y, -x, -y) or ((+,+), (-,+), (-,-), (+,-))).
template <class T>
struct GroupSums {
    T S, QX, Dx, Dy;
};
template <class T>
__device__ __forceinline__ GroupSums<T> group_sums(int g, const T q[4]) {
    GroupSums<T> r;
    const T s02 = q[0] + q[2], s13 = q[1] + q[3];
    const T d02 = q[0] - q[2], d13 = q[1] - q[3];
    r.S = s02 + s13;
    r.QX = s02 - s13;
    if (g < 2) { r.Dx = d02; r.Dy = d13; }
    else { r.Dx = d02 - d13; r.Dy = d02 + d13; }
    return r;
}

// Phase 2, per block of moment rows (eta^2 = 25/4 on group 0 only, so
// W_g = V_g except W_0 = V_0 + 25/4):
//   (m1, m5, m4, m14) from S_0..3;  (m2, m12, m10, m8) from Dx_0..3 and
//   (m3, -m13, m11, m9) from Dy_0..3;  (m6, m16, m7, m15) from QX_0..3.
constexpr double kEta2 = 6.25;
template <class T>
__device__ __forceinline__ void moments_S(const T S[4], T m[4]) {
    m[0] = (S[0] + S[1]) + (S[2] + S[3]);
    m[1] = (T)kV(0) * S[0] + (T)kV(1) * S[1] + (T)kV(2) * S[2] + (T)kV(3) * S[3];
    m[2] = (T)kEta2 * S[0] + m[1];
    m[3] = (T)(kV(0) * kW(0)) * S[0] + (T)(kV(1) * kW(1)) * S[1]
         + (T)(kV(2) * kW(2)) * S[2] + (T)(kV(3) * kW(3)) * S[3];
}
template <class T>
__device__ __forceinline__ void moments_D(const T D[4], T m[4]) {
    m[0] = (T)kU(0) * D[0] + (T)kU(1) * D[1] + (T)kU(2) * D[2] + (T)kU(3) * D[3];
    m[1] = (T)(kU(1) * kV(1)) * D[1] + D[0];                 // u^3 on the axis groups
    m[2] = (T)(kU(3) * kV(3)) * D[3] + ((T)(kU(2) * kV(2)) * D[2] + m[1]);
    m[3] = (T)kEta2 * D[0] + m[2];
}
template <class T>
__device__ __forceinline__ void moments_Q(const T QX[4], T m[4]) {
    m[0] = (T)kV(1) * QX[1] + QX[0];
    m[1] = (T)(kV(1) * kW(1)) * QX[1] + (T)(kV(0) * kW(0)) * QX[0];
    m[2] = (T)(0.5 * kV(3)) * QX[3] + (T)(0.5 * kV(2)) * QX[2];
    m[3] = (T)(0.5 * kV(3) * kW(3)) * QX[3] + (T)(0.5 * kV(2) * kW(2)) * QX[2];
}

// Phase 3: the closure P = (e - j^2/rho)/b, T = P/rho (R = 1) and the terms
// the equilibrium moments of every block share (Appendix).
template <class T>
struct EqBase {
    T rinv, ux, uy, kx, ky, j2r, P, Tt, twoP, q5, q6;
};
template <class T>
__device__ __forceinline__ EqBase<T> eq_base(T rho, T jx, T jy, T e, const Coef<T>& k) {
    EqBase<T> b;
    b.rinv = recip<T>(rho);
    b.ux = jx * b.rinv;
    b.uy = jy * b.rinv;
    b.kx = jx * b.ux;
    b.ky = jy * b.uy;
    b.j2r = b.kx + b.ky;                        // j^2 / rho
    b.P = (e - b.j2r) * k.inv_b;
    b.Tt = b.P * b.rinv;
    b.twoP = b.P + b.P;
    b.q5 = b.twoP + b.j2r;
    b.q6 = b.kx - b.ky;                         // (jx^2 - jy^2)/rho
    return b;
}

// Relaxed residuals Delta_k = sigma_k (m_k - m^eq_k), k = 5..16 (-Delta_13 in
// nd13); FP64 keeps m_k - m^eq_k, its constants carry sigma_k.
template <class T>
struct Deltas {
    T d5, d6, d7, d8, d9, d10, d11, d12, nd13, d14, d15, d16;
};
template <class T>
__device__ __forceinline__ T relax(const Coef<T>& k, int j, T r) {
    if constexpr (sizeof(T) == 8) return r; else return k.sig[j] * r;
}
// block S: m5, m14
template <class T>
__device__ __forceinline__ void relax_S(const EqBase<T>& b, T m5, T m14, const Coef<T>& k, Deltas<T>& D) {
    const T u2 = b.ux * b.ux + b.uy * b.uy;
    const T q14 = b.Tt * (k.c14a * b.P + k.c14b * b.j2r) + b.j2r * u2;
    D.d5 = relax(k, 0, m5 - b.q5);
    D.d14 = relax(k, 9, m14 - q14);
}
// block Dx: m8, m10, m12 (e the energy moment m4)
template <class T>
__device__ __forceinline__ void relax_Dx(const EqBase<T>& b, T e, T m8, T m10, T m12, const Coef<T>& k,
                                         Deltas<T>& D) {
    const T e2P = e + b.twoP;
    const T q8 = e2P * b.ux;
    const T h10 = b.twoP + b.q5;                // 4P + j^2/rho
    const T q10 = h10 * b.ux;
    const T q12 = (b.twoP + b.q6) * b.ux;
    D.d8 = relax(k, 3, m8 - q8);
    D.d10 = relax(k, 5, m10 - q10);
    D.d12 = relax(k, 7, m12 - q12);
}
// block Dy: m9, m11, -m13
template <class T>
__device__ __forceinline__ void relax_Dy(const EqBase<T>& b, T e, T m9, T m11, T n13, const Coef<T>& k,
                                         Deltas<T>& D) {
    const T e2P = e + b.twoP;
    const T q9 = e2P * b.uy;
    const T h10 = b.twoP + b.q5;
    const T q11 = h10 * b.uy;
    const T nq13 = (b.twoP - b.q6) * b.uy;      // -q13
    D.d9 = relax(k, 4, m9 - q9);
    D.d11 = relax(k, 6, m11 - q11);
    D.nd13 = relax(k, 8, n13 - nq13);
}
// block Q: m6, m16, m7, m15 (jx the x momentum m2)
template <class T>
__device__ __forceinline__ void relax_Q(const EqBase<T>& b, T jx, T m6, T m16, T m7, T m15, const Coef<T>& k,
                                        Deltas<T>& D) {
    const T q7 = jx * b.uy;
    const T g15 = k.c15 * b.P + b.j2r;
    const T q15 = g15 * (b.ux * b.uy);
    const T q16 = g15 * (b.ux * b.ux - b.uy * b.uy);
    D.d6 = relax(k, 1, m6 - b.q6);
    D.d7 = relax(k, 2, m7 - q7);
    D.d15 = relax(k, 10, m15 - q15);
    D.d16 = relax(k, 11, m16 - q16);
}

// Phase 4, per group g: the collision increment of its four velocities
// (inverse blocks, already scaled by the inverse butterflies' 1/4 or 1/2
// and by -1) and the Lax-Wendroff advection, from the centre values fg and
// the neighbours read through F(plane, pos); writes og.
//
// The FP32 form accumulates the Lax-Wendroff terms as multiply-adds of
// neighbour differences onto the collision increment, so a uniform state is
// left exactly unchanged by the advection.
//
// XT: the unsplit two-dimensional Lax-Wendroff operator, which adds to each
// diagonal velocity the mixed term (c_x c_y / 4)(f(x+1,y+1) - f(x+1,y-1)
// - f(x-1,y+1) + f(x-1,y-1)) of the second-order Taylor expansion in time
// (c_x c_y > 0 for (+,+) and (-,-), < 0 for (-,+) and (+,-)).
template <class T, bool XT, class Fetch>
__device__ __forceinline__ void group_update(int g, const Fetch& F, const Coef<T>& k, const Deltas<T>& D,
                                             const T fg[4], T og[4]) {
    constexpr bool kFold = sizeof(T) == 8;
    T cS, cX, cY;
    if constexpr (kFold) {
        cS = k.kSs[g][0] * D.d5 + k.kSs[g][1] * D.d14;
        cX = k.kDx[g][0] * D.d8 + k.kDx[g][1] * D.d10 + k.kDx[g][2] * D.d12;
        cY = k.kDy[g][0] * D.d9 + k.kDy[g][1] * D.d11 + k.kDy[g][2] * D.nd13;
    } else {
        cS = k.kS[g][0] * D.d5 + k.kS[g][1] * D.d14;
        cX = k.kD[g][0] * D.d8 + k.kD[g][1] * D.d10 + k.kD[g][2] * D.d12;
        cY = k.kD[g][0] * D.d9 + k.kD[g][1] * D.d11 + k.kD[g][2] * D.nd13;
    }
    const T p = k.lwp[g], qq = k.lwq[g];
    const int i0 = 4 * g;  // plane of the group's first velocity
    if constexpr (kFold) {
      if (g < 2) {
        // FP64: out = a0 f + p f_up + q f_down + collision, one
        // multiply-add per neighbour (+x: p on x-1, q on x+1; -x mirrored;
        // +y / -y likewise along y)
        const T cQ = k.kQs[g][0] * D.d6 + k.kQs[g][1] * D.d16;
        const T sp = cS + cQ, sm = cS - cQ;
        const T a0 = k.lw0[g];
        og[0] = a0 * fg[0] + (p * F(i0 + 0, XM) + (qq * F(i0 + 0, XP) + (sp + cX)));
        og[2] = a0 * fg[2] + (p * F(i0 + 2, XP) + (qq * F(i0 + 2, XM) + (sp - cX)));
        og[1] = a0 * fg[1] + (p * F(i0 + 1, YM) + (qq * F(i0 + 1, YP) + (sm + cY)));
        og[3] = a0 * fg[3] + (p * F(i0 + 3, YP) + (qq * F(i0 + 3, YM) + (sm - cY)));
      } else {
        // FP64 diagonal groups: a0 = 1 - 2 c^2; the mixed term of the
        // unsplit operator enters as four more multiply-adds
        const T cXY = k.kXs[g - 2][0] * D.d7 + k.kXs[g - 2][1] * D.d15;
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
            og[0] = a0 * fg[0] + (p * (F(i0 + 0, XM) + F(i0 + 0, YM)) +
                                             (qq * (F(i0 + 0, XP) + F(i0 + 0, YP)) + c0));
        }
        {   // (-,+): p on x+1, y-1; q on x-1, y+1
            const T c1 = mixed(i0 + 1, -w, t2 - s2);
            og[1] = a0 * fg[1] + (p * (F(i0 + 1, XP) + F(i0 + 1, YM)) +
                                             (qq * (F(i0 + 1, XM) + F(i0 + 1, YP)) + c1));
        }
        {   // (-,-): p on x+1, y+1; q on x-1, y-1
            const T c2 = mixed(i0 + 2, w, t1 - s1);
            og[2] = a0 * fg[2] + (p * (F(i0 + 2, XP) + F(i0 + 2, YP)) +
                                             (qq * (F(i0 + 2, XM) + F(i0 + 2, YM)) + c2));
        }
        {   // (+,-): p on x-1, y+1; q on x+1, y-1
            const T c3 = mixed(i0 + 3, -w, t2 + s2);
            og[3] = a0 * fg[3] + (p * (F(i0 + 3, XM) + F(i0 + 3, YP)) +
                                             (qq * (F(i0 + 3, XP) + F(i0 + 3, YM)) + c3));
        }
      }
    } else {
      if (g < 2) {
        const T cQ = k.kQ[g][0] * D.d6 + k.kQ[g][1] * D.d16;
        const T sp = cS + cQ, sm = cS - cQ;
        // +x: p on x-1, q on x+1; -x mirrored; +y / -y likewise along y
        {
            const T fc = fg[0];
            T t = qq * (F(i0 + 0, XP) - fc) + (sp + cX);
            og[0] = fc + (p * (F(i0 + 0, XM) - fc) + t);
        }
        {
            const T fc = fg[2];
            T t = p * (F(i0 + 2, XP) - fc) + (sp - cX);
            og[2] = fc + (qq * (F(i0 + 2, XM) - fc) + t);
        }
        {
            const T fc = fg[1];
            T t = qq * (F(i0 + 1, YP) - fc) + (sm + cY);
            og[1] = fc + (p * (F(i0 + 1, YM) - fc) + t);
        }
        {
            const T fc = fg[3];
            T t = p * (F(i0 + 3, YP) - fc) + (sm - cY);
            og[3] = fc + (qq * (F(i0 + 3, YM) - fc) + t);
        }
    } else {
        const T cXY = k.kX[g - 2][0] * D.d7 + k.kX[g - 2][1] * D.d15;
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
            const T fc = fg[0];
            const T a = (F(i0 + 0, XM) + F(i0 + 0, YM)) - (fc + fc);
            const T b = (F(i0 + 0, XP) + F(i0 + 0, YP)) - (fc + fc);
            og[0] = fc + (p * a + (qq * b + with_mixed((t1 + s1), e0)));
        }
        {   // (-,+): q on x-1, p on x+1; p on y-1, q on y+1
            const T fc = fg[1];
            const T a = (F(i0 + 1, XP) + F(i0 + 1, YM)) - (fc + fc);
            const T b = (F(i0 + 1, XM) + F(i0 + 1, YP)) - (fc + fc);
            og[1] = fc + (p * a + (qq * b + with_mixed((t2 - s2), e1)));
        }
        {   // (-,-): q on x-1, y-1; p on x+1, y+1
            const T fc = fg[2];
            const T a = (F(i0 + 2, XP) + F(i0 + 2, YP)) - (fc + fc);
            const T b = (F(i0 + 2, XM) + F(i0 + 2, YM)) - (fc + fc);
            og[2] = fc + (p * a + (qq * b + with_mixed((t1 - s1), e2)));
        }
        {   // (+,-): p on x-1, q on x+1; q on y-1, p on y+1
            const T fc = fg[3];
            const T a = (F(i0 + 3, XM) + F(i0 + 3, YP)) - (fc + fc);
            const T b = (F(i0 + 3, XP) + F(i0 + 3, YM)) - (fc + fc);
            og[3] = fc + (p * a + (qq * b + with_mixed((t2 + s2), e3)));
        }
      }
    }
}

// One cell of one time step (Eq. 3, forward Euler + Lax-Wendroff): reads
// the stencil through F(i, pos), writes f^{n+1} to out and returns the
// cell's input rho and P for the health check.
template <class T, bool XT = false, class Fetch>
__device__ __forceinline__ void cell_update(const Fetch& F, const Coef<T>& k, T out[NV],
                                            T& rho_in, T& P_in) {
    T f[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) f[i] = F(i, C);
    T S[4], Dx[4], Dy[4], QX[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const GroupSums<T> gs = group_sums<T>(g, f + 4 * g);
        S[g] = gs.S;
        QX[g] = gs.QX;
        Dx[g] = gs.Dx;
        Dy[g] = gs.Dy;
    }
    T mS[4], mX[4], mY[4], mQ[4];
    moments_S<T>(S, mS);
    moments_D<T>(Dx, mX);
    moments_D<T>(Dy, mY);
    moments_Q<T>(QX, mQ);
    // rho = m1, jx = m2, jy = m3, e = m4
    const EqBase<T> b = eq_base<T>(mS[0], mX[0], mY[0], mS[2], k);
    rho_in = mS[0];
    P_in = b.P;
    Deltas<T> D;
    relax_S<T>(b, mS[1], mS[3], k, D);
    relax_Dx<T>(b, mS[2], mX[3], mX[2], mX[1], k, D);
    relax_Dy<T>(b, mS[2], mY[3], mY[2], mY[1], k, D);
    relax_Q<T>(b, mX[0], mQ[0], mQ[1], mQ[2], mQ[3], k, D);
#pragma unroll
    for (int g = 0; g < 4; ++g) group_update<T, XT>(g, F, k, D, f + 4 * g, out + 4 * g);
}

#endif  // __CUDACC__

}  // namespace mrt
