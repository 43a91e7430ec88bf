// api.cu - the C ABI declared in include/mrtfdlb.h: grid creation from
// macroscopic fields (f = M^-1 fhat^eq, Sect. (b)), the time-step driver,
// macroscopic readout, conserved totals and raw state access.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/mrtfdlb.h"
#include "host_state.h"

using namespace mrt;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static mrt_status fail(mrt_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

void mrt::set_last_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

#define CUDA_TRY(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? MRT_ENOMEM : MRT_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                     \
    } while (0)

// ---------------------------------------------------------------------------
// Model blocks (host, FP64)
// ---------------------------------------------------------------------------
namespace {

// Gauss-Jordan with partial pivoting on an n x n matrix (n <= 4).
bool invert_small(int n, const double* A, double* Ainv) {
    double a[4][8];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) a[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(a[r][c]) > std::fabs(a[p][c])) p = r;
        if (a[p][c] == 0.0) return false;
        if (p != c)
            for (int k = 0; k < 2 * n; ++k) std::swap(a[p][k], a[c][k]);
        const double d = a[c][c];
        for (int k = 0; k < 2 * n; ++k) a[c][k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double m = a[r][c];
            for (int k = 0; k < 2 * n; ++k) a[r][k] -= m * a[c][k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r][n + c];
    return true;
}

// The five blocks of M in the group-combination basis (see model.cuh).
bool build_blocks(double A[16], double B[16], double C1[4], double C2[4]) {
    for (int g = 0; g < 4; ++g) {
        A[0 * 4 + g] = 1.0;
        A[1 * 4 + g] = kW(g);
        A[2 * 4 + g] = kV(g);
        A[3 * 4 + g] = kV(g) * kW(g);
        B[0 * 4 + g] = kU(g);
        B[1 * 4 + g] = kU(g) * kW(g);
        B[2 * 4 + g] = kU(g) * kV(g);
        B[3 * 4 + g] = g < 2 ? kU(g) * kV(g) : 0.0;
    }
    for (int g = 0; g < 2; ++g) {
        C1[0 * 2 + g] = kV(g);
        C1[1 * 2 + g] = kV(g) * kW(g);
        C2[0 * 2 + g] = 0.5 * kV(2 + g);
        C2[1 * 2 + g] = 0.5 * kV(2 + g) * kW(2 + g);
    }
    return true;
}

}  // namespace

namespace mrt {

int mrt_init_coef_build(double b, InitCoef* o) {
    double A[16], B[16], C1[4], C2[4];
    build_blocks(A, B, C1, C2);
    if (!invert_small(4, A, &o->Ainv[0][0]) || !invert_small(4, B, &o->Binv[0][0]) ||
        !invert_small(2, C1, &o->C1inv[0][0]) || !invert_small(2, C2, &o->C2inv[0][0]))
        return -1;
    o->b = b;
    return 0;
}

int mrt_model_build(double dx, double dt, double b, const double s[16], Coef<double>* k) {
    InitCoef ic;
    if (mrt_init_coef_build(b, &ic) != 0) return -1;
    for (int g = 0; g < 4; ++g) {
        const double scS = -0.25;
        const double scD = g < 2 ? -0.5 : -0.25;
        k->kS[g][0] = scS * ic.Ainv[g][2];  // m5
        k->kS[g][1] = scS * ic.Ainv[g][3];  // m14
        k->kD[g][0] = scD * ic.Binv[g][1];  // m8 / m9
        k->kD[g][1] = scD * ic.Binv[g][2];  // m10 / m11
        k->kD[g][2] = scD * ic.Binv[g][3];  // m12 / -m13
        const double c = kU(g) * dt / dx;
        k->lwp[g] = 0.5 * (c * c + c);
        k->lwq[g] = 0.5 * (c * c - c);
        if (g >= 2) k->kxy[g - 2] = 0.25 * c * c;   // |c_x c_y| / 4 on a diagonal
    }
    for (int g = 0; g < 2; ++g)
        for (int j = 0; j < 2; ++j) {
            k->kQ[g][j] = -0.25 * ic.C1inv[g][j];
            k->kX[g][j] = -0.25 * ic.C2inv[g][j];
        }
    for (int kk = 0; kk < 12; ++kk) k->sig[kk] = s[4 + kk] * dt;
    // FP64 kernels: sigma_k folded into the inverse-block constants, and the
    // Lax-Wendroff centre weights (p + q = c^2 per axis)
    const double* sg = k->sig;  // sigma_5 .. sigma_16 at 0 .. 11
    for (int g = 0; g < 4; ++g) {
        k->kSs[g][0] = k->kS[g][0] * sg[0];
        k->kSs[g][1] = k->kS[g][1] * sg[9];
        for (int j = 0; j < 3; ++j) {
            k->kDx[g][j] = k->kD[g][j] * sg[3 + 2 * j];   // sigma_8, sigma_10, sigma_12
            k->kDy[g][j] = k->kD[g][j] * sg[4 + 2 * j];   // sigma_9, sigma_11, sigma_13
        }
        const double c = kU(g) * dt / dx;
        k->lw0[g] = g < 2 ? 1.0 - c * c : 1.0 - 2.0 * c * c;
    }
    for (int g = 0; g < 2; ++g) {
        k->kQs[g][0] = k->kQ[g][0] * sg[1];    // sigma_6
        k->kQs[g][1] = k->kQ[g][1] * sg[11];   // sigma_16
        k->kXs[g][0] = k->kX[g][0] * sg[2];    // sigma_7
        k->kXs[g][1] = k->kX[g][1] * sg[10];   // sigma_15
    }
    k->inv_b = 1.0 / b;
    k->c14a = 2.0 * (b + 2.0);
    k->c14b = 6.0 + b;
    k->c15 = b + 4.0;
    return 0;
}

}  // namespace mrt

// ---------------------------------------------------------------------------
// Small kernels: initialisation, ghosts, macroscopic fields, reductions
// ---------------------------------------------------------------------------
namespace {

// The validity test of an input cell on bit patterns, in integer
// instructions: rho and T positive and finite (a positive finite double's
// pattern lies in [1, 0x7fefffffffffffff]), u and v finite.
__device__ __forceinline__ bool init_valid(double r, double u, double v, double t) {
    const unsigned long long kInf = 0x7ff0000000000000ull;
    const unsigned long long br = (unsigned long long)__double_as_longlong(r) - 1ull;
    const unsigned long long bt = (unsigned long long)__double_as_longlong(t) - 1ull;
    return br < kInf - 1ull && bt < kInf - 1ull && ((unsigned long long)__double_as_longlong(u) & kInf) != kInf &&
           ((unsigned long long)__double_as_longlong(v) & kInf) != kInf;
}

// Double-float arithmetic for the initialisation of FP32 grids: a value is
// the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2), about 44
// significant bits, kept on the FP32 pipe.  Sums use Knuth's TwoSum and the
// "sloppy" double-word addition, products the FMA-based exact product and
// the double-word product (Joldes, Muller and Popescu, ACM TOMS 44(2),
// 2017): each operation errs by about 2^-44 of its operands' magnitudes, so
// rounding a result to FP32 gives the FP32 rounding of the FP64 formula's
// value except within about 2^-44 of a rounding boundary.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ DF operator+(DF x, DF y) {
    const float s = x.hi + y.hi, bb = s - x.hi;
    float e = (x.hi - (s - bb)) + (y.hi - bb);   // TwoSum error of the high parts
    e += x.lo + y.lo;
    return df_fast_two_sum(s, e);
}
__device__ __forceinline__ DF operator-(DF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ DF operator-(DF x, DF y) { return x + (-y); }
__device__ __forceinline__ DF operator*(DF x, DF y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);                // exact error of the high product
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF operator*(int k, DF x) { return {(float)k * x.hi, (float)k * x.lo}; }  // k = 2, 4: exact

template <class A>
__device__ __forceinline__ A init_in(double x);
template <>
__device__ __forceinline__ double init_in<double>(double x) { return x; }
template <>
__device__ __forceinline__ DF init_in<DF>(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}
__device__ __forceinline__ double init_out(double x) { return x; }
__device__ __forceinline__ float init_out(DF x) { return x.hi + x.lo; }

// f = M^-1 fhat^eq(rho, u, T) per cell in arithmetic A (FP64 grids: double;
// FP32 grids: double-float), stored as T.  Blocks take runs of one row, so
// no cell index is divided.  The inverse blocks' 1/4 and 1/2 factors are
// folded into the constants (InitK), which scales every product and sum by
// a power of two and so changes no rounding.
template <class A>
struct InitK {
    A Ainv[4][4];    // 1/4 Ainv
    A Bax[4][4];     // 1/2 Binv for the axis groups, 1/4 for the diagonal ones
    A C1inv[2][2];   // 1/4 C1inv
    A C2inv[2][2];   // 1/4 C2inv
    A b, c13a, c13b, c14;   // b, 2 (b + 2), 6 + b, b + 4
};
static double init_const(double x, double*) { return x; }
static DF init_const(double x, DF*) {
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}
template <class A>
static InitK<A> init_k(const InitCoef& ic) {
    InitK<A> o;
    A* tag = nullptr;
    for (int g = 0; g < 4; ++g)
        for (int k = 0; k < 4; ++k) {
            o.Ainv[g][k] = init_const(0.25 * ic.Ainv[g][k], tag);
            o.Bax[g][k] = init_const((g < 2 ? 0.5 : 0.25) * ic.Binv[g][k], tag);
        }
    for (int g = 0; g < 2; ++g)
        for (int j = 0; j < 2; ++j) {
            o.C1inv[g][j] = init_const(0.25 * ic.C1inv[g][j], tag);
            o.C2inv[g][j] = init_const(0.25 * ic.C2inv[g][j], tag);
        }
    o.b = init_const(ic.b, tag);
    o.c13a = init_const(2 * (ic.b + 2), tag);
    o.c13b = init_const(6 + ic.b, tag);
    o.c14 = init_const(ic.b + 4, tag);
    return o;
}

template <class T, class A>
__global__ void init_kernel(Layout L, InitK<A> K, const double* __restrict__ rho,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            const double* __restrict__ Tf, T* __restrict__ f, unsigned* flag, int y0, int y1) {
    for (int y = y0 + blockIdx.y; y < y1; y += gridDim.y) {
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < L.nx; x += gridDim.x * blockDim.x) {
            const long c = (long)y * L.nx + x;
            const double rd = rho[c], ud = ux[c], vd = uy[c], td = Tf[c];
            if (!init_valid(rd, ud, vd, td)) atomicOr(flag, FLAG_UNSTABLE);
            const A r = init_in<A>(rd), u = init_in<A>(ud), v = init_in<A>(vd), t = init_in<A>(td);
            const A jx = r * u, jy = r * v;
            const A P = r * t;
            const A j2r = jx * u + jy * v;
            const A e = K.b * P + j2r;
            // Appendix equilibria (R = 1)
            A m[16];
            m[0] = r; m[1] = jx; m[2] = jy; m[3] = e;
            m[4] = 2 * P + j2r;
            m[5] = jx * u - jy * v;
            m[6] = jx * v;
            m[7] = (e + 2 * P) * u;
            m[8] = (e + 2 * P) * v;
            m[9] = (4 * P + j2r) * u;
            m[10] = (4 * P + j2r) * v;
            m[11] = (2 * P + m[5]) * u;
            m[12] = (m[5] - 2 * P) * v;
            const A u2 = u * u + v * v;
            m[13] = K.c13a * P * t + K.c13b * t * j2r + j2r * u2;
            m[14] = (K.c14 * P + j2r) * u * v;
            m[15] = (K.c14 * P + j2r) * (u * u - v * v);
            // block inverses (scaled: S = Ainv a / 4, Dx = Binv ex / 2 or / 4, ...)
            const A a1[4] = {m[0], m[3], m[4], m[13]};
            const A ex[4] = {m[1], m[7], m[9], m[11]};
            const A ey[4] = {m[2], m[8], m[10], -m[12]};
            const A b1[2] = {m[5], m[15]};
            const A b2[2] = {m[6], m[14]};
            A out[16];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                A S = K.Ainv[g][0] * a1[0], Dx = K.Bax[g][0] * ex[0], Dy = K.Bax[g][0] * ey[0];
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    S = S + K.Ainv[g][k] * a1[k];
                    Dx = Dx + K.Bax[g][k] * ex[k];
                    Dy = Dy + K.Bax[g][k] * ey[k];
                }
                if (g < 2) {
                    const A Q = K.C1inv[g][0] * b1[0] + K.C1inv[g][1] * b1[1];
                    out[4 * g + 0] = S + Dx + Q;
                    out[4 * g + 2] = S - Dx + Q;
                    out[4 * g + 1] = S + Dy - Q;
                    out[4 * g + 3] = S - Dy - Q;
                } else {
                    const A X = K.C2inv[g - 2][0] * b2[0] + K.C2inv[g - 2][1] * b2[1];
                    out[4 * g + 0] = S + Dx + Dy + X;
                    out[4 * g + 1] = S - Dx + Dy - X;
                    out[4 * g + 2] = S - Dx - Dy + X;
                    out[4 * g + 3] = S + Dx - Dy - X;
                }
            }
            const long o = (long)(y + 1) * L.pitch + L.G + x;
#pragma unroll
            for (int i = 0; i < 16; ++i) f[i * L.plane + o] = (T)init_out(out[i]);
        }
    }
}

// Ghost columns, then ghost rows, of every plane.  Per side: GH_KEEP leaves
// the ghost alone, GH_COPY copies the adjacent domain cell (a fixed
// equilibrium at creation), GH_WRAP copies the opposite edge (periodic),
// GH_MIRROR copies the adjacent cell with its velocities mirrored across the
// wall (reflecting).
enum { GH_KEEP = 0, GH_COPY = 1, GH_WRAP = 2, GH_MIRROR = 3 };

template <class T>
__global__ void ghost_cols_kernel(Layout L, int lo, int hi, T* f) {
    const long n = 16L * L.ny;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / L.ny), y = (int)(t % L.ny);
        const long r = (long)(y + 1) * L.pitch;
        T* row = f + i * L.plane + r;
        if (lo == GH_COPY) row[L.G - 1] = row[L.G];
        if (lo == GH_WRAP) row[L.G - 1] = row[L.G + L.nx - 1];
        if (lo == GH_MIRROR) row[L.G - 1] = f[mirror_plane(i, 0) * L.plane + r + L.G];
        if (hi == GH_COPY) row[L.G + L.nx] = row[L.G + L.nx - 1];
        if (hi == GH_WRAP) row[L.G + L.nx] = row[L.G];
    }
}

// The ghost rows span the ghost columns too (x = -1 and nx), after those
// were set: a corner then holds the ghost-row rule applied to the ghost
// column, which is what the unsplit operator reads there.
template <class T>
__global__ void ghost_rows_kernel(Layout L, int lo, int hi, T* f) {
    const long w = L.nx + 2;
    const long n = 16L * w;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / w), x = (int)(t % w) - 1;
        T* p = f + i * L.plane + L.G + x;
        if (lo == GH_COPY) p[0] = p[L.pitch];
        if (lo == GH_WRAP) p[0] = p[(long)L.ny * L.pitch];
        if (lo == GH_MIRROR) p[0] = f[mirror_plane(i, 1) * L.plane + L.pitch + L.G + x];
        if (hi == GH_COPY) p[(long)(L.ny + 1) * L.pitch] = p[(long)L.ny * L.pitch];
        if (hi == GH_WRAP) p[(long)(L.ny + 1) * L.pitch] = p[L.pitch];
    }
}

// The border of a padded buffer, everything but the interior cells: rows 0
// and ny + 1 whole, and in rows 1 .. ny the columns before the interior
// (padding and the left ghost) and after it (the right ghost and padding).
// border_kernel zeroes it in dst (src == nullptr) or copies it from src.
template <class T>
__global__ void border_kernel(Layout L, const T* __restrict__ src, T* __restrict__ dst) {
    const long side = L.pitch - L.nx;                    // border columns of an interior row
    const long per_plane = 2L * L.pitch + (long)L.ny * side;
    const long n = 16L * per_plane;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const long i = t / per_plane, k = t % per_plane;
        long o;
        if (k < L.pitch) {
            o = k;                                       // row 0
        } else if (k < 2L * L.pitch) {
            o = (long)(L.ny + 1) * L.pitch + (k - L.pitch);   // row ny + 1
        } else {
            const long r = (k - 2L * L.pitch) / side, c = (k - 2L * L.pitch) % side;
            o = (r + 1) * L.pitch + (c < L.G ? c : c + L.nx);
        }
        o += i * L.plane;
        dst[o] = src ? src[o] : (T)0;
    }
}

template <class T>
__device__ __forceinline__ void cons_moments(const T* f, const Layout& L, long o, double q[4]) {
    double v[16];
    for (int i = 0; i < 16; ++i) v[i] = (double)f[i * L.plane + o];
    double S[4], Dx[4], Dy[4];
    for (int g = 0; g < 4; ++g) {
        const double* a = v + 4 * g;
        S[g] = (a[0] + a[2]) + (a[1] + a[3]);
        const double d02 = a[0] - a[2], d13 = a[1] - a[3];
        Dx[g] = g < 2 ? d02 : d02 - d13;
        Dy[g] = g < 2 ? d13 : d02 + d13;
    }
    q[0] = (S[0] + S[1]) + (S[2] + S[3]);
    q[1] = kU(0) * Dx[0] + kU(1) * Dx[1] + kU(2) * Dx[2] + kU(3) * Dx[3];
    q[2] = kU(0) * Dy[0] + kU(1) * Dy[1] + kU(2) * Dy[2] + kU(3) * Dy[3];
    q[3] = kW(0) * S[0] + kW(1) * S[1] + kW(2) * S[2] + kW(3) * S[3];
}

// The conserved moments (rho, jx, jy, e) of an FP32 cell in double-float
// arithmetic: each butterfly pair sum is exact (TwoSum of two floats), the
// weighted block sums carry about 44 bits.
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__host__ __device__ constexpr DF df_c(double x) {   // a constant, split at compile time
    return {(float)x, (float)(x - (double)(float)x)};
}
__device__ __forceinline__ void cons_moments_df(const float* f, const Layout& L, long o, DF q[4]) {
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = f[i * L.plane + o];
    DF S[4], Dx[4], Dy[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float* a = v + 4 * g;
        S[g] = df_two_sum(a[0], a[2]) + df_two_sum(a[1], a[3]);
        const DF d02 = df_two_sum(a[0], -a[2]), d13 = df_two_sum(a[1], -a[3]);
        Dx[g] = g < 2 ? d02 : d02 - d13;
        Dy[g] = g < 2 ? d13 : d02 + d13;
    }
    constexpr DF u1 = df_c(kU(1)), u2 = df_c(kU(2)), u3 = df_c(kU(3));
    constexpr DF w0 = df_c(kW(0)), w1 = df_c(kW(1)), w2 = df_c(kW(2)), w3 = df_c(kW(3));
    q[0] = (S[0] + S[1]) + (S[2] + S[3]);
    q[1] = Dx[0] + u1 * Dx[1] + u2 * Dx[2] + u3 * Dx[3];   // kU(0) = 1
    q[2] = Dy[0] + u1 * Dy[1] + u2 * Dy[2] + u3 * Dy[3];
    q[3] = w0 * S[0] + w1 * S[1] + w2 * S[2] + w3 * S[3];
}
__device__ __forceinline__ double df_out(DF x) { return (double)x.hi + (double)x.lo; }

// rho, u, T per cell of rows [y0, y1); u = j/rho, T = (e - j^2/rho)/(b rho)
// with one reciprocal of rho per cell.  FP64 grids in FP64; FP32 grids in
// double-float arithmetic (1/rho by one Newton step from the FP32
// quotient), which leaves only the final conversions to FP64 on the FP64
// pipe that bounded this kernel.
template <class T>
__global__ void macro_kernel(Layout L, double inv_b, const T* __restrict__ f, double* rho, double* ux,
                             double* uy, double* Tf, int y0, int y1) {
    DF ib = {0.f, 0.f};
    if constexpr (sizeof(T) == 4) {
        const float h = __double2float_rn(inv_b);
        ib = {h, __double2float_rn(inv_b - (double)h)};
    }
    for (int y = y0 + blockIdx.y; y < y1; y += gridDim.y) {
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < L.nx; x += gridDim.x * blockDim.x) {
            const long c = (long)y * L.nx + x;
            const long o = (long)(y + 1) * L.pitch + L.G + x;
            if constexpr (sizeof(T) == 8) {
                double q[4];
                cons_moments<T>(f, L, o, q);
                const double ri = 1.0 / q[0];
                const double u = q[1] * ri, v = q[2] * ri;
                if (rho) rho[c] = q[0];
                if (ux) ux[c] = u;
                if (uy) uy[c] = v;
                if (Tf) Tf[c] = (q[3] - (q[1] * u + q[2] * v)) * (ri * inv_b);
            } else {
                DF q[4];
                cons_moments_df(f, L, o, q);
                const DF r0 = {1.0f / q[0].hi, 0.f};
                const DF ri = r0 + r0 * (DF{1.f, 0.f} - q[0] * r0);
                const DF u = q[1] * ri, v = q[2] * ri;
                if (rho) rho[c] = df_out(q[0]);
                if (ux) ux[c] = df_out(u);
                if (uy) uy[c] = df_out(v);
                if (Tf) Tf[c] = df_out((q[3] - (q[1] * u + q[2] * v)) * (ri * ib));
            }
        }
    }
}

// Launch shape of the row-range kernels: blocks of 256 along a row, blocks
// in y over the rows.
static dim3 rows_grid(const Layout& L, int rows) {
    return dim3((unsigned)std::min<long>((L.nx + 255) / 256, 64), (unsigned)std::max(1, std::min(rows, 4096)));
}

// Row chunks of a host upload or readout of the four fields: about 64 MB
// of fields each, at most 8.
static int field_chunks(const Layout& L) {
    const long bytes = 32L * L.nx * L.ny;
    long k = (bytes + (64L << 20) - 1) / (64L << 20);
    if (k > 8) k = 8;
    if (k > L.ny) k = L.ny;
    return (int)std::max(1L, k);
}

constexpr int RED_THREADS = 256;

// FP64 block partials of (rho, jx, jy, e) over the whole state.
template <class T>
__global__ void __launch_bounds__(RED_THREADS) totals_partial_kernel(Layout L, const T* __restrict__ f,
                                                                     double* partials) {
    __shared__ double red[RED_THREADS / 32][4];
    const long n = (long)L.nx * L.ny;
    double acc[4] = {0, 0, 0, 0};
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
        const int x = (int)(c % L.nx), y = (int)(c / L.nx);
        double q[4];
        cons_moments<T>(f, L, (long)(y + 1) * L.pitch + L.G + x, q);
        for (int k = 0; k < 4; ++k) acc[k] += q[k];
    }
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 4; ++k) red[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) {
            double s = 0;
            for (int w = 0; w < RED_THREADS / 32; ++w) s += red[w][k];
            partials[4 * blockIdx.x + k] = s;
        }
}

// Fixed-order sum of nparts block partials, times dx*dy, into out[0..3];
// out[4] takes the flag word, so one copy brings back totals and health.
// Two passes spread the FP64 additions over many SMs (one SM of this part
// retires only two FP64 lanes per clock): block b of the first pass sums
// partials [b*chunk, (b+1)*chunk) - thread t those at t, t+FINAL_THREADS,
// ... - and a fixed tree; the second pass sums the block results the same
// way.  Blocks of 128 threads (32 registers each, 4 KB of shared memory)
// fit beside a step kernel's resident CTAs, so the side-stream reduction of
// one step runs while the next step does.
constexpr int FINAL_THREADS = 128;
constexpr int FINAL_PER_BLOCK = 4 * FINAL_THREADS;  // partials per first-pass block
constexpr int FINAL_MAX_BLOCKS = 1024;

__device__ __forceinline__ void tree_sum4(double acc[4], double (*red)[4], double* dst, double scale) {
    for (int k = 0; k < 4; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = FINAL_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 4; ++k) red[threadIdx.x][k] += red[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) dst[k] = red[0][k] * scale;
}

__global__ void __launch_bounds__(FINAL_THREADS, 16) totals_pass_kernel(const double* partials, int nparts,
                                                                        int chunk, double* block_sums) {
    __shared__ double red[FINAL_THREADS][4];
    double acc[4] = {0, 0, 0, 0};
    const int p0 = blockIdx.x * chunk, p1 = min(nparts, p0 + chunk);
    const double2* P = reinterpret_cast<const double2*>(partials);
#pragma unroll 4
    for (int p = p0 + threadIdx.x; p < p1; p += FINAL_THREADS) {
        const double2 a = P[2 * p], b = P[2 * p + 1];
        acc[0] += a.x;
        acc[1] += a.y;
        acc[2] += b.x;
        acc[3] += b.y;
    }
    tree_sum4(acc, red, block_sums + 4 * blockIdx.x, 1.0);
}

__global__ void __launch_bounds__(FINAL_THREADS, 16) totals_final_kernel(const double* block_sums, int nblocks,
                                                                         double scale, const unsigned* flag,
                                                                         const unsigned long long* stamp,
                                                                         double* out) {
    __shared__ double red[FINAL_THREADS][4];
    double acc[4] = {0, 0, 0, 0};
    for (int p = threadIdx.x; p < nblocks; p += FINAL_THREADS)
        for (int k = 0; k < 4; ++k) acc[k] += block_sums[4 * p + k];
    tree_sum4(acc, red, out, scale);
    if (threadIdx.x == 0) {
        out[4] = (double)*flag;
        out[5] = (double)*stamp;
    }
}

// Sequence stamp of the partials a step is about to write: the grid's
// counter, advanced on the grid's stream, so stamps follow step order.
__global__ void totals_stamp_kernel(unsigned long long* seq, int slot) {
    seq[1 + slot] = ++seq[0];
}

// Copy the totals slot with the newer stamp (the side stream's latest or
// the captured graph's) into the pick slot a reader copies out.
__global__ void totals_pick_kernel(double* totals, int side_slot, int cap_slot, int pick_slot) {
    const double* a = totals + mrt_grid::kTotalsSlot * side_slot;
    const double* c = totals + mrt_grid::kTotalsSlot * cap_slot;
    const double* src = c[5] > a[5] ? c : a;
    double* dst = totals + mrt_grid::kTotalsSlot * pick_slot;
    for (int k = 0; k < mrt_grid::kTotalsSlot; ++k) dst[k] = src[k];
}

// Both passes of one reduction: the partials of slot b (0, 1: the side
// stream's double buffer; kCapSlot: a captured graph's) into totals slot b.
// The side-stream slots share block_sums, used by one reduction at a time
// in the side stream's order; the captured slot has its own.
static cudaError_t reduce_totals_on(mrt_grid* g, int b, int nparts, cudaStream_t st) {
    int chunk = FINAL_PER_BLOCK;
    int blocks = (nparts + chunk - 1) / chunk;
    if (blocks > FINAL_MAX_BLOCKS) {
        blocks = FINAL_MAX_BLOCKS;
        chunk = (nparts + blocks - 1) / blocks;
    }
    if (blocks < 1) blocks = 1;
    const bool cap = b == mrt_grid::kCapSlot;
    const double* parts = cap ? g->cap_partials : g->partials + (size_t)b * 4 * g->max_parts;
    double* sums = cap ? g->cap_block_sums : g->block_sums;
    totals_pass_kernel<<<blocks, FINAL_THREADS, 0, st>>>(parts, nparts, chunk, sums);
    totals_final_kernel<<<1, FINAL_THREADS, 0, st>>>(sums, blocks, g->p.dx * g->p.dx, g->flag, g->seq + 1 + b,
                                                     g->totals_dev + mrt_grid::kTotalsSlot * b);
    return cudaGetLastError();
}

// The side stream waits for everything enqueued on the grid's stream so far
// (a read of the totals comes after the steps that produced them, also when
// those ran inside a graph the caller captured and launched there).
static cudaError_t tail_to_side(mrt_grid* g) {
    cudaError_t e = cudaEventRecord(g->ev_tail, g->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(g->tstream, g->ev_tail, 0);
}

// Partials buffer for the next totals reduction.  Outside a capture: the
// side stream's next buffer, after the grid's stream has waited until the
// side stream finished reading it.  Inside a capture: the captured slot's
// own buffer, which only the grid's stream touches.  Once the grid has been
// captured, a stamp of the step order precedes the partials.
static cudaError_t begin_totals(mrt_grid* g, double** partials, bool capturing) {
    int slot;
    if (capturing) {
        g->cap_used = true;
        slot = mrt_grid::kCapSlot;
        *partials = g->cap_partials;
    } else {
        slot = g->tnext;
        if (g->red_pending[slot]) {
            cudaError_t e = cudaStreamWaitEvent(g->stream, g->ev_red[slot], 0);
            if (e != cudaSuccess) return e;
        }
        *partials = g->partials + (size_t)slot * 4 * g->max_parts;
    }
    if (g->cap_used) {
        totals_stamp_kernel<<<1, 1, 0, g->stream>>>(g->seq, slot);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

// After the partials of the next reduction were enqueued on the grid's
// stream: the side stream waits for them and reduces them.  While the
// grid's stream is being captured into a caller's graph the reduction stays
// on that stream (a fork to the side stream would leave the capture
// unjoined).
static cudaError_t end_totals(mrt_grid* g, int nparts, bool capturing) {
    const int b = g->tnext;
    cudaError_t e;
    if (capturing) {
        // no event: every later use of the captured slot is ordered behind
        // it on the grid's stream, where the caller launches the graph
        return reduce_totals_on(g, mrt_grid::kCapSlot, nparts, g->stream);
    }
    if ((e = cudaEventRecord(g->ev_step[b], g->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(g->tstream, g->ev_step[b], 0)) != cudaSuccess) return e;
    if ((e = reduce_totals_on(g, b, nparts, g->tstream)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(g->ev_red[b], g->tstream)) != cudaSuccess) return e;
    g->red_pending[b] = true;
    g->tlast = b;
    g->tnext = b ^ 1;
    return cudaSuccess;
}

int grid_for(long n, int threads, int cap = 4096) {
    long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > cap ? cap : b);
}

}  // namespace

// ---------------------------------------------------------------------------
// Grid object
// ---------------------------------------------------------------------------
static EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

mrt_status mrt_encode_maps(const mrt_grid* g, void* buf, CUtensorMap* in, CUtensorMap* out) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return fail(MRT_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    const int boxw = g->fp64 ? tma_boxw<double>() : tma_boxw<float>();
    const CUtensorMapDataType dt = g->fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t strides[2] = {(cuuint64_t)(g->L.pitch * g->elem), (cuuint64_t)(g->L.plane * g->elem)};
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint64_t dims[3] = {(cuuint64_t)g->L.pitch, (cuuint64_t)(g->L.ny + 2), 16};
    cuuint32_t box[3] = {(cuuint32_t)boxw, 1, 16};
    CUresult r = enc(in, dt, 3, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MRT_ECUDA, "cuTensorMapEncodeTiled (load) failed (%d)", (int)r);
    // store map: the kernel issues row stores only for whole 128-column
    // strips, which end at or before column G + nx
    cuuint64_t odims[3] = {(cuuint64_t)(g->L.G + g->L.nx), (cuuint64_t)(g->L.ny + 2), 16};
    cuuint32_t obox[3] = {(cuuint32_t)TMA_W, 1, 16};
    r = enc(out, dt, 3, buf, odims, strides, obox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MRT_ECUDA, "cuTensorMapEncodeTiled (store) failed (%d)", (int)r);
    return MRT_OK;
}

static mrt_status make_maps(mrt_grid* g) {
    for (int b = 0; b < 2; ++b) {
        mrt_status st = mrt_encode_maps(g, g->f[b], &g->maps[b], &g->maps_out[b]);
        if (st != MRT_OK) return st;
    }
    return MRT_OK;
}

static mrt_status validate(const mrt_params* p) {
    if (!p) return fail(MRT_EINVAL, "params is NULL");
    if (p->nx < 3 || p->ny < 3) return fail(MRT_EINVAL, "nx and ny must be >= 3 (got %d x %d)", p->nx, p->ny);
    if ((long)p->nx * p->ny > (1L << 31)) return fail(MRT_EINVAL, "grid too large");
    if (!(p->dx > 0) || !std::isfinite(p->dx)) return fail(MRT_EINVAL, "dx must be finite and > 0");
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(MRT_EINVAL, "dt must be finite and > 0");
    if (!(p->gamma > 1) || !std::isfinite(p->gamma)) return fail(MRT_EINVAL, "gamma must be > 1");
    for (int k = 0; k < 16; ++k)
        if (!(p->s[k] >= 0) || !std::isfinite(p->s[k]))
            return fail(MRT_EINVAL, "rate s_%d must be finite and >= 0", k + 1);
    if (!std::isfinite(p->Pr)) return fail(MRT_EINVAL, "Pr must be finite");
    if (p->bc_x < MRT_BC_PERIODIC || p->bc_x > MRT_BC_REFLECT_FIXED) return fail(MRT_EINVAL, "bad bc_x");
    if (p->bc_y < MRT_BC_PERIODIC || p->bc_y > MRT_BC_REFLECT_FIXED) return fail(MRT_EINVAL, "bad bc_y");
    if (p->precision != MRT_FP32 && p->precision != MRT_FP64) return fail(MRT_EINVAL, "bad precision");
    if (p->kernel < MRT_KERNEL_AUTO || p->kernel > MRT_KERNEL_SPLIT) return fail(MRT_EINVAL, "bad kernel");
    if (p->tile < 0 || p->tile >= NUM_TILES) return fail(MRT_EINVAL, "bad tile %d", p->tile);
    if (p->advection != MRT_ADV_LW && p->advection != MRT_ADV_LW2D)
        return fail(MRT_EINVAL, "bad advection %d", p->advection);
    if (p->advection == MRT_ADV_LW2D && (p->kernel == MRT_KERNEL_AUTO || p->kernel == MRT_KERNEL_TMA) &&
        !tile_supports_xt(p->tile))
        return fail(MRT_EINVAL, "the unsplit operator runs on tiles 0, 1, 4, 5, 6 and 7");
    return MRT_OK;
}

static void release(mrt_grid* g) {
    if (!g) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->tstream) cudaStreamSynchronize(g->tstream);
    if (g->xstream) cudaStreamSynchronize(g->xstream);
    cudaFree(g->f[0]);
    cudaFree(g->f[1]);
    cudaFree(g->flag);
    cudaFree(g->partials);
    cudaFree(g->totals_dev);
    cudaFree(g->block_sums);
    cudaFree(g->cap_block_sums);
    cudaFree(g->cap_partials);
    cudaFree(g->seq);
    cudaFree(g->qnext);
    cudaFree(g->tile_done);
    cudaFreeHost(g->host_stage);
    for (int k = 0; k < mrt_grid::kTotalsEvents; ++k)
        if (g->tev[k]) cudaEventDestroy(g->tev[k]);
    if (g->ev_tail) cudaEventDestroy(g->ev_tail);
    for (int b = 0; b < 2; ++b) {
        if (g->ev_step[b]) cudaEventDestroy(g->ev_step[b]);
        if (g->ev_red[b]) cudaEventDestroy(g->ev_red[b]);
    }
    if (g->tstream) cudaStreamDestroy(g->tstream);
    if (g->xstream) cudaStreamDestroy(g->xstream);
    if (g->ev_x) cudaEventDestroy(g->ev_x);
    for (int c = 0; c < 2; ++c)
        for (int q = 0; q < 2; ++q)
            if (g->pair_exec[c][q]) cudaGraphExecDestroy(g->pair_exec[c][q]);
    cudaFree(g->macro_tmp);
    mrt_tape_free(g->tape);
    if (prev >= 0) cudaSetDevice(prev);
    delete g;
}

// Ghost modes of an axis at creation (every ghost set) and on a refresh
// after the state was replaced (fixed-equilibrium ghosts keep their values).
static void ghost_modes(int bc, bool creation, int* lo, int* hi) {
    if (bc == MRT_BC_PERIODIC) {
        *lo = *hi = GH_WRAP;
    } else if (bc == MRT_BC_REFLECT_FIXED) {
        *lo = GH_MIRROR;
        *hi = creation ? GH_COPY : GH_KEEP;
    } else {
        *lo = *hi = creation ? GH_COPY : GH_KEEP;
    }
}

template <class T>
static void launch_ghost_kernels(mrt_grid* g, T* f, bool creation) {
    int xl, xh, yl, yh;
    ghost_modes(g->p.bc_x, creation, &xl, &xh);
    ghost_modes(g->p.bc_y, creation, &yl, &yh);
    if (xl != GH_KEEP || xh != GH_KEEP)
        ghost_cols_kernel<T><<<grid_for(16L * g->L.ny, 256), 256, 0, g->stream>>>(g->L, xl, xh, f);
    if (yl != GH_KEEP || yh != GH_KEEP)
        ghost_rows_kernel<T><<<grid_for(16L * (g->L.nx + 2), 256), 256, 0, g->stream>>>(g->L, yl, yh, f);
}

template <class T>
static void launch_ghosts(mrt_grid* g, int buf) {
    launch_ghost_kernels<T>(g, static_cast<T*>(g->f[buf]), true);
}

// The initial state of rows [y0, y1) (fields indexed over the whole grid):
// FP64 grids in FP64, FP32 grids in double-float arithmetic.
template <class T>
static mrt_status init_rows(mrt_grid* g, const InitCoef& ic, const double* rho, const double* ux,
                            const double* uy, const double* T_, int y0, int y1) {
    if constexpr (sizeof(T) == 8)
        init_kernel<T, double><<<rows_grid(g->L, y1 - y0), 256, 0, g->stream>>>(
            g->L, init_k<double>(ic), rho, ux, uy, T_, static_cast<T*>(g->f[0]), g->flag, y0, y1);
    else
        init_kernel<T, DF><<<rows_grid(g->L, y1 - y0), 256, 0, g->stream>>>(
            g->L, init_k<DF>(ic), rho, ux, uy, T_, static_cast<T*>(g->f[0]), g->flag, y0, y1);
    CUDA_TRY(cudaGetLastError());
    return MRT_OK;
}

// The initial state from device fields, or from host fields uploaded in row
// chunks on the copy stream, each chunk initialised on the grid's stream
// once its upload is done (the next chunk's upload overlapping it); then
// the ghosts and the copy into the second buffer.
template <class T>
static mrt_status do_init(mrt_grid* g, const double* rho, const double* ux, const double* uy,
                          const double* T_, bool host) {
    InitCoef ic;
    if (mrt_init_coef_build(g->b, &ic) != 0) return fail(MRT_ECUDA, "model blocks singular");
    const long n = (long)g->L.nx * g->L.ny;
    // padding zero (a guard band no kernel writes) and ghosts cleared for
    // the ghost kernels; the initialisation writes the interior
    border_kernel<T><<<grid_for(16L * (2L * g->L.pitch + (long)g->L.ny * (g->L.pitch - g->L.nx)), 256), 256, 0,
                       g->stream>>>(g->L, nullptr, static_cast<T*>(g->f[0]));
    CUDA_TRY(cudaGetLastError());
    if (!host) {
        mrt_status st = init_rows<T>(g, ic, rho, ux, uy, T_, 0, g->L.ny);
        if (st != MRT_OK) return st;
    } else {
        if (!g->macro_tmp) {
            cudaError_t e = cudaMalloc(&g->macro_tmp, 4 * sizeof(double) * (size_t)n);
            if (e != cudaSuccess) return fail(MRT_ENOMEM, "cudaMalloc staging: %s", cudaGetErrorString(e));
        }
        const double* h[4] = {rho, ux, uy, T_};
        double* d = g->macro_tmp;
        // the copy stream starts behind the grid's stream (an earlier readout
        // of the staging buffer, a re-initialisation of a stepping grid)
        CUDA_TRY(cudaEventRecord(g->ev_x, g->stream));
        CUDA_TRY(cudaStreamWaitEvent(g->xstream, g->ev_x, 0));
        const int k = field_chunks(g->L), rows = (g->L.ny + k - 1) / k;
        for (int y0 = 0; y0 < g->L.ny; y0 += rows) {
            const int y1 = std::min(g->L.ny, y0 + rows);
            const long c0 = (long)y0 * g->L.nx, cn = (long)(y1 - y0) * g->L.nx;
            for (int q = 0; q < 4; ++q)
                CUDA_TRY(cudaMemcpyAsync(d + q * n + c0, h[q] + c0, cn * sizeof(double), cudaMemcpyHostToDevice,
                                         g->xstream));
            CUDA_TRY(cudaEventRecord(g->ev_x, g->xstream));
            CUDA_TRY(cudaStreamWaitEvent(g->stream, g->ev_x, 0));
            mrt_status st = init_rows<T>(g, ic, d, d + n, d + 2 * n, d + 3 * n, y0, y1);
            if (st != MRT_OK) return st;
        }
    }
    launch_ghosts<T>(g, 0);
    CUDA_TRY(cudaGetLastError());
    // both buffers carry the same ghosts (fixed ones are never rewritten) and
    // zero padding; the first step writes the other buffer's interior
    border_kernel<T><<<grid_for(16L * (2L * g->L.pitch + (long)g->L.ny * (g->L.pitch - g->L.nx)), 256), 256, 0,
                       g->stream>>>(g->L, static_cast<const T*>(g->f[0]), static_cast<T*>(g->f[1]));
    CUDA_TRY(cudaGetLastError());
    return MRT_OK;
}

extern "C" mrt_status mrt_create(const mrt_params* params, const double* rho, const double* ux,
                                 const double* uy, const double* T, int fields_on_device,
                                 void* stream, mrt_grid** out) {
    NvtxRange range("mrt_create");
    mrt_status st = validate(params);
    if (st != MRT_OK) return st;
    if (!out || !rho || !ux || !uy || !T) return fail(MRT_EINVAL, "null pointer argument");
    *out = nullptr;
    mrt_grid* g = new (std::nothrow) mrt_grid();
    if (!g) return fail(MRT_ENOMEM, "host allocation failed");
    g->p = *params;
    if (g->p.Pr > 0) g->p.s[7] = g->p.s[8] = g->p.Pr * g->p.s[5];
    g->fp64 = params->precision == MRT_FP64;
    g->xt = params->advection == MRT_ADV_LW2D;
    g->elem = g->fp64 ? 8 : 4;
    g->b = 2.0 / (params->gamma - 1.0);
    g->stream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&g->device);
    const int G = (int)(128 / g->elem);
    const long per128 = 128 / (long)g->elem;
    g->L.nx = params->nx;
    g->L.ny = params->ny;
    g->L.G = G;
    g->L.refl_x = params->bc_x == MRT_BC_REFLECT_FIXED;
    g->L.refl_y = params->bc_y == MRT_BC_REFLECT_FIXED;
    // room for the right ghost column, and for a whole TMA box even when the
    // grid is narrower than one strip
    const long need = std::max<long>(G + params->nx + 1, G + TMA_W + 16 / (long)g->elem);
    g->L.pitch = (need + per128 - 1) / per128 * per128;
    g->L.plane = g->L.pitch * (params->ny + 2);
    if (mrt_model_build(params->dx, params->dt, g->b, g->p.s, &g->kd) != 0) {
        delete g;
        return fail(MRT_ECUDA, "model blocks singular");
    }
    coef_cast<float, double>(g->kd, &g->kf);

    auto bail = [&](mrt_status s) { release(g); return s; };
    const size_t bytes = 16 * (size_t)g->L.plane * g->elem;
    cudaError_t e;
    if ((e = cudaMalloc(&g->f[0], bytes)) != cudaSuccess || (e = cudaMalloc(&g->f[1], bytes)) != cudaSuccess)
        return bail(fail(e == cudaErrorMemoryAllocation ? MRT_ENOMEM : MRT_ECUDA,
                         "cudaMalloc of 2 x %zu bytes failed: %s", bytes, cudaGetErrorString(e)));
    // the initialisation writes every word of buffer 0 (interior, ghosts,
    // zero padding) and the border of buffer 1
    if ((e = cudaMalloc(&g->flag, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemsetAsync(g->flag, 0, sizeof(unsigned), g->stream)) != cudaSuccess ||
        (e = cudaMalloc(&g->totals_dev, 4 * mrt_grid::kTotalsSlot * sizeof(double))) != cudaSuccess ||
        (e = cudaMemsetAsync(g->totals_dev, 0, 4 * mrt_grid::kTotalsSlot * sizeof(double), g->stream)) !=
            cudaSuccess ||
        (e = cudaMalloc(&g->seq, 4 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemsetAsync(g->seq, 0, 4 * sizeof(unsigned long long), g->stream)) != cudaSuccess ||
        (e = cudaMalloc(&g->block_sums, 4 * sizeof(double) * FINAL_MAX_BLOCKS)) != cudaSuccess ||
        (e = cudaMalloc(&g->cap_block_sums, 4 * sizeof(double) * FINAL_MAX_BLOCKS)) != cudaSuccess ||
        (e = cudaMallocHost(&g->host_stage, 8 * sizeof(double))) != cudaSuccess)
        return bail(fail(MRT_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e)));
    for (int k = 0; k < mrt_grid::kTotalsEvents; ++k)
        if ((e = cudaEventCreateWithFlags(&g->tev[k], cudaEventDisableTiming)) != cudaSuccess)
            return bail(fail(MRT_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e)));
    if ((e = cudaEventCreateWithFlags(&g->ev_tail, cudaEventDisableTiming)) != cudaSuccess)
        return bail(fail(MRT_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e)));
    for (int b = 0; b < 2; ++b)
        if ((e = cudaEventCreateWithFlags(&g->ev_step[b], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&g->ev_red[b], cudaEventDisableTiming)) != cudaSuccess)
            return bail(fail(MRT_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e)));
    if ((e = cudaStreamCreateWithFlags(&g->tstream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&g->xstream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&g->ev_x, cudaEventDisableTiming)) != cudaSuccess)
        return bail(fail(MRT_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));

    // kernel choice and launch geometry
    // AUTO: the TMA strip kernel, except for small FP64 grids, where the
    // direct kernel's small blocks spread the FP64 arithmetic over more SMs
    const long cells = (long)params->nx * params->ny;
    int kernel = params->kernel;
    if (kernel == MRT_KERNEL_AUTO) {
        if (cells <= (g->fp64 ? kSplitFp64Cells : kSplitFp32Cells)) kernel = MRT_KERNEL_SPLIT;
        else kernel = (g->fp64 && cells < kSmallFp64Cells) ? MRT_KERNEL_DIRECT : MRT_KERNEL_TMA;
    }
    int parts = 0;
    if (kernel == MRT_KERNEL_TMA) {
        int occ = 0, sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        const int strips = (params->nx + TMA_W - 1) / TMA_W;
        auto occupancy = [&](int tile, int* o) {
            return g->fp64 ? tma_occupancy<double>(tile, g->xt, o) : tma_occupancy<float>(tile, g->xt, o);
        };
        g->tile = params->tile;
        if (g->tile == 0) {
            // the work-queue tile when the grid gives every resident CTA at
            // least two items, else one static chunk of rows per CTA
            const int qt = g->xt ? kQueueTileXT : kQueueTile, qr = queue_rows(qt, g->xt);
            if ((e = occupancy(qt, &occ)) != cudaSuccess)
                return bail(fail(MRT_ECUDA, "occupancy query: %s", cudaGetErrorString(e)));
            const long items = (long)strips * ((params->ny + qr - 1) / qr);
            g->tile = items >= 2L * sms * std::max(occ, 1) ? qt : (g->fp64 ? kStaticTileF64 : kStaticTileF32);
        }
        e = occupancy(g->tile, &occ);
        if (e != cudaSuccess) return bail(fail(MRT_ECUDA, "occupancy query: %s", cudaGetErrorString(e)));
        if (occ < 1) occ = 1;
        const long resident = (long)sms * occ;
        const int qrows = queue_rows(g->tile, g->xt);
        g->strips = strips;
        if (qrows > 0) {
            // one wave of resident CTAs taking (row band, strip) items
            g->rows_per_cta = qrows;
            g->nitems = strips * ((params->ny + qrows - 1) / qrows);
            g->tma_grid_x = (int)std::min<long>(resident, g->nitems);
            g->tma_grid_y = 1;
            parts = g->nitems * (TMA_W / 32);  // one totals partial per warp of each item
            if ((e = cudaMalloc(&g->qnext, 2 * sizeof(unsigned))) != cudaSuccess ||
                (e = cudaMemsetAsync(g->qnext, 0, 2 * sizeof(unsigned), g->stream)) != cudaSuccess)
                return bail(fail(MRT_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e)));
        } else {
            // as many row chunks as fit in one wave of resident CTAs
            long chunks = resident / strips;
            if (chunks < 1) chunks = 1;
            int rows = (int)((params->ny + chunks - 1) / chunks);
            if (rows < 1) rows = 1;
            g->rows_per_cta = rows;
            g->tma_grid_x = strips;
            g->tma_grid_y = (params->ny + rows - 1) / rows;
            parts = g->tma_grid_x * g->tma_grid_y;
        }
    } else {
        dim3 gr, bl;
        if (kernel == MRT_KERNEL_SPLIT) split_grid(g->L, &gr, &bl);
        else if (g->fp64) direct_grid<double>(g->L, &gr, &bl);
        else direct_grid<float>(g->L, &gr, &bl);
        parts = (int)(gr.x * gr.y);
        if (kernel == MRT_KERNEL_SPLIT) {
            // the multi-step launch keeps every block resident: one block per
            // tile, as many as fit on the device at once
            int coop = 0, blocks = 0;
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
            e = g->fp64 ? split_persist_blocks<double>(g->xt, &blocks) : split_persist_blocks<float>(g->xt, &blocks);
            if (e != cudaSuccess) return bail(fail(MRT_ECUDA, "occupancy query: %s", cudaGetErrorString(e)));
            if (coop && blocks > 0) {
                if ((e = cudaMalloc(&g->tile_done, sizeof(unsigned) * (size_t)parts)) != cudaSuccess)
                    return bail(fail(MRT_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e)));
                g->persist_blocks = std::min(blocks, parts);
            }
        }
    }
    g->kernel = kernel;
    g->parts = parts;
    const int red_parts = grid_for((long)params->nx * params->ny, RED_THREADS, 1024);
    g->max_parts = parts > red_parts ? parts : red_parts;
    if ((e = cudaMalloc(&g->partials, 2 * 4 * sizeof(double) * (size_t)g->max_parts)) != cudaSuccess ||
        (e = cudaMalloc(&g->cap_partials, 4 * sizeof(double) * (size_t)g->max_parts)) != cudaSuccess)
        return bail(fail(MRT_ENOMEM, "cudaMalloc partials: %s", cudaGetErrorString(e)));

    if (kernel == MRT_KERNEL_TMA) {
        st = make_maps(g);
        if (st != MRT_OK) return bail(st);
    }
    st = mrt_reinit(g, rho, ux, uy, T, fields_on_device);
    if (st != MRT_OK) return bail(st);
    *out = g;
    return MRT_OK;
}

mrt_status mrt_fail(mrt_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

mrt_status mrt_reinit(mrt_grid* g, const double* rho, const double* ux, const double* uy, const double* T,
                      int on_device) {
    if (!rho || !ux || !uy || !T) return fail(MRT_EINVAL, "null field pointer");
    cudaError_t e;
    // host fields go through the grid's readout buffer (four fields of the
    // grid's size, kept for mrt_get_macro to host memory)
    CUDA_TRY(cudaMemsetAsync(g->flag, 0, sizeof(unsigned), g->stream));
    mrt_status st = g->fp64 ? do_init<double>(g, rho, ux, uy, T, !on_device)
                            : do_init<float>(g, rho, ux, uy, T, !on_device);
    // the initial state is validated by the init kernel through the flag
    unsigned h = 0;
    if (st == MRT_OK) {
        if ((e = cudaMemcpyAsync(&h, g->flag, sizeof h, cudaMemcpyDeviceToHost, g->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(g->stream)) != cudaSuccess)
            st = fail(MRT_ECUDA, "init: %s", cudaGetErrorString(e));
    } else {
        cudaStreamSynchronize(g->stream);
    }
    // no upload from the caller's memory outlives the call, even a failed one
    if (!on_device) cudaStreamSynchronize(g->xstream);
    if (st != MRT_OK) return st;
    if (h & FLAG_UNSTABLE) return fail(MRT_EINVAL, "initial state: rho and T must be finite and > 0");
    g->cur = 0;
    g->steps = 0;
    g->totals_fresh = false;
    return MRT_OK;
}

// Work-queue arguments of one launch; consecutive launches on the grid's
// stream alternate between the two counters.
static void queue_args(mrt_grid* g, StepArgsBase& a) {
    a.strips = g->strips;
    a.nitems = g->nitems;
    a.next = g->qnext;
    a.parity = g->qpar;
    if (g->qnext) g->qpar ^= 1;
}

// One step from buffer `in` to buffer `out` (padded layout, same grid), with
// the TMA maps of those buffers when the TMA kernel is in use.
template <class T>
mrt_status step_between(mrt_grid* g, const void* in, void* out, const CUtensorMap* map_in,
                        const CUtensorMap* map_out, bool totals) {
    StepArgs<T> a;
    a.L = g->L;
    a.per_x = g->p.bc_x == MRT_BC_PERIODIC;
    a.per_y = g->p.bc_y == MRT_BC_PERIODIC;
    a.rows_per_cta = g->rows_per_cta;
    a.partials = g->partials;
    a.flag = g->flag;
    if constexpr (sizeof(T) == 8) a.k = g->kd; else a.k = g->kf;
    a.in = static_cast<const T*>(in);
    a.out = static_cast<T*>(out);
    queue_args(g, a);
    cudaError_t e = g->kernel == MRT_KERNEL_TMA
        ? launch_step_tma<T>(g->tile, g->xt, map_in, map_out, a, g->tma_grid_x, g->tma_grid_y, totals, g->stream)
        : g->kernel == MRT_KERNEL_SPLIT ? launch_step_split<T>(a, g->xt, totals, g->stream)
                                        : launch_step_direct<T>(a, g->xt, totals, g->stream);
    if (e != cudaSuccess) return fail(MRT_ECUDA, "step launch: %s", cudaGetErrorString(e));
    return MRT_OK;
}
template mrt_status step_between<float>(mrt_grid*, const void*, void*, const CUtensorMap*, const CUtensorMap*, bool);
template mrt_status step_between<double>(mrt_grid*, const void*, void*, const CUtensorMap*, const CUtensorMap*, bool);

mrt_status mrt_reinit(mrt_grid* g, const double* rho, const double* ux, const double* uy, const double* T,
                      int on_device);

// One step of the grid on stream st (the last one of a call also reduces
// totals), advancing cur, the queue parity and the step count.
template <class T>
static mrt_status enqueue_step(mrt_grid* g, StepArgs<T>& a, bool totals, cudaStream_t st, bool capturing = false) {
    a.in = static_cast<const T*>(g->f[g->cur]);
    a.out = static_cast<T*>(g->f[g->cur ^ 1]);
    queue_args(g, a);
    if (totals) CUDA_TRY(begin_totals(g, &a.partials, capturing));
    cudaError_t e;
    if (g->kernel == MRT_KERNEL_TMA) {
        e = launch_step_tma<T>(g->tile, g->xt, &g->maps[g->cur], &g->maps_out[g->cur ^ 1], a, g->tma_grid_x,
                               g->tma_grid_y, totals, st);
    } else if (g->kernel == MRT_KERNEL_SPLIT) {
        e = launch_step_split<T>(a, g->xt, totals, st);
    } else {
        e = launch_step_direct<T>(a, g->xt, totals, st);
    }
    if (e != cudaSuccess) return fail(MRT_ECUDA, "step launch: %s", cudaGetErrorString(e));
    if (totals) CUDA_TRY(end_totals(g, g->parts, capturing));
    g->cur ^= 1;
    g->steps++;
    return MRT_OK;
}

template <class T>
static StepArgs<T> step_args(mrt_grid* g) {
    StepArgs<T> a;
    a.L = g->L;
    a.per_x = g->p.bc_x == MRT_BC_PERIODIC;
    a.per_y = g->p.bc_y == MRT_BC_PERIODIC;
    a.rows_per_cta = g->rows_per_cta;
    a.partials = g->partials;
    a.flag = g->flag;
    if constexpr (sizeof(T) == 8) a.k = g->kd; else a.k = g->kf;
    return a;
}

// Graph of two plain steps from the grid's present (cur, queue parity),
// captured on the side stream (never the legacy stream) and instantiated;
// after two steps cur and the parity are back where they started, so one
// graph serves every pair of steps begun in that state.
template <class T>
static mrt_status pair_graph(mrt_grid* g, cudaGraphExec_t* out) {
    const int cur0 = g->cur, q0 = g->qpar;
    const long steps0 = g->steps;
    StepArgs<T> a = step_args<T>(g);
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(g->tstream, cudaStreamCaptureModeThreadLocal));
    mrt_status st = enqueue_step<T>(g, a, false, g->tstream);
    if (st == MRT_OK) st = enqueue_step<T>(g, a, false, g->tstream);
    const cudaError_t e = cudaStreamEndCapture(g->tstream, &graph);
    g->cur = cur0;
    g->qpar = q0;
    g->steps = steps0;
    if (st != MRT_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != MRT_OK ? st : fail(MRT_ECUDA, "step graph capture: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(MRT_ECUDA, "step graph: %s", cudaGetErrorString(ei));
    return MRT_OK;
}

// All but the last step of a call replay two-step graphs (fewer launch gaps
// on small grids); the last step, which also reduces totals, and an odd one
// before it are launched directly.
// All steps of a call in one launch of the split kernel's multi-step form,
// the last one reducing totals.  At most 2^31 - 1 steps per launch.
template <class T>
static mrt_status persist_steps(mrt_grid* g, long nsteps) {
    StepArgs<T> a = step_args<T>(g);
    CUDA_TRY(begin_totals(g, &a.partials, false));
    CUDA_TRY(cudaMemsetAsync(g->tile_done, 0, sizeof(unsigned) * (size_t)g->parts, g->stream));
    T* b0 = static_cast<T*>(g->f[g->cur]);
    T* b1 = static_cast<T*>(g->f[g->cur ^ 1]);
    a.in = b0;
    a.out = b1;
    const cudaError_t e = launch_step_split_persist<T>(a, g->xt, b0, b1, (int)nsteps, true, g->tile_done,
                                                       g->persist_blocks, g->stream);
    if (e != cudaSuccess) return fail(MRT_ECUDA, "multi-step launch: %s", cudaGetErrorString(e));
    CUDA_TRY(end_totals(g, g->parts, false));
    g->cur ^= (int)(nsteps & 1);
    g->steps += nsteps;
    g->totals_fresh = true;
    return MRT_OK;
}

template <class T>
static mrt_status step_impl(mrt_grid* g, long nsteps, bool allow_persist = true) {
    StepArgs<T> a = step_args<T>(g);
    // while a caller captures the grid's stream, every step is launched
    // directly and the totals are reduced on that stream
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(g->stream, &cs));
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    if (allow_persist && g->persist_blocks > 0 && nsteps >= 2 && !capturing) {
        for (long done = 0; done < nsteps;) {
            const long n = std::min<long>(nsteps - done, 1L << 30);
            mrt_status st = persist_steps<T>(g, n);
            if (st != MRT_OK) return st;
            done += n;
        }
        return MRT_OK;
    }
    long plain = nsteps - 1;
    if (plain >= 2 && !capturing) {
        cudaGraphExec_t& ex = g->pair_exec[g->cur][g->qpar & 1];
        if (!ex) {
            mrt_status st = pair_graph<T>(g, &ex);
            if (st != MRT_OK) return st;
        }
        const long pairs = plain / 2;
        for (long k = 0; k < pairs; ++k) CUDA_TRY(cudaGraphLaunch(ex, g->stream));
        g->steps += 2 * pairs;
        plain -= 2 * pairs;
    }
    for (long s = 0; s < plain; ++s) {
        mrt_status st = enqueue_step<T>(g, a, false, g->stream);
        if (st != MRT_OK) return st;
    }
    if (nsteps > 0) {
        mrt_status st = enqueue_step<T>(g, a, true, g->stream, capturing);
        if (st != MRT_OK) return st;
        g->totals_fresh = true;
    }
    return MRT_OK;
}

// Steps launched one at a time (the form the reverse sweep recomputes a
// segment with), for the recorded forward run of the reverse mode.
mrt_status mrt_step_single_launches(mrt_grid* g, long nsteps) {
    if (nsteps <= 0) return MRT_OK;
    return g->fp64 ? step_impl<double>(g, nsteps, false) : step_impl<float>(g, nsteps, false);
}

extern "C" mrt_status mrt_step(mrt_grid* g, long nsteps) {
    NvtxRange range("mrt_step");
    if (!g) return fail(MRT_EINVAL, "grid is NULL");
    if (nsteps < 0) return fail(MRT_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return MRT_OK;
    return g->fp64 ? step_impl<double>(g, nsteps) : step_impl<float>(g, nsteps);
}

template <class T>
static mrt_status macro_impl(mrt_grid* g, double* rho, double* ux, double* uy, double* Tf, int y0, int y1) {
    macro_kernel<T><<<rows_grid(g->L, y1 - y0), 256, 0, g->stream>>>(
        g->L, 1.0 / g->b, static_cast<const T*>(g->f[g->cur]), rho, ux, uy, Tf, y0, y1);
    CUDA_TRY(cudaGetLastError());
    return MRT_OK;
}

extern "C" mrt_status mrt_get_macro(mrt_grid* g, double* rho, double* ux, double* uy, double* T,
                                    int dst_on_device) {
    if (!g) return fail(MRT_EINVAL, "grid is NULL");
    const long n = (long)g->L.nx * g->L.ny;
    if (dst_on_device)
        return g->fp64 ? macro_impl<double>(g, rho, ux, uy, T, 0, g->L.ny)
                       : macro_impl<float>(g, rho, ux, uy, T, 0, g->L.ny);
    if (!g->macro_tmp) CUDA_TRY(cudaMalloc(&g->macro_tmp, 4 * sizeof(double) * (size_t)n));
    double* d[4];
    double* h[4] = {rho, ux, uy, T};
    for (int q = 0; q < 4; ++q) d[q] = h[q] ? g->macro_tmp + q * n : nullptr;
    // row chunks: the kernel on the grid's stream, each chunk's download on
    // the copy stream once its kernel is done (overlapping the next chunk's)
    const int k = field_chunks(g->L), rows = (g->L.ny + k - 1) / k;
    mrt_status st = MRT_OK;
    for (int y0 = 0; y0 < g->L.ny && st == MRT_OK; y0 += rows) {
        const int y1 = std::min(g->L.ny, y0 + rows);
        const long c0 = (long)y0 * g->L.nx, cn = (long)(y1 - y0) * g->L.nx;
        st = g->fp64 ? macro_impl<double>(g, d[0], d[1], d[2], d[3], y0, y1)
                     : macro_impl<float>(g, d[0], d[1], d[2], d[3], y0, y1);
        cudaError_t e = cudaSuccess;
        if (st == MRT_OK && ((e = cudaEventRecord(g->ev_x, g->stream)) != cudaSuccess ||
                             (e = cudaStreamWaitEvent(g->xstream, g->ev_x, 0)) != cudaSuccess))
            st = fail(MRT_ECUDA, "readout: %s", cudaGetErrorString(e));
        for (int q = 0; q < 4 && st == MRT_OK; ++q)
            if (h[q] && (e = cudaMemcpyAsync(h[q] + c0, d[q] + c0, cn * sizeof(double), cudaMemcpyDeviceToHost,
                                             g->xstream)) != cudaSuccess)
                st = fail(MRT_ECUDA, "readout: %s", cudaGetErrorString(e));
    }
    // no download into the caller's memory outlives the call, even a failed one
    const cudaError_t e = cudaStreamSynchronize(g->xstream);
    if (st == MRT_OK && e != cudaSuccess) st = fail(MRT_ECUDA, "readout: %s", cudaGetErrorString(e));
    return st;
}

template <class T>
static mrt_status totals_impl(mrt_grid* g) {
    const long n = (long)g->L.nx * g->L.ny;
    const int blocks = grid_for(n, RED_THREADS, 1024);
    double* parts = nullptr;
    CUDA_TRY(begin_totals(g, &parts, false));
    totals_partial_kernel<T><<<blocks, RED_THREADS, 0, g->stream>>>(g->L, static_cast<const T*>(g->f[g->cur]),
                                                                     parts);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(end_totals(g, blocks, false));
    g->totals_fresh = true;
    return MRT_OK;
}

// Totals slot a reader copies, on the side stream after everything enqueued
// on the grid's stream: the side stream's latest, or, once the grid has been
// captured, whichever of that and the captured slot has the newer stamp
// (a replay and direct steps may alternate in any order).
static mrt_status reader_slot(mrt_grid* g, int* slot) {
    CUDA_TRY(tail_to_side(g));
    *slot = g->tlast;
    if (g->cap_used) {
        totals_pick_kernel<<<1, 1, 0, g->tstream>>>(g->totals_dev, g->tlast, mrt_grid::kCapSlot,
                                                    mrt_grid::kPickSlot);
        CUDA_TRY(cudaGetLastError());
        *slot = mrt_grid::kPickSlot;
    }
    return MRT_OK;
}

// The totals readers copy on the side stream, which a capture of the grid's
// stream cannot take in: they refuse to run inside one.
static mrt_status refuse_in_capture(mrt_grid* g) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(g->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) return fail(MRT_EINVAL, "the grid's stream is being captured");
    return MRT_OK;
}

extern "C" mrt_status mrt_conserved_totals(mrt_grid* g, double out[4]) {
    if (!g || !out) return fail(MRT_EINVAL, "null argument");
    if (mrt_status st = refuse_in_capture(g); st != MRT_OK) return st;
    if (!g->totals_fresh) {
        mrt_status st = g->fp64 ? totals_impl<double>(g) : totals_impl<float>(g);
        if (st != MRT_OK) return st;
    }
    int slot = 0;
    if (mrt_status st = reader_slot(g, &slot); st != MRT_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(g->host_stage, g->totals_dev + mrt_grid::kTotalsSlot * slot, 5 * sizeof(double),
                             cudaMemcpyDeviceToHost, g->tstream));
    CUDA_TRY(cudaStreamSynchronize(g->tstream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    for (int k = 0; k < 4; ++k) out[k] = g->host_stage[k];
    const unsigned flag = (unsigned)g->host_stage[4];
    if (flag & FLAG_TIMEOUT) return fail(MRT_ETIMEOUT, "a device-side wait ran out");
    if (flag & FLAG_UNSTABLE) return fail(MRT_EUNSTABLE, "non-positive or non-finite rho or pressure");
    return MRT_OK;
}

extern "C" mrt_status mrt_conserved_totals_async(mrt_grid* g, double* dst, long* ticket) {
    if (!g || !dst || !ticket) return fail(MRT_EINVAL, "null argument");
    if (mrt_status st = refuse_in_capture(g); st != MRT_OK) return st;
    if (!g->totals_fresh) {
        mrt_status st = g->fp64 ? totals_impl<double>(g) : totals_impl<float>(g);
        if (st != MRT_OK) return st;
    }
    // on the side stream, after the reduction of the latest totals; the
    // grid's stream runs on meanwhile
    int slot = 0;
    if (mrt_status st = reader_slot(g, &slot); st != MRT_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(dst, g->totals_dev + mrt_grid::kTotalsSlot * slot, 5 * sizeof(double),
                             cudaMemcpyDeviceToHost, g->tstream));
    const long t = g->tickets;
    CUDA_TRY(cudaEventRecord(g->tev[t % mrt_grid::kTotalsEvents], g->tstream));
    // a replay of a captured graph writes its totals slot on the grid's
    // stream: later work there waits until this copy has read it
    if (g->cap_used) CUDA_TRY(cudaStreamWaitEvent(g->stream, g->tev[t % mrt_grid::kTotalsEvents], 0));
    g->tickets = t + 1;
    *ticket = t;
    return MRT_OK;
}

extern "C" mrt_status mrt_totals_wait(mrt_grid* g, long ticket) {
    if (!g) return fail(MRT_EINVAL, "grid is NULL");
    if (ticket < 0 || ticket >= g->tickets) return fail(MRT_EINVAL, "ticket %ld was never issued", ticket);
    CUDA_TRY(cudaEventSynchronize(g->tev[ticket % mrt_grid::kTotalsEvents]));
    return MRT_OK;
}

mrt_status mrt_refresh_periodic_ghosts(mrt_grid* g, void* buf);

static mrt_status copy_f(mrt_grid* g, void* f, int on_device, bool to_grid) {
    const size_t rowb = (size_t)g->L.nx * g->elem;
    const size_t dpitch = (size_t)g->L.pitch * g->elem;
    const cudaMemcpyKind kind = to_grid ? (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                                        : (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    char* dev = static_cast<char*>(g->f[g->cur]);
    char* usr = static_cast<char*>(f);
    for (int i = 0; i < 16; ++i) {
        char* dplane = dev + ((size_t)i * g->L.plane + g->L.pitch + g->L.G) * g->elem;
        char* uplane = usr + (size_t)i * g->L.nx * g->L.ny * g->elem;
        cudaError_t e = to_grid
            ? cudaMemcpy2DAsync(dplane, dpitch, uplane, rowb, rowb, g->L.ny, kind, g->stream)
            : cudaMemcpy2DAsync(uplane, rowb, dplane, dpitch, rowb, g->L.ny, kind, g->stream);
        if (e != cudaSuccess) return fail(MRT_ECUDA, "state copy: %s", cudaGetErrorString(e));
    }
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(g->stream));
    return MRT_OK;
}

extern "C" mrt_status mrt_get_f(mrt_grid* g, void* f, int on_device) {
    if (!g || !f) return fail(MRT_EINVAL, "null argument");
    return copy_f(g, f, on_device, false);
}

extern "C" mrt_status mrt_set_f(mrt_grid* g, const void* f, int on_device) {
    if (!g || !f) return fail(MRT_EINVAL, "null argument");
    mrt_status st = copy_f(g, const_cast<void*>(f), on_device, true);
    if (st != MRT_OK) return st;
    // periodic ghosts follow the new state; fixed-equilibrium ghosts keep the
    // boundary values set at creation
    st = mrt_refresh_periodic_ghosts(g, g->f[g->cur]);
    if (st != MRT_OK) return st;
    g->totals_fresh = false;
    return MRT_OK;
}

// Periodic and reflecting-wall ghosts of a padded buffer from its own data
// (fixed-equilibrium ghosts keep their values).
mrt_status mrt_refresh_periodic_ghosts(mrt_grid* g, void* buf) {
    if (g->fp64)
        launch_ghost_kernels<double>(g, static_cast<double*>(buf), false);
    else
        launch_ghost_kernels<float>(g, static_cast<float*>(buf), false);
    CUDA_TRY(cudaGetLastError());
    return MRT_OK;
}

extern "C" mrt_status mrt_health(mrt_grid* g) {
    if (!g) return fail(MRT_EINVAL, "grid is NULL");
    unsigned* flag = reinterpret_cast<unsigned*>(g->host_stage + 6);
    CUDA_TRY(cudaMemcpyAsync(flag, g->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (*flag & FLAG_TIMEOUT) return fail(MRT_ETIMEOUT, "a device-side wait ran out");
    if (*flag & FLAG_UNSTABLE) return fail(MRT_EUNSTABLE, "non-positive or non-finite rho or pressure");
    return MRT_OK;
}

extern "C" mrt_status mrt_info(const mrt_grid* g, long* steps, long* pitch, long* plane_stride,
                               int* kernel_in_use, int* tile_in_use) {
    if (!g) return fail(MRT_EINVAL, "grid is NULL");
    if (steps) *steps = g->steps;
    if (pitch) *pitch = g->L.pitch;
    if (plane_stride) *plane_stride = g->L.plane;
    if (kernel_in_use) *kernel_in_use = g->kernel;
    if (tile_in_use) *tile_in_use = g->tile;
    return MRT_OK;
}

extern "C" void mrt_destroy(mrt_grid* g) { release(g); }

extern "C" const char* mrt_status_str(mrt_status s) {
    switch (s) {
        case MRT_OK: return "MRT_OK";
        case MRT_EINVAL: return "MRT_EINVAL";
        case MRT_ENOMEM: return "MRT_ENOMEM";
        case MRT_ECUDA: return "MRT_ECUDA";
        case MRT_EUNSTABLE: return "MRT_EUNSTABLE";
        case MRT_ETIMEOUT: return "MRT_ETIMEOUT";
    }
    return "MRT_UNKNOWN";
}

extern "C" const char* mrt_last_error(void) { return g_err; }
