/*
 * FP64 CPU oracle for the two-dimensional 16-velocity (D2V16) thermal
 * multiple-relaxation-time finite-difference lattice Boltzmann step of
 * Chen, Xu, Zhang, Li and Succi, "Multiple-Relaxation-Time Lattice Boltzmann
 * Approach to Compressible Flows with Flexible Specific-Heat Ratio and Prandtl
 * Number" (arXiv:1004.5442).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the GPU library computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code, header
 * or table with the CUDA library: the model (velocities, eta, M) is built here
 * from the paper's definitions and inverted here by Gauss-Jordan elimination.
 *
 * Everything is FP64, dense 16x16 loops, no blocking, fusion or reordering
 * beyond what the method states:
 *   Eq. 3        d_t f_i + v_ia d_a f_i = -Minv_il S_lk (fhat_k - fhat_k^eq)
 *   Sect. "Construction of energy-conserving MRT LB model": velocity set,
 *                eta_i, gamma = (b+2)/b, forward-Euler time stepping and
 *                Lax-Wendroff space discretisation
 *   Appendix     rows m_1..m_16 of M and the equilibria fhat^eq_1..16
 *   Eq. 12 text  P = rho R T, e = b rho R T + j^2/rho (R = 1 throughout,
 *                Sect. "Numerical Simulation and Analysis")
 *   Sect. (b)    boundary nodes held at f^eq = Minv fhat^eq; y periodic
 *
 * Readings where the paper is silent:
 *   - order inside the "cyc" groups: (1,0),(0,1),(-1,0),(0,-1) and
 *     (1,1),(-1,1),(-1,-1),(1,-1) times the group speed factor;
 *   - "first-order upwind" in time is forward Euler; the Lax-Wendroff space
 *     operator is applied axis by axis with the dt-dependent second
 *     difference, without a mixed x-y term; the collision is explicit at t_n;
 *   - eta enters M only as eta_i^2 = 25/4 for i = 1..4, 0 otherwise;
 *   - a fixed-equilibrium boundary is one ghost cell beyond the domain that
 *     holds, for ever, the initial f (= f^eq of the initial state) of the
 *     adjacent domain cell;
 *   - a reflecting boundary (Sect. (d): the velocity component normal to the
 *     wall is the reverse of the one at the mirror-image interior point) is
 *     one ghost cell beyond the domain holding, at every step, the adjacent
 *     domain cell's f with each velocity mirrored across the wall: f_i of
 *     the ghost = f_j of the cell, v_j the mirror image of v_i.  Axis kind
 *     ORC_BC_REFLECT_FIXED puts such a wall at the low end and a
 *     fixed-equilibrium inflow at the high end.
 *
 * Storage: f[i][y][x], i = 0..15 (paper's i = 1..16), x fastest, no padding.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 16

enum { ORC_BC_PERIODIC = 0, ORC_BC_FIXED_EQ = 1, ORC_BC_REFLECT_FIXED = 2 };

typedef struct {
    int nx, ny;
    double dx, dt;     /* dy == dx */
    double b;          /* total number of degrees of freedom; gamma = (b+2)/b */
    double s[NV];      /* relaxation rates s_1..s_16 in 1/time */
    int bc_x, bc_y;    /* ORC_BC_PERIODIC, ORC_BC_FIXED_EQ or ORC_BC_REFLECT_FIXED */
    int advection;     /* ORC_ADV_* below */
} orc_cfg;

/* Space discretisation of v_ia d_a f_i.
 *   ORC_ADV_LW      the paper's Lax-Wendroff operator, axis by axis (the
 *                   reading taken for the method);
 *   ORC_ADV_LW2D    the unsplit two-dimensional Lax-Wendroff operator: the
 *                   same plus the mixed term c_x c_y d_xy f of the
 *                   second-order Taylor expansion in time, on the four
 *                   diagonal neighbours (the other reading of the paper's
 *                   "Lax-Wendroff");
 *   ORC_ADV_MINMOD,
 *   ORC_ADV_VANLEER flux-limited variants outside the paper (it names flux
 *                   limiters only as earlier work on stabilising LB
 *                   schemes): per velocity and axis the Lax-Wendroff flux is
 *                   the first-order upwind flux plus a correction scaled by
 *                   a limiter phi (Sweby's form); phi = 1 gives ORC_ADV_LW;
 *   ORC_ADV_LWFULL  another reading of the time scheme: the Lax-Wendroff
 *                   (second-order Taylor) step of the whole kinetic
 *                   equation, Eq. 3 including its collision term:
 *                     f^{n+1} = f + dt f_t + (dt^2/2) f_tt,
 *                     f_t  = -v.grad f + Omega(f),
 *                     f_tt = (v.grad)^2 f - v.grad Omega + J (-v.grad f + Omega),
 *                   J = dOmega/df at the cell; v.grad by central differences,
 *                   (v.grad)^2 as in ORC_ADV_LW2D (second differences and the
 *                   four-corner mixed term), so with S = 0 it is ORC_ADV_LW2D.
 *                   Forward step only (no reverse mode). */
enum { ORC_ADV_LW = 0, ORC_ADV_LW2D = 1, ORC_ADV_MINMOD = 2, ORC_ADV_VANLEER = 3, ORC_ADV_LWFULL = 4 };

/* ------------------------------------------------------------------------ */
/* Model: velocity set, eta_i, M and its inverse.                            */
/* ------------------------------------------------------------------------ */

/* D2V16 velocity set (Sect. "Construction of energy-conserving MRT LB model",
 * velocity table): cyc(+-1,0) for i=1..4, cyc(+-6,0) for i=5..8,
 * sqrt(2)(+-1,+-1) for i=9..12, (3/sqrt(2))(+-1,+-1) for i=13..16. */
void orc_velocities(double vx[NV], double vy[NV], double eta2[NV])
{
    static const double axis[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
    static const double diag[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    const double c_diag2 = sqrt(2.0);
    const double c_diag3 = 3.0 / sqrt(2.0);
    for (int k = 0; k < 4; ++k) {
        vx[k] = axis[k][0];            vy[k] = axis[k][1];
        vx[4 + k] = 6.0 * axis[k][0];  vy[4 + k] = 6.0 * axis[k][1];
        vx[8 + k] = c_diag2 * diag[k][0];  vy[8 + k] = c_diag2 * diag[k][1];
        vx[12 + k] = c_diag3 * diag[k][0]; vy[12 + k] = c_diag3 * diag[k][1];
    }
    /* eta_i = 5/2 for i = 1..4 and 0 otherwise; it enters only squared. */
    for (int i = 0; i < NV; ++i) eta2[i] = (i < 4) ? 6.25 : 0.0;
}

/* Transformation matrix, Appendix: M = (m_1, ..., m_16)^T with
 *   m_1 = 1, m_2 = vx, m_3 = vy, m_4 = v^2 + eta^2, m_5 = v^2,
 *   m_6 = vx^2 - vy^2, m_7 = vx vy, m_8 = vx (v^2+eta^2), m_9 = vy (v^2+eta^2),
 *   m_10 = vx v^2, m_11 = vy v^2, m_12 = vx (vx^2-vy^2), m_13 = vy (vx^2-vy^2),
 *   m_14 = v^2 (v^2+eta^2), m_15 = vx vy (v^2+eta^2),
 *   m_16 = (vx^2-vy^2)(v^2+eta^2).
 * M[k*16 + i] = m_{k+1, i+1}. */
void orc_build_M(const double vx[NV], const double vy[NV], const double eta2[NV],
                 double *M)
{
    for (int i = 0; i < NV; ++i) {
        const double x = vx[i], y = vy[i];
        const double v2 = x * x + y * y;
        const double w = v2 + eta2[i];
        const double d = x * x - y * y;
        M[0 * NV + i] = 1.0;
        M[1 * NV + i] = x;
        M[2 * NV + i] = y;
        M[3 * NV + i] = w;
        M[4 * NV + i] = v2;
        M[5 * NV + i] = d;
        M[6 * NV + i] = x * y;
        M[7 * NV + i] = x * w;
        M[8 * NV + i] = y * w;
        M[9 * NV + i] = x * v2;
        M[10 * NV + i] = y * v2;
        M[11 * NV + i] = x * d;
        M[12 * NV + i] = y * d;
        M[13 * NV + i] = v2 * w;
        M[14 * NV + i] = x * y * w;
        M[15 * NV + i] = d * w;
    }
}

/* Gauss-Jordan elimination with partial pivoting on an n x n row-major
 * matrix.  Returns 0 on success, -1 if a pivot is exactly zero. */
int orc_invert(const double *A, double *Ainv, int n)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(2 * n));
    if (!a) return -1;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            a[r * 2 * n + c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * 2 * n + col]) > fabs(a[piv * 2 * n + col])) piv = r;
        if (a[piv * 2 * n + col] == 0.0) { free(a); return -1; }
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = a[col * 2 * n + c];
                a[col * 2 * n + c] = a[piv * 2 * n + c];
                a[piv * 2 * n + c] = t;
            }
        const double p = a[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) a[col * 2 * n + c] /= p;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double m = a[r * 2 * n + col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) a[r * 2 * n + c] -= m * a[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r * 2 * n + n + c];
    free(a);
    return 0;
}

/* The oracle's model, built once per process. */
static double g_vx[NV], g_vy[NV], g_eta2[NV], g_M[NV * NV], g_Minv[NV * NV];
static int g_model_ready = 0;

static void ensure_model(void)
{
    if (g_model_ready) return;
    orc_velocities(g_vx, g_vy, g_eta2);
    orc_build_M(g_vx, g_vy, g_eta2, g_M);
    orc_invert(g_M, g_Minv, NV);
    g_model_ready = 1;
}

/* Copy out the oracle's model: velocities, eta^2, M and M^-1 (row-major). */
void orc_model(double vx[NV], double vy[NV], double eta2[NV], double *M, double *Minv)
{
    ensure_model();
    memcpy(vx, g_vx, sizeof g_vx);
    memcpy(vy, g_vy, sizeof g_vy);
    memcpy(eta2, g_eta2, sizeof g_eta2);
    memcpy(M, g_M, sizeof g_M);
    memcpy(Minv, g_Minv, sizeof g_Minv);
}

/* ------------------------------------------------------------------------ */
/* Equilibrium moments (Appendix) and the macroscopic closure (Eq. 12 text). */
/* ------------------------------------------------------------------------ */

/* fhat^eq_1..16 from the conserved moments rho, jx, jy, e (R = 1):
 * P = rho R T with e = b rho R T + j^2/rho, so P = (e - j^2/rho)/b. */
void orc_feq_moments(double rho, double jx, double jy, double e, double b,
                     double out[NV])
{
    const double R = 1.0;
    const double j2 = jx * jx + jy * jy;
    const double P = (e - j2 / rho) / b;
    const double T = P / (rho * R);
    const double dj = jx * jx - jy * jy;
    out[0] = rho;
    out[1] = jx;
    out[2] = jy;
    out[3] = e;
    out[4] = 2.0 * P + j2 / rho;
    out[5] = dj / rho;
    out[6] = jx * jy / rho;
    out[7] = (e + 2.0 * P) * jx / rho;
    out[8] = (e + 2.0 * P) * jy / rho;
    out[9] = (4.0 * P + jx * jx / rho + jy * jy / rho) * jx / rho;
    out[10] = (4.0 * P + jx * jx / rho + jy * jy / rho) * jy / rho;
    out[11] = (2.0 * P + jx * jx / rho - jy * jy / rho) * jx / rho;
    out[12] = (-2.0 * P + jx * jx / rho - jy * jy / rho) * jy / rho;
    out[13] = 2.0 * (b + 2.0) * rho * R * R * T * T
            + (6.0 + b) * R * T * j2 / rho
            + j2 * j2 / (rho * rho * rho);
    out[14] = ((b + 4.0) * P + j2 / rho) * jx * jy / (rho * rho);
    out[15] = ((b + 4.0) * P + j2 / rho) * dj / (rho * rho);
}

/* Velocity-space equilibrium f^eq = M^-1 fhat^eq (Sect. (b), boundary nodes;
 * also the initial state). */
void orc_feq(double rho, double ux, double uy, double T, double b, double feq[NV])
{
    ensure_model();
    const double jx = rho * ux, jy = rho * uy;
    const double e = b * rho * T + (jx * jx + jy * jy) / rho;
    double m[NV];
    orc_feq_moments(rho, jx, jy, e, b, m);
    for (int i = 0; i < NV; ++i) {
        double acc = 0.0;
        for (int k = 0; k < NV; ++k) acc += g_Minv[i * NV + k] * m[k];
        feq[i] = acc;
    }
}

/* Initial state: f_i(x, y) = f^eq_i(rho, u, T) for every cell. */
void orc_init(int nx, int ny, double b, const double *rho, const double *ux,
              const double *uy, const double *T, double *f)
{
    const size_t n = (size_t)nx * (size_t)ny;
    for (size_t c = 0; c < n; ++c) {
        double feq[NV];
        orc_feq(rho[c], ux[c], uy[c], T[c], b, feq);
        for (int i = 0; i < NV; ++i) f[(size_t)i * n + c] = feq[i];
    }
}

/* Fixed-equilibrium ghost cells, taken from the initial f: gx[i][side][y]
 * (side 0 = x = -1, side 1 = x = nx) and gy[i][side][x] (side 0 = y = -1,
 * side 1 = y = ny).  Each ghost copies the adjacent domain cell. */
void orc_ghosts_from_initial(int nx, int ny, const double *f0, double *gx, double *gy)
{
    const size_t n = (size_t)nx * (size_t)ny;
    for (int i = 0; i < NV; ++i) {
        for (int y = 0; y < ny; ++y) {
            gx[((size_t)i * 2 + 0) * ny + y] = f0[(size_t)i * n + (size_t)y * nx + 0];
            gx[((size_t)i * 2 + 1) * ny + y] = f0[(size_t)i * n + (size_t)y * nx + (nx - 1)];
        }
        for (int x = 0; x < nx; ++x) {
            gy[((size_t)i * 2 + 0) * nx + x] = f0[(size_t)i * n + 0 * (size_t)nx + x];
            gy[((size_t)i * 2 + 1) * nx + x] = f0[(size_t)i * n + (size_t)(ny - 1) * nx + x];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One time step.                                                           */
/* ------------------------------------------------------------------------ */

/* Index j of the velocity whose v_j is the mirror image of v_i across a
 * wall normal to x (axis 0) or to y (axis 1), found in the velocity table. */
static int mirror_index(int i, int axis)
{
    const double tx = axis == 0 ? -g_vx[i] : g_vx[i];
    const double ty = axis == 1 ? -g_vy[i] : g_vy[i];
    for (int j = 0; j < NV; ++j)
        if (fabs(g_vx[j] - tx) < 1e-12 && fabs(g_vy[j] - ty) < 1e-12 && g_eta2[j] == g_eta2[i]) return j;
    return -1;
}

/* f_i at (x, y) for x in -2..nx+1 and y in -2..ny+1, either axis or both
 * outside the domain.  Each axis is mapped in turn, x first:
 *   periodic            the wrapped index;
 *   reflecting wall     (low end) the mirrored velocity at the mirror-image
 *                       cell: -1 <-> 0, -2 <-> 1;
 *   fixed equilibrium   the ghost, whose every layer holds the initial f of
 *                       the adjacent domain cell (a corner beyond two fixed
 *                       ends: the initial f of the corner cell).
 * A fixed ghost is looked up at the other axis's mapped index. */
static double fat(const orc_cfg *c, const double *f, const double *gx,
                  const double *gy, int i, int x, int y)
{
    const int nx = c->nx, ny = c->ny;
    const size_t n = (size_t)nx * (size_t)ny;
    int side_x = -1, side_y = -1;      /* fixed ghost on that side, or -1 */
    if (x < 0 || x >= nx) {
        if (c->bc_x == ORC_BC_PERIODIC) {
            x = ((x % nx) + nx) % nx;
        } else if (c->bc_x == ORC_BC_REFLECT_FIXED && x < 0) {
            i = mirror_index(i, 0);
            x = -x - 1;
        } else {
            side_x = (x < 0) ? 0 : 1;
            x = (x < 0) ? 0 : nx - 1;
        }
    }
    if (y < 0 || y >= ny) {
        if (c->bc_y == ORC_BC_PERIODIC) {
            y = ((y % ny) + ny) % ny;
        } else if (c->bc_y == ORC_BC_REFLECT_FIXED && y < 0) {
            i = mirror_index(i, 1);
            y = -y - 1;
        } else {
            side_y = (y < 0) ? 0 : 1;
            y = (y < 0) ? 0 : ny - 1;
        }
    }
    if (side_x >= 0) return gx[((size_t)i * 2 + side_x) * ny + y];
    if (side_y >= 0) return gy[((size_t)i * 2 + side_y) * nx + x];
    return f[(size_t)i * n + (size_t)y * nx + x];
}

/* Limiter phi(theta) of the flux-limited variants, theta = ratio of the
 * upwind-side difference to the local difference at a face:
 *   minmod:   phi = max(0, min(1, theta))
 *   van Leer: phi = (theta + |theta|) / (1 + |theta|)   (-> 2 as theta -> inf)
 * Any other value of lim is phi = 1 (the Lax-Wendroff flux). */
static double limiter_phi(int lim, double theta)
{
    if (lim == ORC_ADV_MINMOD) return fmax(0.0, fmin(1.0, theta));
    if (lim == ORC_ADV_VANLEER) {
        if (!(theta > 0.0)) return 0.0;
        if (isinf(theta)) return 2.0;
        return (theta + fabs(theta)) / (1.0 + fabs(theta));
    }
    return 1.0;
}

/* d phi / d theta, with the one-sided value that the forward branch takes
 * at the kinks (a subgradient): minmod 1 on 0 < theta < 1 and 0 elsewhere
 * (theta = 0 and theta = 1 take 0); van Leer 2/(1+theta)^2 for theta > 0
 * and 0 for theta <= 0. */
static double limiter_dphi(int lim, double theta)
{
    if (lim == ORC_ADV_MINMOD) return (theta > 0.0 && theta < 1.0) ? 1.0 : 0.0;
    if (lim == ORC_ADV_VANLEER) {
        if (!(theta > 0.0) || isinf(theta)) return 0.0;
        return 2.0 / ((1.0 + theta) * (1.0 + theta));
    }
    return 0.0;
}

/* Flux of one velocity through the face between cells j and j+1 along one
 * axis, in units of f per step, c = v dt/dx (|c| <= 1):
 *   F = c f_upwind + (|c| (1 - |c|) / 2) phi(theta) (f_{j+1} - f_j),
 *   f_upwind = f_j, theta = (f_j - f_{j-1}) / (f_{j+1} - f_j)        (c >= 0)
 *   f_upwind = f_{j+1}, theta = (f_{j+2} - f_{j+1}) / (f_{j+1} - f_j) (c < 0)
 * and the correction is 0 where f_{j+1} = f_j.  With phi = 1 the
 * difference of two such fluxes is the Lax-Wendroff operator
 * -(c/2)(f_+ - f_-) + (c^2/2)(f_+ - 2 f + f_-).
 * d[0..3] receives dF/d(f_{j-1}, f_j, f_{j+1}, f_{j+2}) (subgradient at
 * the limiter's kinks, see limiter_dphi). */
static double face_flux(int lim, double c, double fjm1, double fj, double fj1, double fj2, double d[4])
{
    const double ac = fabs(c);
    const double K = 0.5 * ac * (1.0 - ac);
    const double dloc = fj1 - fj;
    const double dup = (c >= 0.0) ? fj - fjm1 : fj2 - fj1;
    double F = (c >= 0.0) ? c * fj : c * fj1;
    double dcorr_dup = 0.0, dcorr_dloc = 0.0;
    if (dloc != 0.0) {
        const double th = dup / dloc;
        const double ph = limiter_phi(lim, th), dph = limiter_dphi(lim, th);
        F += K * ph * dloc;
        dcorr_dup = dph;
        dcorr_dloc = ph - th * dph;
    }
    d[0] = d[1] = d[2] = d[3] = 0.0;
    if (c >= 0.0) {
        d[1] += c;
        d[1] += K * dcorr_dup;   d[0] -= K * dcorr_dup;
    } else {
        d[2] += c;
        d[3] += K * dcorr_dup;   d[2] -= K * dcorr_dup;
    }
    d[2] += K * dcorr_dloc;  d[1] -= K * dcorr_dloc;
    return F;
}

/* Advection increment of velocity i at (x, y) in a flux-limited variant:
 * minus the flux difference across the cell along x and along y.  If dA is
 * not NULL it receives dAdv/df_i at (x+m, y), m = -2..2 (dA[0..4]), and at
 * (x, y+m) (dA[5..9]). */
static double adv_limited(const orc_cfg *c, const double *f, const double *gx, const double *gy,
                          int i, int x, int y, double dA[10])
{
    const double lam = c->dt / c->dx;
    const double cv[2] = {g_vx[i] * lam, g_vy[i] * lam};
    double adv = 0.0;
    if (dA) for (int m = 0; m < 10; ++m) dA[m] = 0.0;
    for (int ax = 0; ax < 2; ++ax) {
        double v[5];                       /* f at offsets -2..2 along the axis */
        for (int m = -2; m <= 2; ++m)
            v[m + 2] = ax == 0 ? fat(c, f, gx, gy, i, x + m, y) : fat(c, f, gx, gy, i, x, y + m);
        double dp[4], dm[4];
        const double Fp = face_flux(c->advection, cv[ax], v[1], v[2], v[3], v[4], dp);  /* face +1/2 */
        const double Fm = face_flux(c->advection, cv[ax], v[0], v[1], v[2], v[3], dm);  /* face -1/2 */
        adv += -(Fp - Fm);
        if (dA)
            for (int q = 0; q < 4; ++q) {
                dA[5 * ax + q + 1] -= dp[q];
                dA[5 * ax + q] += dm[q];
            }
    }
    return adv;
}

/* f^{n+1} from f^n.  For every cell and every velocity i (Eq. 3 with
 * forward Euler in time and Lax-Wendroff in space; ORC_ADV_LW2D adds the
 * mixed term (c_x c_y / 4)(f_{++} - f_{+-} - f_{-+} + f_{--}), the flux-limited
 * variants take Adv_i = adv_limited instead):
 *   fhat = M f                          (moments, Appendix rows)
 *   fhat^eq from rho, jx, jy, e          (Appendix equilibria)
 *   Omega_i = -sum_k Minv_ik s_k (fhat_k - fhat^eq_k)
 *   Adv_i = sum_{a in x,y} [ -(c/2)(f_+ - f_-) + (c^2/2)(f_+ - 2 f + f_-) ],
 *           c = v_ia dt/dx, f_+- the neighbours at +-1 along a
 *   f_i^{n+1} = f_i + Adv_i + dt Omega_i
 * gx/gy are the fixed-equilibrium ghosts (ignored on periodic axes). */
static void step_lwfull(const orc_cfg *c, const double *f, const double *gx, const double *gy,
                        double *fnew);

void orc_step(const orc_cfg *c, const double *f, const double *gx, const double *gy,
              double *fnew)
{
    ensure_model();
    if (c->advection == ORC_ADV_LWFULL) {
        step_lwfull(c, f, gx, gy, fnew);
        return;
    }
    const int nx = c->nx, ny = c->ny;
    const size_t n = (size_t)nx * (size_t)ny;
    const double lam = c->dt / c->dx;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double fl[NV], fh[NV], fe[NV], om[NV];
            for (int i = 0; i < NV; ++i) fl[i] = f[(size_t)i * n + (size_t)y * nx + x];
            for (int k = 0; k < NV; ++k) {
                double acc = 0.0;
                for (int i = 0; i < NV; ++i) acc += g_M[k * NV + i] * fl[i];
                fh[k] = acc;
            }
            orc_feq_moments(fh[0], fh[1], fh[2], fh[3], c->b, fe);
            double delta[NV];
            for (int k = 0; k < NV; ++k) delta[k] = c->s[k] * (fh[k] - fe[k]);
            for (int i = 0; i < NV; ++i) {
                double acc = 0.0;
                for (int k = 0; k < NV; ++k) acc += g_Minv[i * NV + k] * delta[k];
                om[i] = -acc;
            }
            for (int i = 0; i < NV; ++i) {
                const double f0 = fl[i];
                if (c->advection == ORC_ADV_MINMOD || c->advection == ORC_ADV_VANLEER) {
                    const double adv = adv_limited(c, f, gx, gy, i, x, y, NULL);
                    fnew[(size_t)i * n + (size_t)y * nx + x] = f0 + adv + c->dt * om[i];
                    continue;
                }
                const double cx = g_vx[i] * lam, cy = g_vy[i] * lam;
                const double fxp = fat(c, f, gx, gy, i, x + 1, y);
                const double fxm = fat(c, f, gx, gy, i, x - 1, y);
                const double fyp = fat(c, f, gx, gy, i, x, y + 1);
                const double fym = fat(c, f, gx, gy, i, x, y - 1);
                const double adv_x = -0.5 * cx * (fxp - fxm) + 0.5 * cx * cx * (fxp - 2.0 * f0 + fxm);
                const double adv_y = -0.5 * cy * (fyp - fym) + 0.5 * cy * cy * (fyp - 2.0 * f0 + fym);
                double adv_xy = 0.0;
                if (c->advection == ORC_ADV_LW2D && cx != 0.0 && cy != 0.0)
                    adv_xy = 0.25 * cx * cy * (fat(c, f, gx, gy, i, x + 1, y + 1) - fat(c, f, gx, gy, i, x + 1, y - 1)
                                               - fat(c, f, gx, gy, i, x - 1, y + 1) + fat(c, f, gx, gy, i, x - 1, y - 1));
                fnew[(size_t)i * n + (size_t)y * nx + x] = f0 + adv_x + adv_y + adv_xy + c->dt * om[i];
            }
        }
    }
}

/* nsteps steps from f in place; work holds one more f (16*nx*ny doubles). */
void orc_run(const orc_cfg *c, double *f, const double *gx, const double *gy,
             long nsteps, double *work)
{
    const size_t bytes = sizeof(double) * NV * (size_t)c->nx * (size_t)c->ny;
    double *a = f, *bb = work;
    for (long s = 0; s < nsteps; ++s) {
        orc_step(c, a, gx, gy, bb);
        double *t = a; a = bb; bb = t;
    }
    if (a != f) memcpy(f, a, bytes);
}

/* ------------------------------------------------------------------------ */
/* Macroscopic fields and conserved totals.                                 */
/* ------------------------------------------------------------------------ */

/* rho = fhat_1, u = j/rho, T = (e - j^2/rho)/(b rho R) (Eq. 12 text). */
void orc_macro(int nx, int ny, double b, const double *f, double *rho, double *ux,
               double *uy, double *T)
{
    ensure_model();
    const size_t n = (size_t)nx * (size_t)ny;
    for (size_t c = 0; c < n; ++c) {
        double m[4] = {0, 0, 0, 0};
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < NV; ++i) m[k] += g_M[k * NV + i] * f[(size_t)i * n + c];
        rho[c] = m[0];
        ux[c] = m[1] / m[0];
        uy[c] = m[2] / m[0];
        T[c] = (m[3] - (m[1] * m[1] + m[2] * m[2]) / m[0]) / (b * m[0]);
    }
}

/* Pairwise (recursive halving) summation of v[0..n-1]. */
static double pairwise_sum(const double *v, size_t n)
{
    if (n <= 8) {
        double s = 0.0;
        for (size_t i = 0; i < n; ++i) s += v[i];
        return s;
    }
    const size_t h = n / 2;
    return pairwise_sum(v, h) + pairwise_sum(v + h, n - h);
}

/* Conserved totals sum over cells of (rho, jx, jy, e) times dx*dy: the four
 * collision invariants fhat_1..fhat_4 (Sect. "Construction ...": density,
 * momentum and energy are conserved by the collision). */
void orc_totals(int nx, int ny, double dx, const double *f, double out[4])
{
    ensure_model();
    const size_t n = (size_t)nx * (size_t)ny;
    double *q = (double *)malloc(sizeof(double) * n);
    if (!q) { out[0] = out[1] = out[2] = out[3] = NAN; return; }
    for (int k = 0; k < 4; ++k) {
        for (size_t c = 0; c < n; ++c) {
            double acc = 0.0;
            for (int i = 0; i < NV; ++i) acc += g_M[k * NV + i] * f[(size_t)i * n + c];
            q[c] = acc;
        }
        out[k] = pairwise_sum(q, n) * dx * dx;
    }
    free(q);
}

/* Thread control for the OpenMP loops (1 = serial). */
void orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Reverse mode (adjoint) of the step, for gradients of a loss of f^N.      */
/* ------------------------------------------------------------------------ */
#include <complex.h>

/* fhat^eq (Appendix) in complex arithmetic, for complex-step derivatives
 * (Squire and Trapp's method: for an analytic g, g'(x) = Im g(x + i h)/h
 * with no subtractive cancellation).  Same formulas as orc_feq_moments. */
static void feq_moments_cplx(double complex rho, double complex jx, double complex jy,
                             double complex e, double b, double complex out[NV])
{
    const double R = 1.0;
    const double complex j2 = jx * jx + jy * jy;
    const double complex P = (e - j2 / rho) / b;
    const double complex T = P / (rho * R);
    const double complex dj = jx * jx - jy * jy;
    out[0] = rho;
    out[1] = jx;
    out[2] = jy;
    out[3] = e;
    out[4] = 2.0 * P + j2 / rho;
    out[5] = dj / rho;
    out[6] = jx * jy / rho;
    out[7] = (e + 2.0 * P) * jx / rho;
    out[8] = (e + 2.0 * P) * jy / rho;
    out[9] = (4.0 * P + jx * jx / rho + jy * jy / rho) * jx / rho;
    out[10] = (4.0 * P + jx * jx / rho + jy * jy / rho) * jy / rho;
    out[11] = (2.0 * P + jx * jx / rho - jy * jy / rho) * jx / rho;
    out[12] = (-2.0 * P + jx * jx / rho - jy * jy / rho) * jy / rho;
    out[13] = 2.0 * (b + 2.0) * rho * R * R * T * T
            + (6.0 + b) * R * T * j2 / rho
            + j2 * j2 / (rho * rho * rho);
    out[14] = ((b + 4.0) * P + j2 / rho) * jx * jy / (rho * rho);
    out[15] = ((b + 4.0) * P + j2 / rho) * dj / (rho * rho);
}

/* J[k*4 + j] = d fhat^eq_k / d m_j for m = (rho, jx, jy, e), by complex step. */
void orc_feq_jacobian(double rho, double jx, double jy, double e, double b, double J[NV * 4])
{
    const double h = 1e-30;
    for (int j = 0; j < 4; ++j) {
        double complex m[4] = {rho, jx, jy, e};
        m[j] += I * h;
        double complex out[NV];
        feq_moments_cplx(m[0], m[1], m[2], m[3], b, out);
        for (int k = 0; k < NV; ++k) J[k * 4 + j] = cimag(out[k]) / h;
    }
}

/* Collision term of Eq. 3 for one cell's 16 values:
 * Omega = -Minv S (M f - fhat^eq(M f)). */
static void collision(const orc_cfg *c, const double fl[NV], double om[NV])
{
    double fh[NV], fe[NV], delta[NV];
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        for (int i = 0; i < NV; ++i) acc += g_M[k * NV + i] * fl[i];
        fh[k] = acc;
    }
    orc_feq_moments(fh[0], fh[1], fh[2], fh[3], c->b, fe);
    for (int k = 0; k < NV; ++k) delta[k] = c->s[k] * (fh[k] - fe[k]);
    for (int i = 0; i < NV; ++i) {
        double acc = 0.0;
        for (int k = 0; k < NV; ++k) acc += g_Minv[i * NV + k] * delta[k];
        om[i] = -acc;
    }
}

/* J w = (dOmega/df) w at f, by a complex step: Omega is analytic in f, and
 * Im Omega(f + i h w) / h = J w with no subtractive cancellation. */
static void collision_dir(const orc_cfg *c, const double fl[NV], const double w[NV], double Jw[NV])
{
    const double h = 1e-30;
    double complex fh[NV], fe[NV], delta[NV];
    for (int k = 0; k < NV; ++k) {
        double complex acc = 0.0;
        for (int i = 0; i < NV; ++i) acc += g_M[k * NV + i] * (fl[i] + I * h * w[i]);
        fh[k] = acc;
    }
    feq_moments_cplx(fh[0], fh[1], fh[2], fh[3], c->b, fe);
    for (int k = 0; k < NV; ++k) delta[k] = c->s[k] * (fh[k] - fe[k]);
    for (int i = 0; i < NV; ++i) {
        double complex acc = 0.0;
        for (int k = 0; k < NV; ++k) acc += g_Minv[i * NV + k] * delta[k];
        Jw[i] = -cimag(acc) / h;
    }
}

/* One ORC_ADV_LWFULL step (see the enum): per cell and velocity i, with
 * c_a = v_ia dt/dx, the neighbours' Omega computed from their own f (the
 * ghosts' f on fixed and wall sides, as every read goes through fat), and
 * w = dt (-v.grad f + Omega) at the cell:
 *   f_i^{n+1} = f_i + [the ORC_ADV_LW2D advection of f_i] + dt Omega_i
 *             - (dt/4) [c_x (Omega_i(x+1) - Omega_i(x-1)) + c_y (Omega_i(y+1) - Omega_i(y-1))]
 *             + (dt/2) (J w)_i. */
static void step_lwfull(const orc_cfg *c, const double *f, const double *gx, const double *gy,
                        double *fnew)
{
    const int nx = c->nx, ny = c->ny;
    const size_t n = (size_t)nx * (size_t)ny;
    const double lam = c->dt / c->dx;
    static const int off[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double fl[NV], om[NV], fn[4][NV], omn[4][NV], w[NV], Jw[NV];
            for (int i = 0; i < NV; ++i) fl[i] = f[(size_t)i * n + (size_t)y * nx + x];
            collision(c, fl, om);
            for (int q = 0; q < 4; ++q) {
                for (int i = 0; i < NV; ++i) fn[q][i] = fat(c, f, gx, gy, i, x + off[q][0], y + off[q][1]);
                collision(c, fn[q], omn[q]);
            }
            for (int i = 0; i < NV; ++i) {
                const double cx = g_vx[i] * lam, cy = g_vy[i] * lam;
                w[i] = -0.5 * cx * (fn[0][i] - fn[1][i]) - 0.5 * cy * (fn[2][i] - fn[3][i]) + c->dt * om[i];
            }
            collision_dir(c, fl, w, Jw);
            for (int i = 0; i < NV; ++i) {
                const double f0 = fl[i];
                const double cx = g_vx[i] * lam, cy = g_vy[i] * lam;
                const double fxp = fn[0][i], fxm = fn[1][i], fyp = fn[2][i], fym = fn[3][i];
                const double adv_x = -0.5 * cx * (fxp - fxm) + 0.5 * cx * cx * (fxp - 2.0 * f0 + fxm);
                const double adv_y = -0.5 * cy * (fyp - fym) + 0.5 * cy * cy * (fyp - 2.0 * f0 + fym);
                double adv_xy = 0.0;
                if (cx != 0.0 && cy != 0.0)
                    adv_xy = 0.25 * cx * cy * (fat(c, f, gx, gy, i, x + 1, y + 1) - fat(c, f, gx, gy, i, x + 1, y - 1)
                                               - fat(c, f, gx, gy, i, x - 1, y + 1) + fat(c, f, gx, gy, i, x - 1, y - 1));
                const double src = c->dt * om[i]
                                 - 0.25 * c->dt * (cx * (omn[0][i] - omn[1][i]) + cy * (omn[2][i] - omn[3][i]))
                                 + 0.5 * c->dt * Jw[i];
                fnew[(size_t)i * n + (size_t)y * nx + x] = f0 + adv_x + adv_y + adv_xy + src;
            }
        }
    }
}

/* Real part of the complex-arithmetic equilibria (consistency check). */
void orc_feq_moments_via_cplx(double rho, double jx, double jy, double e, double b, double out[NV])
{
    double complex o[NV];
    feq_moments_cplx(rho, jx, jy, e, b, o);
    for (int k = 0; k < NV; ++k) out[k] = creal(o[k]);
}

/* Add v at (x, y) of plane i to the adjoint of the value read there: the
 * transpose of fat, with the same mapping of each axis (a domain cell, a
 * wrapped cell, the mirrored cell behind a reflecting wall, or a fixed
 * ghost whose adjoint is accumulated in gxb / gyb, same layout as gx / gy). */
static void scatter(const orc_cfg *c, double *lam, double *gxb, double *gyb, int i, int x, int y,
                    double v)
{
    const int nx = c->nx, ny = c->ny;
    const size_t n = (size_t)nx * (size_t)ny;
    int side_x = -1, side_y = -1;
    if (x < 0 || x >= nx) {
        if (c->bc_x == ORC_BC_PERIODIC) {
            x = ((x % nx) + nx) % nx;
        } else if (c->bc_x == ORC_BC_REFLECT_FIXED && x < 0) {
            i = mirror_index(i, 0);
            x = -x - 1;
        } else {
            side_x = (x < 0) ? 0 : 1;
            x = (x < 0) ? 0 : nx - 1;
        }
    }
    if (y < 0 || y >= ny) {
        if (c->bc_y == ORC_BC_PERIODIC) {
            y = ((y % ny) + ny) % ny;
        } else if (c->bc_y == ORC_BC_REFLECT_FIXED && y < 0) {
            i = mirror_index(i, 1);
            y = -y - 1;
        } else {
            side_y = (y < 0) ? 0 : 1;
            y = (y < 0) ? 0 : ny - 1;
        }
    }
    if (side_x >= 0) { gxb[((size_t)i * 2 + side_x) * ny + y] += v; return; }
    if (side_y >= 0) { gyb[((size_t)i * 2 + side_y) * nx + x] += v; return; }
    lam[(size_t)i * n + (size_t)y * nx + x] += v;
}

/* Transpose of one step.  With f^{n+1} = step(f^n) as in orc_step and
 * lam_next = dL/df^{n+1}, writes lam = dL/df^n (the contribution through
 * this step), adds dL/d(ghost) to gxb / gyb (fixed-equilibrium axes) and
 * adds dL/ds_k to gs[k].  Every forward dependence is transposed literally:
 *   f^{n+1}_i(x) = f_i(x) + sum over the LW stencil + dt Omega_i(f(x)),
 *   dt Omega = -dt Minv S (M f - E(M f)),
 *   d(dt Omega)/df = -dt Minv S (I - JE) M,  JE = d fhat^eq / d fhat
 *                                               (non-zero in columns 1..4),
 *   d f^{n+1}_i/d s_k = -dt Minv_ik (fhat_k - fhat^eq_k).
 * With ORC_ADV_LW2D the mixed term is scattered to the four diagonal
 * neighbours.  In a flux-limited variant the advection part is transposed from the
 * derivatives of adv_limited, which reads the forward ghosts gx_fwd / gy_fwd
 * (the limiter's branch depends on them); at a kink the branch the forward
 * step takes supplies the derivative (a subgradient).
 * Serial (the scatter form writes to neighbours). */
void orc_step_adjoint(const orc_cfg *c, const double *f, const double *gx_fwd, const double *gy_fwd,
                      const double *lam_next, double *lam, double *gxb, double *gyb, double gs[NV])
{
    ensure_model();
    const int nx = c->nx, ny = c->ny;
    const size_t n = (size_t)nx * (size_t)ny;
    const double lam_r = c->dt / c->dx;
    memset(lam, 0, sizeof(double) * NV * n);
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double fl[NV], ln[NV], fh[NV], fe[NV], mu[NV], w[NV], J[NV * 4];
            for (int i = 0; i < NV; ++i) {
                fl[i] = f[(size_t)i * n + (size_t)y * nx + x];
                ln[i] = lam_next[(size_t)i * n + (size_t)y * nx + x];
            }
            /* advection and identity: scatter to the cells the output read */
            for (int i = 0; i < NV; ++i) {
                if (c->advection == ORC_ADV_MINMOD || c->advection == ORC_ADV_VANLEER) {
                    /* flux-limited variant: the local derivatives of Adv_i
                     * (subgradients at the limiter's kinks) */
                    double dA[10];
                    adv_limited(c, f, gx_fwd, gy_fwd, i, x, y, dA);
                    scatter(c, lam, gxb, gyb, i, x, y, ln[i]);
                    for (int m = -2; m <= 2; ++m) {
                        scatter(c, lam, gxb, gyb, i, x + m, y, dA[m + 2] * ln[i]);
                        scatter(c, lam, gxb, gyb, i, x, y + m, dA[5 + m + 2] * ln[i]);
                    }
                    continue;
                }
                const double cx = g_vx[i] * lam_r, cy = g_vy[i] * lam_r;
                /* f_new = f0 + ax_m f(x-1) + ax_p f(x+1) + (-cx^2) f0 + (same in y) */
                const double am_x = 0.5 * cx + 0.5 * cx * cx, ap_x = -0.5 * cx + 0.5 * cx * cx;
                const double am_y = 0.5 * cy + 0.5 * cy * cy, ap_y = -0.5 * cy + 0.5 * cy * cy;
                const double a0 = 1.0 - cx * cx - cy * cy;
                scatter(c, lam, gxb, gyb, i, x, y, a0 * ln[i]);
                scatter(c, lam, gxb, gyb, i, x - 1, y, am_x * ln[i]);
                scatter(c, lam, gxb, gyb, i, x + 1, y, ap_x * ln[i]);
                scatter(c, lam, gxb, gyb, i, x, y - 1, am_y * ln[i]);
                scatter(c, lam, gxb, gyb, i, x, y + 1, ap_y * ln[i]);
                if (c->advection == ORC_ADV_LW2D && cx != 0.0 && cy != 0.0) {
                    const double wxy = 0.25 * cx * cy * ln[i];
                    scatter(c, lam, gxb, gyb, i, x + 1, y + 1, wxy);
                    scatter(c, lam, gxb, gyb, i, x + 1, y - 1, -wxy);
                    scatter(c, lam, gxb, gyb, i, x - 1, y + 1, -wxy);
                    scatter(c, lam, gxb, gyb, i, x - 1, y - 1, wxy);
                }
            }
            /* collision, local */
            for (int k = 0; k < NV; ++k) {
                double acc = 0.0;
                for (int i = 0; i < NV; ++i) acc += g_M[k * NV + i] * fl[i];
                fh[k] = acc;
            }
            orc_feq_moments(fh[0], fh[1], fh[2], fh[3], c->b, fe);
            orc_feq_jacobian(fh[0], fh[1], fh[2], fh[3], c->b, J);
            for (int k = 0; k < NV; ++k) {       /* mu = Minv^T lam_next */
                double acc = 0.0;
                for (int i = 0; i < NV; ++i) acc += g_Minv[i * NV + k] * ln[i];
                mu[k] = acc;
            }
            for (int k = 0; k < NV; ++k) gs[k] += -c->dt * mu[k] * (fh[k] - fe[k]);
            /* w = (I - JE)^T S mu, JE[k][j] = J[k*4+j] for j < 4, 0 otherwise */
            for (int j = 0; j < NV; ++j) {
                double acc = c->s[j] * mu[j];
                if (j < 4)
                    for (int k = 0; k < NV; ++k) acc -= J[k * 4 + j] * c->s[k] * mu[k];
                w[j] = acc;
            }
            /* lam += -dt M^T w */
            for (int i = 0; i < NV; ++i) {
                double acc = 0.0;
                for (int j = 0; j < NV; ++j) acc += g_M[j * NV + i] * w[j];
                lam[(size_t)i * n + (size_t)y * nx + x] += -c->dt * acc;
            }
        }
    }
}

/* Transpose of the initial state f^0 = Minv fhat^eq(m(rho, u, T)) with
 * m = (rho, rho ux, rho uy, b rho T + rho (ux^2 + uy^2)): from lam0 =
 * dL/df^0 writes dL/d(rho, ux, uy, T) per cell. */
void orc_init_adjoint(int nx, int ny, double b, const double *rho, const double *ux,
                      const double *uy, const double *T, const double *lam0, double *g_rho,
                      double *g_ux, double *g_uy, double *g_T)
{
    ensure_model();
    const size_t n = (size_t)nx * (size_t)ny;
    for (size_t cidx = 0; cidx < n; ++cidx) {
        const double r = rho[cidx], u = ux[cidx], v = uy[cidx], t = T[cidx];
        const double m[4] = {r, r * u, r * v, b * r * t + r * (u * u + v * v)};
        double J[NV * 4], mu[NV], mb[4];
        orc_feq_jacobian(m[0], m[1], m[2], m[3], b, J);
        for (int k = 0; k < NV; ++k) {
            double acc = 0.0;
            for (int i = 0; i < NV; ++i) acc += g_Minv[i * NV + k] * lam0[(size_t)i * n + cidx];
            mu[k] = acc;
        }
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int k = 0; k < NV; ++k) acc += J[k * 4 + j] * mu[k];
            mb[j] = acc;
        }
        /* dm/d(rho, u, v, T) */
        g_rho[cidx] = mb[0] + mb[1] * u + mb[2] * v + mb[3] * (b * t + u * u + v * v);
        g_ux[cidx] = mb[1] * r + mb[3] * 2.0 * r * u;
        g_uy[cidx] = mb[2] * r + mb[3] * 2.0 * r * v;
        g_T[cidx] = mb[3] * b * r;
    }
}

/* Adjoint of the fixed-equilibrium ghosts: each ghost holds the initial f
 * of its adjacent cell, so its accumulated adjoint adds to lam0 there. */
void orc_ghosts_adjoint(int nx, int ny, int bc_x, int bc_y, const double *gxb, const double *gyb,
                        double *lam0)
{
    const size_t n = (size_t)nx * (size_t)ny;
    for (int i = 0; i < NV; ++i) {
        /* fixed ghosts hold the initial f of the adjacent cell (behind a
         * reflecting wall nothing is accumulated: gxb / gyb stay 0 there) */
        if (bc_x == ORC_BC_FIXED_EQ || bc_x == ORC_BC_REFLECT_FIXED)
            for (int y = 0; y < ny; ++y) {
                lam0[(size_t)i * n + (size_t)y * nx + 0] += gxb[((size_t)i * 2 + 0) * ny + y];
                lam0[(size_t)i * n + (size_t)y * nx + (nx - 1)] += gxb[((size_t)i * 2 + 1) * ny + y];
            }
        if (bc_y == ORC_BC_FIXED_EQ || bc_y == ORC_BC_REFLECT_FIXED)
            for (int x = 0; x < nx; ++x) {
                lam0[(size_t)i * n + 0 * (size_t)nx + x] += gyb[((size_t)i * 2 + 0) * nx + x];
                lam0[(size_t)i * n + (size_t)(ny - 1) * nx + x] += gyb[((size_t)i * 2 + 1) * nx + x];
            }
    }
}
