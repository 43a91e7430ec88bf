// adjoint_kernels.cu - kernels of the reverse sweep (gradients of a loss of
// rho_N with respect to the initial fields and the relaxation rates):
//   adjoint_step   dL/df^n from dL/df^{n+1} and f^n (cell_adjoint), with the
//                  rate gradients and the fixed-ghost adjoints accumulated
//   lam_from_drho  dL/df^N = dL/drho_N on every plane (rho = sum_i f_i)
//   ghost_adjoint  adds the accumulated ghost adjoints to their cells
//                  (a fixed ghost holds the initial f of its adjacent cell)
//   init_adjoint   dL/d(rho, u, T) of f^0 = M^-1 fhat^eq(rho, u, T)
//   sum_partials   fixed-order sum of the per-block rate partials
#include "adjoint.cuh"
#include "internal.h"

namespace mrt {
namespace {

constexpr int ABX = 32, ABY = 8;

template <class T, bool STORE_GHOSTS>
__device__ __forceinline__ void store_plain(T* __restrict__ out, const Layout& L, int per_x, int per_y, int x,
                                            int y, const T v[NV]) {
    const long row = (long)(y + 1) * L.pitch;
    const long col = L.G + x;
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i * L.plane + row + col] = v[i];
    if (STORE_GHOSTS) {
        if (per_x && x == 0)
            for (int i = 0; i < NV; ++i) out[i * L.plane + row + L.G + L.nx] = v[i];
        if (per_x && x == L.nx - 1)
            for (int i = 0; i < NV; ++i) out[i * L.plane + row + L.G - 1] = v[i];
        if (per_y && y == 0)
            for (int i = 0; i < NV; ++i) out[i * L.plane + (long)(L.ny + 1) * L.pitch + col] = v[i];
        if (per_y && y == L.ny - 1)
            for (int i = 0; i < NV; ++i) out[i * L.plane + col] = v[i];
    }
}

template <class T>
__global__ void __launch_bounds__(ABX* ABY) adjoint_step_kernel(AdjArgs<T> a) {
    const Layout& L = a.L;
    const int x = blockIdx.x * ABX + threadIdx.x;
    const int y = blockIdx.y * ABY + threadIdx.y;
    T gs[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) gs[j] = 0;
    if (x < L.nx && y < L.ny) {
        const long base = (long)(y + 1) * L.pitch + L.G + x;
        const T* __restrict__ lam = a.lam_in;
        auto LF = [&](int i, int pos) -> T {
            const long o = i * L.plane + base;
            switch (pos) {
                case C: return __ldg(lam + o);
                case XM: return __ldg(lam + o - 1);
                case XP: return __ldg(lam + o + 1);
                case YM: return __ldg(lam + o - L.pitch);
                default: return __ldg(lam + o + L.pitch);
            }
        };
        T f[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) f[i] = __ldg(a.f + i * L.plane + base);
        T out[NV];
        cell_adjoint<T>(LF, f, a.k, out, gs);
        store_plain<T, true>(a.lam_out, L, a.per_x, a.per_y, x, y, out);
        // a fixed ghost beyond an edge cell received the forward weight of
        // that neighbour position; accumulate its adjoint (one writer each)
        if (!a.per_x && (x == 0 || x == L.nx - 1)) {
            const int side = x == 0 ? 0 : 1;
            for (int i = 0; i < NV; ++i) {
                const T wgt = lw_weight<T>(a.k, i, side == 0 ? XM : XP);
                a.gxb[((long)i * 2 + side) * L.ny + y] += (double)(wgt * LF(i, C));
            }
        }
        if (!a.per_y && (y == 0 || y == L.ny - 1)) {
            const int side = y == 0 ? 0 : 1;
            for (int i = 0; i < NV; ++i) {
                const T wgt = lw_weight<T>(a.k, i, side == 0 ? YM : YP);
                a.gyb[((long)i * 2 + side) * L.nx + x] += (double)(wgt * LF(i, C));
            }
        }
    }
    // block sum of the 12 rate partials, accumulated into this block's slot:
    // within a warp in the state precision (32 terms), across warps and steps
    // in FP64
    __shared__ double red[ABX * ABY / 32][12];
    const int t = threadIdx.y * ABX + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        T v = gs[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = (double)v;
    }
    __syncthreads();
    if (t < 12) {
        double s = 0;
        for (int w = 0; w < ABX * ABY / 32; ++w) s += red[w][t];
        a.gpart[(long)(blockIdx.y * gridDim.x + blockIdx.x) * 12 + t] += s;
    }
}

template <class T>
__global__ void lam_from_drho_kernel(Layout L, const double* __restrict__ drho, T* __restrict__ lam) {
    const long n = (long)L.nx * L.ny;
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
        const int x = (int)(c % L.nx), y = (int)(c / L.nx);
        const T v = (T)drho[c];
        for (int i = 0; i < NV; ++i) lam[i * L.plane + (long)(y + 1) * L.pitch + L.G + x] = v;
    }
}

template <class T>
__global__ void ghost_adjoint_kernel(Layout L, int fix_x, int fix_y, const double* __restrict__ gxb,
                                     const double* __restrict__ gyb, T* __restrict__ lam) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    // x ghosts: 16 planes x 2 sides x ny rows; then y ghosts: 16 x 2 x nx
    const long nxg = fix_x ? 32L * L.ny : 0, nyg = fix_y ? 32L * L.nx : 0;
    if (t < nxg) {
        const int i = (int)(t / (2L * L.ny)), side = (int)((t / L.ny) % 2), y = (int)(t % L.ny);
        const int x = side == 0 ? 0 : L.nx - 1;
        T* p = lam + i * L.plane + (long)(y + 1) * L.pitch + L.G + x;
        *p = (T)((double)*p + gxb[t]);
    }
    __syncthreads();  // corners get both contributions in a fixed order (x then y)
    if (t < nyg) {
        const int i = (int)(t / (2L * L.nx)), side = (int)((t / L.nx) % 2), x = (int)(t % L.nx);
        const int y = side == 0 ? 0 : L.ny - 1;
        T* p = lam + i * L.plane + (long)(y + 1) * L.pitch + L.G + x;
        *p = (T)((double)*p + gyb[t]);
    }
}

// dL/d(rho, ux, uy, T) from lam0 = dL/df^0, f^0 = Minv fhat^eq(m), m =
// (rho, rho ux, rho uy, b rho T + rho (ux^2 + uy^2)).  FP64 throughout.
template <class T>
__global__ void init_adjoint_kernel(Layout L, InitCoef ic, Coef<double> kd, const T* __restrict__ lam,
                                    const double* __restrict__ rho, const double* __restrict__ ux,
                                    const double* __restrict__ uy, const double* __restrict__ Tf,
                                    double* g_rho, double* g_ux, double* g_uy, double* g_T) {
    const long n = (long)L.nx * L.ny;
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
        const int x = (int)(c % L.nx), y = (int)(c / L.nx);
        double l[NV];
        for (int i = 0; i < NV; ++i) l[i] = (double)lam[i * L.plane + (long)(y + 1) * L.pitch + L.G + x];
        // Minv = (inverse butterfly) o (block inverse); transpose = scaled
        // butterfly, then the transposed block inverses
        double bS[4], bX[4], bY[4], bQ[4];
        for (int g = 0; g < 4; ++g) {
            const double* v = l + 4 * g;
            const double s02 = v[0] + v[2], s13 = v[1] + v[3], d02 = v[0] - v[2], d13 = v[1] - v[3];
            bS[g] = 0.25 * (s02 + s13);
            bQ[g] = 0.25 * (s02 - s13);
            if (g < 2) { bX[g] = 0.5 * d02; bY[g] = 0.5 * d13; }
            else { bX[g] = 0.25 * (d02 - d13); bY[g] = 0.25 * (d02 + d13); }
        }
        double muA[4], muX[4], muY[4];
        for (int kk = 0; kk < 4; ++kk) {
            muA[kk] = muX[kk] = muY[kk] = 0;
            for (int g = 0; g < 4; ++g) {
                muA[kk] += ic.Ainv[g][kk] * bS[g];
                muX[kk] += ic.Binv[g][kk] * bX[g];
                muY[kk] += ic.Binv[g][kk] * bY[g];
            }
        }
        muY[3] = -muY[3];  // the m13 row of the y block is negated
        const double mu6 = ic.C1inv[0][0] * bQ[0] + ic.C1inv[1][0] * bQ[1];
        const double mu16 = ic.C1inv[0][1] * bQ[0] + ic.C1inv[1][1] * bQ[1];
        const double mu7 = ic.C2inv[0][0] * bQ[2] + ic.C2inv[1][0] * bQ[3];
        const double mu15 = ic.C2inv[0][1] * bQ[2] + ic.C2inv[1][1] * bQ[3];
        // (m1, m4, m5, m14) = muA, (m2, m8, m10, m12) = muX, (m3, m9, m11, m13) = muY
        const double nu[12] = {muA[2], mu6, mu7, muX[1], muY[1], muX[2], muY[2], muX[3], muY[3], muA[3], mu15, mu16};
        const double r = rho[c], u = ux[c], v = uy[c], t = Tf[c];
        const double b = ic.b;
        const double jx = r * u, jy = r * v, e = b * r * t + r * (u * u + v * v);
        double a_r, a_jx, a_jy, a_e;
        adj_equilibrium<double>(r, jx, jy, e, kd, nu, a_r, a_jx, a_jy, a_e);
        const double mb1 = muA[0] + a_r, mb2 = muX[0] + a_jx, mb3 = muY[0] + a_jy, mb4 = muA[1] + a_e;
        g_rho[c] = mb1 + mb2 * u + mb3 * v + mb4 * (b * t + u * u + v * v);
        g_ux[c] = mb2 * r + mb4 * 2.0 * r * u;
        g_uy[c] = mb3 * r + mb4 * 2.0 * r * v;
        g_T[c] = mb4 * b * r;
    }
}

__global__ void sum_partials_kernel(const double* __restrict__ gpart, int nparts, double* out) {
    __shared__ double red[256];
    for (int j = 0; j < 12; ++j) {
        double s = 0;
        for (int p = threadIdx.x; p < nparts; p += 256) s += gpart[(long)p * 12 + j];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[j] = red[0];
        __syncthreads();
    }
}

int blocks_for(long n, int t) {
    long b = (n + t - 1) / t;
    return (int)(b < 1 ? 1 : b > 4096 ? 4096 : b);
}

}  // namespace

template <class T>
void adjoint_grid(const Layout& L, dim3* grid, dim3* block) {
    *block = dim3(ABX, ABY);
    *grid = dim3((L.nx + ABX - 1) / ABX, (L.ny + ABY - 1) / ABY);
}

template <class T>
cudaError_t launch_adjoint_step(const AdjArgs<T>& a, cudaStream_t st) {
    dim3 grid, block;
    adjoint_grid<T>(a.L, &grid, &block);
    adjoint_step_kernel<T><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_lam_from_drho(const Layout& L, const double* drho, T* lam, cudaStream_t st) {
    lam_from_drho_kernel<T><<<blocks_for((long)L.nx * L.ny, 256), 256, 0, st>>>(L, drho, lam);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_ghost_adjoint(const Layout& L, int fix_x, int fix_y, const double* gxb, const double* gyb,
                                 T* lam, cudaStream_t st) {
    const long n = std::max(fix_x ? 32L * L.ny : 0L, fix_y ? 32L * L.nx : 0L);
    if (n == 0) return cudaSuccess;
    // one block covers everything so the x-then-y order holds at corners
    if (n <= 1024) {
        ghost_adjoint_kernel<T><<<1, 1024, 0, st>>>(L, fix_x, fix_y, gxb, gyb, lam);
    } else {
        // large edges: x pass then y pass as separate launches (stream order)
        const int bx = blocks_for(fix_x ? 32L * L.ny : 0L, 256);
        if (fix_x) ghost_adjoint_kernel<T><<<bx, 256, 0, st>>>(L, 1, 0, gxb, gyb, lam);
        const int by = blocks_for(fix_y ? 32L * L.nx : 0L, 256);
        if (fix_y) ghost_adjoint_kernel<T><<<by, 256, 0, st>>>(L, 0, 1, gxb, gyb, lam);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_init_adjoint(const Layout& L, const InitCoef& ic, const Coef<double>& kd, const T* lam,
                                const double* rho, const double* ux, const double* uy, const double* Tf,
                                double* g_rho, double* g_ux, double* g_uy, double* g_T, cudaStream_t st) {
    init_adjoint_kernel<T><<<blocks_for((long)L.nx * L.ny, 256), 256, 0, st>>>(L, ic, kd, lam, rho, ux, uy, Tf,
                                                                              g_rho, g_ux, g_uy, g_T);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* gpart, int nparts, double* out, cudaStream_t st) {
    sum_partials_kernel<<<1, 256, 0, st>>>(gpart, nparts, out);
    return cudaGetLastError();
}

#define INST(T)                                                                                                 \
    template void adjoint_grid<T>(const Layout&, dim3*, dim3*);                                                 \
    template cudaError_t launch_adjoint_step<T>(const AdjArgs<T>&, cudaStream_t);                               \
    template cudaError_t launch_lam_from_drho<T>(const Layout&, const double*, T*, cudaStream_t);               \
    template cudaError_t launch_ghost_adjoint<T>(const Layout&, int, int, const double*, const double*, T*,     \
                                                 cudaStream_t);                                                 \
    template cudaError_t launch_init_adjoint<T>(const Layout&, const InitCoef&, const Coef<double>&, const T*,  \
                                                const double*, const double*, const double*, const double*,     \
                                                double*, double*, double*, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace mrt
