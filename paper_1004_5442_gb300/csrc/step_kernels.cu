// step_kernels.cu - the fused MRT-FDLB time step (Eq. 3: moments, relaxation
// toward the Appendix equilibria, inverse transform, Lax-Wendroff advection
// and forward-Euler update in one pass over the state).
//
// Two kernels compute the same cell update (model.cuh):
//
//  * step_tma: CTAs of TMA_W = 128 threads work on strips of 128 columns.
//    One elected thread streams the rows of all 16 planes (plus a 16-byte
//    halo on each side for the x neighbours) from HBM into a ring of shared
//    memory slots with 3-D cp.async.bulk.tensor loads completing on
//    mbarriers; every thread computes one cell per row from rows r-1, r, r+1
//    of the ring (step_strip.cuh).  The 16 outputs of a row go either
//    straight to global memory (one coalesced store per plane and thread) or
//    into a shared-memory row that the elected thread writes back with one
//    3-D TMA store.  Static tiles give each CTA one chunk of rows of one
//    strip; work-queue tiles let one wave of resident CTAs take (row band,
//    strip) items from an atomic counter, row band by row band, so that the
//    items in flight share their boundary rows and halo columns through L2.
//    DRAM reads measure 5-10 % above the 16 per cell of the algorithm.
//  * step_direct: one thread per cell reading its stencil from global memory;
//    used for small FP64 grids (its small blocks spread over more SMs) and
//    for cross-checks.
//
// Both optionally accumulate the conserved totals (rho, jx, jy, e) of the
// output state: FP32 moments summed per thread with an error-free two-sum
// (FP64 moments in the FP64 instantiation), then one partial per CTA (static
// tiles, FP64 across warps) or per warp of each item (work queue,
// double-float FP32 across lanes), summed by two fixed-order FP64 passes.
#include <cstdint>

#include "internal.h"
#include "step_strip.cuh"
#include "tma.cuh"

namespace mrt {

namespace {

using namespace tma;

// Work-queue form: each resident CTA takes (row band, strip) items from the
// launch's counter; the index of its next item is fetched while the current
// one is processed, into the other of two shared slots (the barriers of an
// item separate a slot's read from its next write).  Totals are reduced per
// warp and item (one partial per warp of each item, without a CTA barrier),
// so the fixed-order final sum does not depend on which CTA took which item.
template <class T, bool TOTALS, int NS, bool TSTORE, bool YWIN, bool XT>
__device__ __forceinline__ void step_queue(const CUtensorMap* map_in, const CUtensorMap* map_out,
                                           const StepArgs<T>& a, unsigned char* smem_raw) {
    __shared__ int s_item[2];
    const Layout& L = a.L;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.next[a.parity ^ 1] = 0u;
    if (threadIdx.x == 0) s_item[0] = (int)atomicAdd(&a.next[a.parity], 1u);
    __syncthreads();
    int cur = s_item[0];
    if (cur >= a.nitems) return;
    StripRing<T> R = strip_ring_init<T, NS, TSTORE>(smem_raw);
    for (int k = 1; cur < a.nitems; ++k) {
        if (threadIdx.x == 0) s_item[k & 1] = (int)atomicAdd(&a.next[a.parity], 1u);
        const int band = cur / a.strips;
        const int x0 = (cur - band * a.strips) * TMA_W;
        const int y0 = band * a.rows_per_cta;
        const int nrows = min(a.rows_per_cta, L.ny - y0);
        bool bad = false;
        Acc<T> acc[4];
        if (!strip_chunk<T, TOTALS, NS, TSTORE, YWIN, XT>(R, map_in, map_out, L, a.per_x, a.per_y, a.out, a.k, x0,
                                                          y0, nrows, bad, acc)) {
            strip_drain<T, NS>(R, a.flag);
            return;
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.flag, FLAG_UNSTABLE);
        if (TOTALS) warp_sum4(acc, a.partials + 4 * ((size_t)cur * (TMA_W / 32) + (threadIdx.x >> 5)));
        cur = s_item[k & 1];
    }
}

template <class T, bool TOTALS, int NS, bool TSTORE, int MINB, bool YWIN, bool QUEUE, bool XT>
__global__ void __launch_bounds__(TMA_W, MINB) step_tma(const __grid_constant__ CUtensorMap map_in,
                                                        const __grid_constant__ CUtensorMap map_out,
                                                        const StepArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (QUEUE) {
        step_queue<T, TOTALS, NS, TSTORE, YWIN, XT>(&map_in, &map_out, a, smem_raw);
        return;
    }
    const Layout& L = a.L;
    const int x0 = blockIdx.x * TMA_W;
    const int y0 = blockIdx.y * a.rows_per_cta;
    const int nrows = min(a.rows_per_cta, L.ny - y0);
    if (nrows <= 0) return;  // whole CTA leaves together
    StripRing<T> R = strip_ring_init<T, NS, TSTORE>(smem_raw);
    bool bad = false;
    Acc<T> acc[4];
    if (!strip_chunk<T, TOTALS, NS, TSTORE, YWIN, XT>(R, &map_in, &map_out, L, a.per_x, a.per_y, a.out, a.k, x0,
                                                      y0, nrows, bad, acc)) {
        strip_drain<T, NS>(R, a.flag);
        return;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.flag, FLAG_UNSTABLE);
    if (TOTALS) {
        double v[4] = {acc[0].value(), acc[1].value(), acc[2].value(), acc[3].value()};
        block_sum4(v, a.partials + 4 * (size_t)(blockIdx.y * gridDim.x + blockIdx.x));
    }
}

// --------------------------------------------------------------------------
// One thread per cell, stencil straight from global memory.
// --------------------------------------------------------------------------
constexpr int DIR_BX = 32;
// Block height: the tallest of 8, 4, 2, 1 rows that still gives this many
// blocks (two per SM), so that small grids spread over the SMs; this matters
// most in FP64, where one SM retires only two FP64 lanes per clock.
constexpr long kDirectMinBlocks = 304;

template <class T, bool TOTALS, int BY, bool XT>
__global__ void __launch_bounds__(DIR_BX* BY) step_direct(const StepArgs<T> a) {
    const Layout& L = a.L;
    const int x = blockIdx.x * DIR_BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    const bool active = x < L.nx && y < L.ny;
    bool bad = false;
    T q[4] = {0, 0, 0, 0};
    if (active) {
        const T* __restrict__ in = a.in;
        const long base = (long)(y + 1) * L.pitch + L.G + x;
        auto F = [&](int i, int pos) -> T {
            const long o = i * L.plane + base;
            switch (pos) {
                case C: return __ldg(in + o);
                case XM: return __ldg(in + o - 1);
                case XP: return __ldg(in + o + 1);
                case YM: return __ldg(in + o - L.pitch);
                case YP: return __ldg(in + o + L.pitch);
                case XPYP: return __ldg(in + o + L.pitch + 1);
                case XPYM: return __ldg(in + o - L.pitch + 1);
                case XMYP: return __ldg(in + o + L.pitch - 1);
                default: return __ldg(in + o - L.pitch - 1);
            }
        };
        T out[NV];
        T rho, P;
        cell_update<T, XT>(F, a.k, out, rho, P);
        bad = !healthy(rho, P);
        store_cell<T>(a.out, L, a.per_x, a.per_y, x, y, out);
        if (XT) store_corners<T>(a.out, L, a.per_x, a.per_y, x, y, [&](int j) { return out[j]; });
        if (TOTALS) conserved_moments<T>(out, q[0], q[1], q[2], q[3]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(a.flag, FLAG_UNSTABLE);
    if (TOTALS) {
        double v[4] = {(double)q[0], (double)q[1], (double)q[2], (double)q[3]};
        block_sum4(v, a.partials + 4 * (size_t)(blockIdx.y * gridDim.x + blockIdx.x));
    }
}

// --------------------------------------------------------------------------
// Four warps per 32-cell row segment, one per velocity group: for grids too
// small to fill the SMs with one cell per thread, where one warp per SM
// would wait out the dependent latency of a whole cell update alone.  The
// phases of cell_update run split across the warps, bit for bit the same
// arithmetic: warp g reads the stencil of group g and forms its butterfly
// sums; the warps take one block of moment rows each; every warp forms the
// closure and the relaxed residuals of its block; each warp applies the
// inverse and the Lax-Wendroff update to its own four velocities.  Shared
// memory carries the sums, moments and residuals between the phases.
// --------------------------------------------------------------------------
constexpr int SPLIT_W = 32;

// Store a group's four outputs of cell (x, y) and the ghost copies the next
// step reads (the four-plane form of store_cell: a velocity's mirror image
// lies in its own group).
template <class T>
__device__ __forceinline__ void store_group(T* __restrict__ out, const Layout& L, int per_x, int per_y, int x,
                                            int y, int g, const T og[4]) {
    const long row = (long)(y + 1) * L.pitch;
    const long col = L.G + x;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const long pl = (long)(4 * g + j) * L.plane;
        out[pl + row + col] = og[j];
        if (per_x && x == 0) out[pl + row + L.G + L.nx] = og[j];
        if (per_x && x == L.nx - 1) out[pl + row + L.G - 1] = og[j];
        if (per_y && y == 0) out[pl + (long)(L.ny + 1) * L.pitch + col] = og[j];
        if (per_y && y == L.ny - 1) out[pl + col] = og[j];
        if (L.refl_x && x == 0) out[pl + row + L.G - 1] = og[mirror_plane(4 * g + j, 0) - 4 * g];
        if (L.refl_y && y == 0) out[pl + col] = og[mirror_plane(4 * g + j, 1) - 4 * g];
    }
}

template <class T, bool TOTALS, bool XT, int G>
__device__ __forceinline__ void split_output(const StepArgs<T>& a, const T (&v)[4][9], const Deltas<T>& D, int x,
                                             int y, T og[4]) {
    const T fg[4] = {v[0][C], v[1][C], v[2][C], v[3][C]};
    auto F = [&](int i, int pos) -> T { return v[i - 4 * G][pos]; };
    group_update<T, XT>(G, F, a.k, D, fg, og);
    store_group<T>(a.out, a.L, a.per_x, a.per_y, x, y, G, og);
    if (XT && G >= 2)   // the unsplit operator reads corner ghosts of the diagonal planes only
        store_corners<T>(a.out, a.L, a.per_x, a.per_y, x, y, [&](int j) { return og[j - 4 * G]; }, 4 * G,
                         4 * G + 4);
}

// Shared memory of one split tile.
template <class T>
struct SplitSmem {
    T sum[4][4][SPLIT_W];   // [S, QX, Dx, Dy][group][cell]
    T m[4][4][SPLIT_W];     // [block S, Dx, Dy, Q][row][cell]
    T d[12][SPLIT_W];       // Delta_5 .. Delta_16 (-Delta_13)
    T out[NV][SPLIT_W];     // a totals step's outputs
};

// State loads of the split kernels: through the read-only path when the
// launch only reads the buffer, through L2 alone (ld.global.cg) in the
// multi-step kernel, where the buffer a step reads was written by other
// blocks earlier in the same launch.
template <bool COHERENT, class T>
__device__ __forceinline__ T split_load(const T* p) {
    if constexpr (COHERENT) return __ldcg(p); else return __ldg(p);
}

// One tile of a split kernel: 32 cells of row y from column x0, four warps
// (threadIdx.y = velocity group g).  Returns through bad the health check
// of the tile's cells and, with TOTALS, writes the tile's FP64 totals
// partial to partial[0..3].
template <class T, bool TOTALS, bool XT, bool COHERENT>
__device__ __forceinline__ void split_tile(const StepArgs<T>& a, int x0, int y, SplitSmem<T>& sh, bool& bad,
                                           double* partial) {
    const Layout& L = a.L;
    const int lane = threadIdx.x, g = threadIdx.y;
    const int x = x0 + lane;
    const bool active = x < L.nx;
    // ---- phase 1: group g's stencil and butterfly sums ------------------
    T v[4][9];
    if (active) {
        const T* __restrict__ in = a.in;
        const long base = (long)(y + 1) * L.pitch + L.G + x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T* p = in + (long)(4 * g + j) * L.plane + base;
            v[j][C] = split_load<COHERENT>(p);
            v[j][XM] = split_load<COHERENT>(p - 1);
            v[j][XP] = split_load<COHERENT>(p + 1);
            v[j][YM] = split_load<COHERENT>(p - L.pitch);
            v[j][YP] = split_load<COHERENT>(p + L.pitch);
            if (XT && g >= 2) {
                v[j][XPYP] = split_load<COHERENT>(p + L.pitch + 1);
                v[j][XPYM] = split_load<COHERENT>(p - L.pitch + 1);
                v[j][XMYP] = split_load<COHERENT>(p + L.pitch - 1);
                v[j][XMYM] = split_load<COHERENT>(p - L.pitch - 1);
            }
        }
        const T fg[4] = {v[0][C], v[1][C], v[2][C], v[3][C]};
        const GroupSums<T> gs = group_sums<T>(g, fg);
        sh.sum[0][g][lane] = gs.S;
        sh.sum[1][g][lane] = gs.QX;
        sh.sum[2][g][lane] = gs.Dx;
        sh.sum[3][g][lane] = gs.Dy;
    }
    __syncthreads();
    // ---- phase 2: one block of moment rows per warp ---------------------
    if (active) {
        const int kind = g == 0 ? 0 : g == 1 ? 2 : g == 2 ? 3 : 1;
        const T q[4] = {sh.sum[kind][0][lane], sh.sum[kind][1][lane], sh.sum[kind][2][lane], sh.sum[kind][3][lane]};
        T m[4];
        if (g == 0) moments_S<T>(q, m);
        else if (g < 3) moments_D<T>(q, m);
        else moments_Q<T>(q, m);
#pragma unroll
        for (int r = 0; r < 4; ++r) sh.m[g][r][lane] = m[r];
    }
    __syncthreads();
    // ---- phase 3: closure and the relaxed residuals of the warp's block -
    bad = false;
    if (active) {
        const T rho = sh.m[0][0][lane], e = sh.m[0][2][lane], jx = sh.m[1][0][lane], jy = sh.m[2][0][lane];
        const EqBase<T> b = eq_base<T>(rho, jx, jy, e, a.k);
        Deltas<T> D;
        if (g == 0) {
            relax_S<T>(b, sh.m[0][1][lane], sh.m[0][3][lane], a.k, D);
            sh.d[0][lane] = D.d5;
            sh.d[9][lane] = D.d14;
            bad = !healthy(rho, b.P);
        } else if (g == 1) {
            relax_Dx<T>(b, e, sh.m[1][3][lane], sh.m[1][2][lane], sh.m[1][1][lane], a.k, D);
            sh.d[3][lane] = D.d8;
            sh.d[5][lane] = D.d10;
            sh.d[7][lane] = D.d12;
        } else if (g == 2) {
            relax_Dy<T>(b, e, sh.m[2][3][lane], sh.m[2][2][lane], sh.m[2][1][lane], a.k, D);
            sh.d[4][lane] = D.d9;
            sh.d[6][lane] = D.d11;
            sh.d[8][lane] = D.nd13;
        } else {
            relax_Q<T>(b, jx, sh.m[3][0][lane], sh.m[3][1][lane], sh.m[3][2][lane], sh.m[3][3][lane], a.k, D);
            sh.d[1][lane] = D.d6;
            sh.d[11][lane] = D.d16;
            sh.d[2][lane] = D.d7;
            sh.d[10][lane] = D.d15;
        }
    }
    __syncthreads();
    // ---- phase 4: inverse and Lax-Wendroff update of the warp's group ---
    T og[4] = {0, 0, 0, 0};
    if (active) {
        Deltas<T> D;
        D.d5 = sh.d[0][lane]; D.d6 = sh.d[1][lane]; D.d7 = sh.d[2][lane]; D.d8 = sh.d[3][lane];
        D.d9 = sh.d[4][lane]; D.d10 = sh.d[5][lane]; D.d11 = sh.d[6][lane]; D.d12 = sh.d[7][lane];
        D.nd13 = sh.d[8][lane]; D.d14 = sh.d[9][lane]; D.d15 = sh.d[10][lane]; D.d16 = sh.d[11][lane];
        switch (g) {
            case 0: split_output<T, TOTALS, XT, 0>(a, v, D, x, y, og); break;
            case 1: split_output<T, TOTALS, XT, 1>(a, v, D, x, y, og); break;
            case 2: split_output<T, TOTALS, XT, 2>(a, v, D, x, y, og); break;
            default: split_output<T, TOTALS, XT, 3>(a, v, D, x, y, og); break;
        }
    }
    if (TOTALS) {
        // the cell's conserved moments from all 16 outputs (warp 0), one
        // FP64 partial per tile
#pragma unroll
        for (int j = 0; j < 4; ++j) sh.out[4 * g + j][lane] = og[j];
        __syncthreads();
        T q[4] = {0, 0, 0, 0};
        if (g == 0 && active) {
            T o[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) o[i] = sh.out[i][lane];
            conserved_moments<T>(o, q[0], q[1], q[2], q[3]);
        }
        double w[4] = {(double)q[0], (double)q[1], (double)q[2], (double)q[3]};
        block_sum4(w, partial);
    }
}

template <class T, bool TOTALS, bool XT>
__global__ void __launch_bounds__(4 * SPLIT_W) step_split(const StepArgs<T> a) {
    __shared__ SplitSmem<T> sh;
    bool bad = false;
    split_tile<T, TOTALS, XT, false>(a, blockIdx.x * SPLIT_W, blockIdx.y, sh, bad,
                                     a.partials + 4 * (size_t)(blockIdx.y * gridDim.x + blockIdx.x));
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(a.flag, FLAG_UNSTABLE);
}

// --------------------------------------------------------------------------
// All steps of a call in one cooperative launch of split tiles, for grids so
// small that a kernel launch (about 4 us on this part, in a CUDA graph too)
// costs as much as the step.  Each resident block keeps its tiles for the
// whole run.  A tile publishes the number of steps it has completed
// (release, after the block's stores); before step s it waits (acquire,
// bounded) until every tile it reads from - the up to eight neighbours on
// the 32-cell x 1-row tile grid, wrapped on periodic axes, whose cells and
// ghost copies its radius-1 stencil touches - has completed step s - 1.
// That also orders the step's stores after the neighbours' last reads of the
// buffer being overwritten (it held their step s - 1 input).  A tile is
// never more than one step ahead of a neighbour, every wait is for an
// earlier step, and the cooperative launch keeps every block resident, so
// the waits end; a wait that runs out sets the timeout flag and the block
// returns.
// --------------------------------------------------------------------------
template <class T, bool XT>
__global__ void __launch_bounds__(4 * SPLIT_W) step_split_persist(const StepArgs<T> a, T* buf0, T* buf1, int nsteps,
                                                                  int totals, unsigned* done) {
    __shared__ SplitSmem<T> sh;
    const Layout& L = a.L;
    const int ntx = (L.nx + SPLIT_W - 1) / SPLIT_W;
    const int ntiles = ntx * L.ny;
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    bool bad_any = false;
    for (int s = 0; s < nsteps; ++s) {
        StepArgs<T> as = a;
        as.in = (s & 1) ? buf1 : buf0;
        as.out = (s & 1) ? buf0 : buf1;
        const bool tot = totals && s == nsteps - 1;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int sx = t % ntx, y = t / ntx;
            bool ok = true;
            if (s > 0 && threadIdx.y == 0 && threadIdx.x < 9) {
                // lane k of warp 0 waits for neighbour (dx, dy) = (k % 3 - 1, k / 3 - 1)
                int ny = y + (int)threadIdx.x / 3 - 1, nx = sx + (int)threadIdx.x % 3 - 1;
                bool need = true;
                if (ny < 0 || ny >= L.ny) {
                    need = a.per_y;                    // fixed or wall ghosts: constant or written by this tile
                    ny = (ny + L.ny) % L.ny;
                }
                if (nx < 0 || nx >= ntx) {
                    need = need && a.per_x;
                    nx = (nx + ntx) % ntx;
                }
                const int n = ny * ntx + nx;
                if (need && n != t) ok = wait_at_least(done + n, (unsigned)s);
            }
            if (!__syncthreads_and(ok)) {
                if (lead) atomicOr(a.flag, FLAG_TIMEOUT);
                return;
            }
            bool bad = false;
            double* part = a.partials + 4 * (size_t)t;
            if (tot) split_tile<T, true, XT, true>(as, sx * SPLIT_W, y, sh, bad, part);
            else split_tile<T, false, XT, true>(as, sx * SPLIT_W, y, sh, bad, part);
            bad_any |= bad;
            __syncthreads();   // the tile's stores, before its count is published
            if (lead) st_release(done + t, (unsigned)(s + 1));
        }
    }
    if (__syncthreads_or(bad_any) && lead) atomicOr(a.flag, FLAG_UNSTABLE);
}

template <class T, int NS, bool TSTORE, int MINB, bool YWIN = false, bool QUEUE = false, bool XT = false>
struct TmaKernels {
    static cudaError_t launch(const CUtensorMap* mi, const CUtensorMap* mo, const StepArgs<T>& a, dim3 grid,
                              size_t smem, bool totals, cudaStream_t st) {
        if (totals)
            step_tma<T, true, NS, TSTORE, MINB, YWIN, QUEUE, XT><<<grid, TMA_W, smem, st>>>(*mi, *mo, a);
        else
            step_tma<T, false, NS, TSTORE, MINB, YWIN, QUEUE, XT><<<grid, TMA_W, smem, st>>>(*mi, *mo, a);
        return cudaGetLastError();
    }
    static cudaError_t occupancy(size_t smem, int* occ) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(step_tma<T, true, NS, TSTORE, MINB, YWIN, QUEUE, XT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(step_tma<T, false, NS, TSTORE, MINB, YWIN, QUEUE, XT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, step_tma<T, false, NS, TSTORE, MINB, YWIN, QUEUE, XT>, TMA_W, smem);
    }
};

// FP64 rings are capped at 4 rows (16.9 KB per row).
template <class T, int NS> constexpr int ring_depth() { return sizeof(T) == 8 && NS > 4 ? 4 : NS; }

// The unsplit operator (xt) reads rows r-1 and r+1 at x +- 1: tiles 1, 4
// and 7 keep row r-1 in the ring, tiles 5 and 6 keep its diagonal planes'
// x neighbours in registers.
template <class T, class Fn>
cudaError_t with_tile(int tile, bool xt, Fn&& fn) {
    if (xt) {
        switch (tile) {
            case 1: return fn(TmaKernels<T, ring_depth<T, 6>(), false, 4, false, false, true>());
            case 4: return fn(TmaKernels<T, ring_depth<T, 5>(), true, (sizeof(T) == 8 ? 2 : 3), false, false, true>());
            case 5: return fn(TmaKernels<T, ring_depth<T, 4>(), true, (sizeof(T) == 8 ? 2 : 4), true, false, true>());
            case 6: return fn(TmaKernels<T, ring_depth<T, 4>(), true, (sizeof(T) == 8 ? 2 : 4), true, true, true>());
            case 7: return fn(TmaKernels<T, ring_depth<T, 5>(), true, (sizeof(T) == 8 ? 2 : 3), false, true, true>());
            default: return cudaErrorInvalidValue;
        }
    }
    switch (tile) {
        case 1: return fn(TmaKernels<T, ring_depth<T, 6>(), false, 4>());
        case 2: return fn(TmaKernels<T, ring_depth<T, 4>(), true, (sizeof(T) == 8 ? 2 : 4)>());
        case 3: return fn(TmaKernels<T, ring_depth<T, 6>(), true, (sizeof(T) == 8 ? 2 : 3)>());
        case 4: return fn(TmaKernels<T, ring_depth<T, 5>(), true, (sizeof(T) == 8 ? 2 : 3)>());
        case 5: return fn(TmaKernels<T, ring_depth<T, 4>(), true, (sizeof(T) == 8 ? 2 : 4), true>());
        case 6: return fn(TmaKernels<T, ring_depth<T, 4>(), true, (sizeof(T) == 8 ? 2 : 4), true, true>());
        case 7: return fn(TmaKernels<T, ring_depth<T, 5>(), true, (sizeof(T) == 8 ? 2 : 3), false, true>());
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <class T>
cudaError_t launch_step_tma(int tile, bool xt, const CUtensorMap* map_in, const CUtensorMap* map_out,
                            const StepArgs<T>& a, int grid_x, int grid_y, bool totals, cudaStream_t st) {
    const size_t smem = tma_smem_bytes<T>(tile);
    return with_tile<T>(tile, xt, [&](auto k) {
        return k.launch(map_in, map_out, a, dim3(grid_x, grid_y), smem, totals, st);
    });
}

template <class T>
cudaError_t tma_occupancy(int tile, bool xt, int* blocks_per_sm) {
    const size_t smem = tma_smem_bytes<T>(tile);
    return with_tile<T>(tile, xt, [&](auto k) { return k.occupancy(smem, blocks_per_sm); });
}

template <class T>
void direct_grid(const Layout& L, dim3* grid, dim3* block) {
    const long bx = (L.nx + DIR_BX - 1) / DIR_BX;
    int by = 8;
    while (by > 1 && bx * ((L.ny + by - 1) / by) < kDirectMinBlocks) by /= 2;
    *block = dim3(DIR_BX, by);
    *grid = dim3((unsigned)bx, (L.ny + by - 1) / by);
}

template <class T, int BY, bool XT>
static void launch_direct_by(const StepArgs<T>& a, bool totals, dim3 grid, cudaStream_t st) {
    if (totals)
        step_direct<T, true, BY, XT><<<grid, dim3(DIR_BX, BY), 0, st>>>(a);
    else
        step_direct<T, false, BY, XT><<<grid, dim3(DIR_BX, BY), 0, st>>>(a);
}

template <class T, bool XT>
static void launch_direct_xt(const StepArgs<T>& a, bool totals, dim3 grid, int by, cudaStream_t st) {
    switch (by) {
        case 8: launch_direct_by<T, 8, XT>(a, totals, grid, st); break;
        case 4: launch_direct_by<T, 4, XT>(a, totals, grid, st); break;
        case 2: launch_direct_by<T, 2, XT>(a, totals, grid, st); break;
        default: launch_direct_by<T, 1, XT>(a, totals, grid, st); break;
    }
}

template <class T>
cudaError_t launch_step_direct(const StepArgs<T>& a, bool xt, bool totals, cudaStream_t st) {
    dim3 grid, block;
    direct_grid<T>(a.L, &grid, &block);
    if (xt) launch_direct_xt<T, true>(a, totals, grid, (int)block.y, st);
    else launch_direct_xt<T, false>(a, totals, grid, (int)block.y, st);
    return cudaGetLastError();
}

void split_grid(const Layout& L, dim3* grid, dim3* block) {
    *block = dim3(SPLIT_W, 4);
    *grid = dim3((L.nx + SPLIT_W - 1) / SPLIT_W, L.ny);
}

template <class T>
cudaError_t launch_step_split(const StepArgs<T>& a, bool xt, bool totals, cudaStream_t st) {
    dim3 grid, block;
    split_grid(a.L, &grid, &block);
    if (xt) {
        if (totals) step_split<T, true, true><<<grid, block, 0, st>>>(a);
        else step_split<T, false, true><<<grid, block, 0, st>>>(a);
    } else {
        if (totals) step_split<T, true, false><<<grid, block, 0, st>>>(a);
        else step_split<T, false, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t split_persist_blocks(bool xt, int* blocks) {
    int occ = 0, dev = 0, sms = 0;
    cudaError_t e = xt ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_split_persist<T, true>, 4 * SPLIT_W, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_split_persist<T, false>, 4 * SPLIT_W, 0);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *blocks = occ * sms;
    return cudaSuccess;
}

template <class T>
cudaError_t launch_step_split_persist(const StepArgs<T>& a, bool xt, T* buf0, T* buf1, int nsteps, bool totals,
                                      unsigned* done, int blocks, cudaStream_t st) {
    void* args[] = {(void*)&a, (void*)&buf0, (void*)&buf1, (void*)&nsteps, nullptr, (void*)&done};
    int tot = totals ? 1 : 0;
    args[4] = (void*)&tot;
    const void* fn = xt ? (const void*)step_split_persist<T, true> : (const void*)step_split_persist<T, false>;
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(SPLIT_W, 4), args, 0, st);
}

template cudaError_t split_persist_blocks<float>(bool, int*);
template cudaError_t split_persist_blocks<double>(bool, int*);
template cudaError_t launch_step_split_persist<float>(const StepArgs<float>&, bool, float*, float*, int, bool,
                                                       unsigned*, int, cudaStream_t);
template cudaError_t launch_step_split_persist<double>(const StepArgs<double>&, bool, double*, double*, int, bool,
                                                        unsigned*, int, cudaStream_t);
template cudaError_t launch_step_split<float>(const StepArgs<float>&, bool, bool, cudaStream_t);
template cudaError_t launch_step_split<double>(const StepArgs<double>&, bool, bool, cudaStream_t);
template cudaError_t launch_step_tma<float>(int, bool, const CUtensorMap*, const CUtensorMap*,
                                            const StepArgs<float>&, int, int, bool, cudaStream_t);
template cudaError_t launch_step_tma<double>(int, bool, const CUtensorMap*, const CUtensorMap*,
                                             const StepArgs<double>&, int, int, bool, cudaStream_t);
template cudaError_t launch_step_direct<float>(const StepArgs<float>&, bool, bool, cudaStream_t);
template cudaError_t launch_step_direct<double>(const StepArgs<double>&, bool, bool, cudaStream_t);
template cudaError_t tma_occupancy<float>(int, bool, int*);
template cudaError_t tma_occupancy<double>(int, bool, int*);
template void direct_grid<float>(const Layout&, dim3*, dim3*);
template void direct_grid<double>(const Layout&, dim3*, dim3*);

}  // namespace mrt
