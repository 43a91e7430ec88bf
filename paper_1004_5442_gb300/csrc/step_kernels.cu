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
