// step_kernels.cu - the fused MRT-FDLB time step (Eq. 3: moments, relaxation
// toward the Appendix equilibria, inverse transform, Lax-Wendroff advection
// and forward-Euler update in one pass over the state).
//
// Two kernels compute the same cell update (model.cuh):
//
//  * step_tma: a CTA owns a strip of TMA_W = 128 columns and a chunk of rows.
//    One elected thread streams the rows of all 16 planes (plus a 16-byte
//    halo on each side for the x neighbours) from HBM into a ring of shared
//    memory slots with 3-D cp.async.bulk.tensor loads completing on
//    mbarriers; every thread computes one cell per row from rows r-1, r, r+1
//    of the ring.  The 16 outputs of a row go either straight to global
//    memory (one coalesced store per plane and thread) or into a shared
//    memory row that the elected thread writes back with one 3-D TMA store.
//    Each f value is read from HBM once (halo columns and the two
//    chunk-boundary rows are L2 hits), so the traffic is the 16 reads + 16
//    writes per cell of the algorithm.
//  * step_direct: one thread per cell reading its stencil from global memory;
//    the simple form, used for cross-checks.
//
// Both optionally accumulate the conserved totals (rho, jx, jy, e) of the
// output state: FP32 moments summed per thread with an error-free two-sum
// (FP64 moments in the FP64 instantiation), then reduced per CTA in FP64 and
// written as one block partial; a fixed-order finalise pass sums the partials.
#include <cstdint>

#include "internal.h"
#include "tma.cuh"

namespace mrt {

namespace {

using namespace tma;

// Error-free accumulation of FP32 values into (hi, lo); FP64 sums plainly.
template <class T>
struct Acc {
    T hi = 0, lo = 0;
    __device__ __forceinline__ void add(T v) {
        const T s = hi + v;
        const T bb = s - hi;
        lo += (hi - (s - bb)) + (v - bb);
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <>
struct Acc<double> {
    double hi = 0;
    __device__ __forceinline__ void add(double v) { hi += v; }
    __device__ __forceinline__ double value() const { return hi; }
};

// CTA-wide FP64 sum of 4 values; thread 0 writes them to dst[0..3].
__device__ __forceinline__ void block_sum4(double v[4], double* dst) {
    __shared__ double red[32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0)
        for (int q = 0; q < 4; ++q) red[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; ++q) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += red[w][q];
            dst[q] = s;
        }
    }
}

template <class T>
__device__ __forceinline__ bool healthy(T rho, T P) {
    // false for NaN, non-positive or infinite values
    return rho > (T)0 && P > (T)0 && rho < (T)INFINITY && P < (T)INFINITY;
}

// Store a cell's 16 outputs and, on periodic axes, the ghost copies the next
// step reads (column G-1 mirrors x = nx-1, column G+nx mirrors x = 0; row 0
// mirrors y = ny-1, row ny+1 mirrors y = 0).
template <class T>
__device__ __forceinline__ void store_cell(T* __restrict__ out, const Layout& L, int per_x,
                                           int per_y, int x, int y, const T v[NV]) {
    const long row = (long)(y + 1) * L.pitch;
    const long col = L.G + x;
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i * L.plane + row + col] = v[i];
    if (per_x) {
        if (x == 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i) out[i * L.plane + row + L.G + L.nx] = v[i];
        }
        if (x == L.nx - 1) {
#pragma unroll
            for (int i = 0; i < NV; ++i) out[i * L.plane + row + L.G - 1] = v[i];
        }
    }
    if (per_y) {
        if (y == 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i) out[i * L.plane + (long)(L.ny + 1) * L.pitch + col] = v[i];
        }
        if (y == L.ny - 1) {
#pragma unroll
            for (int i = 0; i < NV; ++i) out[i * L.plane + col] = v[i];
        }
    }
}

// --------------------------------------------------------------------------
// TMA-staged strip kernel.
// --------------------------------------------------------------------------
// YWIN: the 12 planes that move along y keep row r-1 in registers, so only
// rows r and r+1 must be resident and the ring holds NS-2 rows in flight.
template <bool YWIN> __device__ __forceinline__ constexpr bool moves_y(int i) {
    return (i >= 8) || (i & 1);
}

template <class T, bool TOTALS, int NS, bool TSTORE, int MINB, bool YWIN>
__global__ void __launch_bounds__(TMA_W, MINB) step_tma(const __grid_constant__ CUtensorMap map_in,
                                                        const __grid_constant__ CUtensorMap map_out,
                                                        const StepArgs<T> a) {
    constexpr int HALO = tma_halo<T>();
    constexpr int BOXW = tma_boxw<T>();
    constexpr uint32_t SLOT_BYTES = (uint32_t)tma_slot_bytes<T>();
    constexpr uint32_t OUT_BYTES = TSTORE ? (uint32_t)tma_out_slot_bytes<T>() : 0u;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);
    T* outbuf = reinterpret_cast<T*>(smem_raw + NS * SLOT_BYTES);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + NS * SLOT_BYTES + 2 * OUT_BYTES);

    const Layout& L = a.L;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TMA_W;
    const int y0 = blockIdx.y * a.rows_per_cta;
    const int nrows = min(a.rows_per_cta, L.ny - y0);
    if (nrows <= 0) return;  // whole CTA leaves together
    const int nload = nrows + 2;           // local rows 0..nrows+1 = padded rows y0..y0+nrows+1
    const int x = x0 + tid;
    const bool active = x < L.nx;
    const int tma_x = L.G + x0 - HALO;     // 16-byte aligned start column of the load box
    // Row stores by TMA only for whole strips: a TMA store that ends inside a
    // 16-byte chunk can write that whole chunk, which for a ragged last strip
    // holds the right ghost column.  The ragged strip copies its staged row
    // out per thread instead.
    const bool tstore = TSTORE && (x0 + TMA_W <= L.nx);

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();

    int issued = 0;     // thread 0: rows whose load has been issued
    int waited0 = 0;    // thread 0: rows it has seen complete
    if (tid == 0) {
        const int first = min(NS, nload);
        for (int l = 0; l < first; ++l) {
            const int s = l % NS;
            mbar_arrive_expect_tx(&full[s], SLOT_BYTES);
            tma_load_3d(ring + (size_t)s * NV * BOXW, &map_in, &full[s], tma_x, y0 + l, 0);
        }
        issued = first;
    }

    auto wait_row = [&](int l) -> bool {
        const bool ok = mbar_wait_bounded(&full[l % NS], (uint32_t)((l / NS) & 1));
        if (tid == 0 && ok && l == waited0) waited0 = l + 1;
        return ok;
    };

    bool ok = wait_row(0);
    ok = wait_row(1) && ok;
    if (!YWIN) ok = wait_row(2) && ok;
    bool bad = false;
    Acc<T> acc[4];
    const int col = tid + HALO;
    T ym[NV], fc[NV];  // YWIN: rows r-1 (y-moving planes) and r at this column
    if (YWIN && ok) {
        const T* s0 = ring;
        const T* s1 = ring + (size_t)(1 % NS) * NV * BOXW;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            if (moves_y<YWIN>(i)) ym[i] = s0[i * BOXW + col];
            fc[i] = s1[i * BOXW + col];
        }
    }

    auto drain = [&]() {
        if (tid == 0) {
            for (int l = waited0; l < issued; ++l)
                mbar_wait_bounded(&full[l % NS], (uint32_t)((l / NS) & 1));
            if (tstore) bulk_wait_all();
            atomicOr(a.flag, FLAG_TIMEOUT);
        }
    };
    if (__syncthreads_or(!ok)) { drain(); return; }
    if (YWIN && tid == 0 && NS < nload) {
        // row 0 now lives in registers: its slot takes row NS
        mbar_arrive_expect_tx(&full[0], SLOT_BYTES);
        tma_load_3d(ring, &map_in, &full[0], tma_x, y0 + NS, 0);
        issued = NS + 1;
    }

#pragma unroll 1
    for (int r = 1; r <= nrows; ++r) {
        const int y = y0 + r - 1;
        T* ob = outbuf + (size_t)(r & 1) * NV * TMA_W;
        if (YWIN) {
            ok = wait_row(r + 1);  // a failed wait is acted on at the barrier below
        }
        if (active && ok) {
            const T* sm = ring + (size_t)((r - 1) % NS) * NV * BOXW;
            const T* sc = ring + (size_t)(r % NS) * NV * BOXW;
            const T* sp = ring + (size_t)((r + 1) % NS) * NV * BOXW;
            T yp[NV];
            if (YWIN) {
#pragma unroll
                for (int i = 0; i < NV; ++i) yp[i] = sp[i * BOXW + col];
            }
            auto F = [&](int i, int pos) -> T {
                switch (pos) {
                    case C: return YWIN ? fc[i] : sc[i * BOXW + col];
                    case XM: return sc[i * BOXW + col - 1];
                    case XP: return sc[i * BOXW + col + 1];
                    case YM: return YWIN ? ym[i] : sm[i * BOXW + col];
                    default: return YWIN ? yp[i] : sp[i * BOXW + col];
                }
            };
            T out[NV];
            T rho, P;
            cell_update<T>(F, a.k, out, rho, P);
            if (YWIN) {
#pragma unroll
                for (int i = 0; i < NV; ++i) {
                    if (moves_y<YWIN>(i)) ym[i] = fc[i];
                    fc[i] = yp[i];
                }
            }
            bad |= !(rho > (T)0) | !(P > (T)0);
            if (TSTORE) {
#pragma unroll
                for (int i = 0; i < NV; ++i) ob[i * TMA_W + tid] = out[i];
            } else {
                store_cell<T>(a.out, L, a.per_x, a.per_y, x, y, out);
            }
            if (TOTALS) {
                T q0, q1, q2, q3;
                conserved_moments<T>(out, q0, q1, q2, q3);
                acc[0].add(q0); acc[1].add(q1); acc[2].add(q2); acc[3].add(q3);
            }
        }
        if (tstore) {
            fence_async_shared();              // make this thread's row visible to the TMA engine
            if (tid == 0) bulk_wait_read_all();  // the store from the other out slot has read it
        }
        if (!YWIN) ok = (r + 2 < nload) ? wait_row(r + 2) : true;
        // every thread is done with the slot released below, and the out row
        // is complete
        if (__syncthreads_or(!ok)) { drain(); return; }
        if (tid == 0) {
            if (tstore) {
                tma_store_3d(&map_out, ob, L.G + x0, y + 1, 0);
                if (a.per_y && y == 0) tma_store_3d(&map_out, ob, L.G + x0, L.ny + 1, 0);
                if (a.per_y && y == L.ny - 1) tma_store_3d(&map_out, ob, L.G + x0, 0, 0);
                bulk_commit();
            }
            // without YWIN row r-1 is the oldest row still read; with it, row r
            const int l = YWIN ? r + NS : r - 1 + NS;
            if (l < nload) {
                const int s = l % NS;
                mbar_arrive_expect_tx(&full[s], SLOT_BYTES);
                tma_load_3d(ring + (size_t)s * NV * BOXW, &map_in, &full[s], tma_x, y0 + l, 0);
                issued = l + 1;
            }
        }
        // after the elected thread has queued its copies
        if (TSTORE) {
            if (!tstore && active) {
                // ragged strip: this thread's column of the staged row, plus
                // the periodic ghost rows
                const long c0 = (long)(y + 1) * L.pitch + L.G + x;
#pragma unroll 4
                for (int i = 0; i < NV; ++i) {
                    const T v = ob[i * TMA_W + tid];
                    a.out[i * L.plane + c0] = v;
                    if (a.per_y && y == 0) a.out[i * L.plane + (long)(L.ny + 1) * L.pitch + L.G + x] = v;
                    if (a.per_y && y == L.ny - 1) a.out[i * L.plane + L.G + x] = v;
                }
            }
            if (a.per_x && (x == 0 || x == L.nx - 1)) {
                // periodic ghost columns are single values: plain stores
                const long gc = (long)(y + 1) * L.pitch + (x == 0 ? L.G + L.nx : L.G - 1);
#pragma unroll 4
                for (int i = 0; i < NV; ++i) a.out[i * L.plane + gc] = ob[i * TMA_W + tid];
            }
        }
    }
    if (tstore && tid == 0) bulk_wait_all();

    if (__syncthreads_or(bad) && tid == 0) atomicOr(a.flag, FLAG_UNSTABLE);
    if (TOTALS) {
        double v[4] = {acc[0].value(), acc[1].value(), acc[2].value(), acc[3].value()};
        block_sum4(v, a.partials + 4 * (size_t)(blockIdx.y * gridDim.x + blockIdx.x));
    }
}

// --------------------------------------------------------------------------
// One thread per cell, stencil straight from global memory.
// --------------------------------------------------------------------------
constexpr int DIR_BX = 32, DIR_BY = 8;

template <class T, bool TOTALS>
__global__ void __launch_bounds__(DIR_BX* DIR_BY) step_direct(const StepArgs<T> a) {
    const Layout& L = a.L;
    const int x = blockIdx.x * DIR_BX + threadIdx.x;
    const int y = blockIdx.y * DIR_BY + threadIdx.y;
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
                default: return __ldg(in + o + L.pitch);
            }
        };
        T out[NV];
        T rho, P;
        cell_update<T>(F, a.k, out, rho, P);
        bad = !healthy(rho, P);
        store_cell<T>(a.out, L, a.per_x, a.per_y, x, y, out);
        if (TOTALS) conserved_moments<T>(out, q[0], q[1], q[2], q[3]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(a.flag, FLAG_UNSTABLE);
    if (TOTALS) {
        double v[4] = {(double)q[0], (double)q[1], (double)q[2], (double)q[3]};
        block_sum4(v, a.partials + 4 * (size_t)(blockIdx.y * gridDim.x + blockIdx.x));
    }
}

template <class T, int NS, bool TSTORE, int MINB, bool YWIN = false>
struct TmaKernels {
    static cudaError_t launch(const CUtensorMap* mi, const CUtensorMap* mo, const StepArgs<T>& a, dim3 grid,
                              size_t smem, bool totals, cudaStream_t st) {
        if (totals)
            step_tma<T, true, NS, TSTORE, MINB, YWIN><<<grid, TMA_W, smem, st>>>(*mi, *mo, a);
        else
            step_tma<T, false, NS, TSTORE, MINB, YWIN><<<grid, TMA_W, smem, st>>>(*mi, *mo, a);
        return cudaGetLastError();
    }
    static cudaError_t occupancy(size_t smem, int* occ) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(step_tma<T, true, NS, TSTORE, MINB, YWIN>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(step_tma<T, false, NS, TSTORE, MINB, YWIN>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, step_tma<T, false, NS, TSTORE, MINB, YWIN>, TMA_W, smem);
    }
};

// FP64 rings are capped at 4 rows (16.9 KB per row).
template <class T, int NS> constexpr int ring_depth() { return sizeof(T) == 8 && NS > 4 ? 4 : NS; }

template <class T, class Fn>
cudaError_t with_tile(int tile, Fn&& fn) {
    switch (tile) {
        case 1: return fn(TmaKernels<T, ring_depth<T, 6>(), false, 4>());
        case 2: return fn(TmaKernels<T, ring_depth<T, 4>(), true, (sizeof(T) == 8 ? 2 : 4)>());
        case 3: return fn(TmaKernels<T, ring_depth<T, 6>(), true, (sizeof(T) == 8 ? 2 : 3)>());
        case 4: return fn(TmaKernels<T, ring_depth<T, 5>(), true, (sizeof(T) == 8 ? 2 : 3)>());
        case 5: return fn(TmaKernels<T, ring_depth<T, 4>(), true, (sizeof(T) == 8 ? 2 : 4), true>());
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <class T>
cudaError_t launch_step_tma(int tile, const CUtensorMap* map_in, const CUtensorMap* map_out, const StepArgs<T>& a,
                            int grid_x, int grid_y, bool totals, cudaStream_t st) {
    const size_t smem = tma_smem_bytes<T>(tile);
    return with_tile<T>(tile, [&](auto k) { return k.launch(map_in, map_out, a, dim3(grid_x, grid_y), smem, totals, st); });
}

template <class T>
cudaError_t tma_occupancy(int tile, int* blocks_per_sm) {
    const size_t smem = tma_smem_bytes<T>(tile);
    return with_tile<T>(tile, [&](auto k) { return k.occupancy(smem, blocks_per_sm); });
}

template <class T>
void direct_grid(const Layout& L, dim3* grid, dim3* block) {
    *block = dim3(DIR_BX, DIR_BY);
    *grid = dim3((L.nx + DIR_BX - 1) / DIR_BX, (L.ny + DIR_BY - 1) / DIR_BY);
}

template <class T>
cudaError_t launch_step_direct(const StepArgs<T>& a, bool totals, cudaStream_t st) {
    dim3 grid, block;
    direct_grid<T>(a.L, &grid, &block);
    if (totals) {
        step_direct<T, true><<<grid, block, 0, st>>>(a);
    } else {
        step_direct<T, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_step_tma<float>(int, const CUtensorMap*, const CUtensorMap*,
                                            const StepArgs<float>&, int, int, bool, cudaStream_t);
template cudaError_t launch_step_tma<double>(int, const CUtensorMap*, const CUtensorMap*,
                                             const StepArgs<double>&, int, int, bool, cudaStream_t);
template cudaError_t launch_step_direct<float>(const StepArgs<float>&, bool, cudaStream_t);
template cudaError_t launch_step_direct<double>(const StepArgs<double>&, bool, cudaStream_t);
template cudaError_t tma_occupancy<float>(int, int*);
template cudaError_t tma_occupancy<double>(int, int*);
template void direct_grid<float>(const Layout&, dim3*, dim3*);
template void direct_grid<double>(const Layout&, dim3*, dim3*);

}  // namespace mrt
