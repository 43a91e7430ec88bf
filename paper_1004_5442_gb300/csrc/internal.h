// internal.h - interfaces between the host API (api.cu) and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "model.cuh"

namespace mrt {

// Records the message mrt_last_error() returns on the calling thread.
void set_last_error(const char* fmt, ...);

// Padded device layout of one distribution buffer:
//   f[i][r][c], i = 0..15, r = 0..ny+1 (row y lives at r = y + 1; rows 0 and
//   ny+1 are ghosts), c = 0..pitch-1 (column x lives at c = G + x; columns
//   G-1 and G+nx are ghosts).  G = 128 bytes / sizeof(T) keeps every data row
//   128-byte aligned; pitch is a multiple of 128 bytes.
struct Layout {
    int nx, ny;
    int G;          // elements before column 0
    long pitch;     // elements per row
    long plane;     // elements per plane = pitch * (ny + 2)
};

// Flag word bits written by the kernels.
constexpr unsigned FLAG_UNSTABLE = 1u;  // rho or P not positive, or not finite
constexpr unsigned FLAG_TIMEOUT = 2u;   // a bounded wait ran out

struct StepArgsBase {
    Layout L;
    int per_x, per_y;        // 1 where the axis is periodic (kernel refreshes ghosts)
    int rows_per_cta;        // TMA kernel: rows per CTA chunk
    double* partials;        // 4 doubles per CTA when totals are requested
    unsigned* flag;
};

template <class T>
struct StepArgs : StepArgsBase {
    const T* in;
    T* out;
    Coef<T> k;
};

// TMA strip kernel geometry.
constexpr int TMA_W = 128;                 // cells per CTA row (= threads per CTA)
template <class T> constexpr int tma_halo() { return 16 / (int)sizeof(T); }
template <class T> constexpr int tma_boxw() { return TMA_W + 2 * tma_halo<T>(); }
template <class T> constexpr size_t tma_slot_bytes() { return (size_t)NV * tma_boxw<T>() * sizeof(T); }
template <class T> constexpr size_t tma_out_slot_bytes() { return (size_t)NV * TMA_W * sizeof(T); }

// Compiled step-kernel variants ("tiles").  stages = rows in the load ring;
// tstore = outputs staged in shared memory and written by one TMA row store
// (else every thread stores its 16 values); minb = CTAs per SM the register
// budget is sized for.
struct TileCfg {
    int stages;
    int tstore;
    int minb;
    const char* name;
};
constexpr int NUM_TILES = 5;
// tile 0 is "automatic"; 1..4 are explicit
inline TileCfg tile_cfg(int tile) {
    switch (tile) {
        case 1: return {6, 0, 4, "ring6-stg-4cta"};
        case 2: return {4, 1, 4, "ring4-tma-4cta"};
        case 3: return {6, 1, 3, "ring6-tma-3cta"};
        default: return {5, 1, 3, "ring5-tma-3cta"};
    }
}
template <class T> constexpr int default_tile() { return sizeof(T) == 4 ? 2 : 1; }

template <class T>
inline size_t tma_smem_bytes(int tile) {
    const TileCfg c = tile_cfg(tile);
    const int stages = sizeof(T) == 8 ? (c.stages > 4 ? 4 : c.stages) : c.stages;
    return stages * tma_slot_bytes<T>() + (c.tstore ? 2 * tma_out_slot_bytes<T>() : 0) + 64;
}

// Launchers (step_kernels.cu).  grid_y = number of row chunks for the TMA
// kernel.  Return the launch status.
template <class T>
cudaError_t launch_step_tma(int tile, const CUtensorMap* map_in, const CUtensorMap* map_out,
                            const StepArgs<T>& a, int grid_x, int grid_y, bool totals, cudaStream_t st);
template <class T>
cudaError_t launch_step_direct(const StepArgs<T>& a, bool totals, cudaStream_t st);
template <class T>
cudaError_t tma_occupancy(int tile, int* blocks_per_sm);
template <class T>
void direct_grid(const Layout& L, dim3* grid, dim3* block);

}  // namespace mrt
