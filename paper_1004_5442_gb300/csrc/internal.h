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
template <class T> constexpr int tma_stages() { return sizeof(T) == 4 ? 6 : 4; }
template <class T> constexpr size_t tma_slot_bytes() { return (size_t)NV * tma_boxw<T>() * sizeof(T); }
template <class T> constexpr size_t tma_smem_bytes() {
    return tma_stages<T>() * tma_slot_bytes<T>() + 64;
}

// Launchers (step_kernels.cu).  grid_y = number of row chunks for the TMA
// kernel.  Return the launch status.
template <class T>
cudaError_t launch_step_tma(const CUtensorMap* map_in, const StepArgs<T>& a, int grid_x,
                            int grid_y, bool totals, cudaStream_t st);
template <class T>
cudaError_t launch_step_direct(const StepArgs<T>& a, bool totals, cudaStream_t st);
template <class T>
cudaError_t tma_occupancy(int* blocks_per_sm);
template <class T>
void direct_grid(const Layout& L, dim3* grid, dim3* block);

}  // namespace mrt
