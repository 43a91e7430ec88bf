// internal.h - interfaces between the host API (api.cu) and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/mrtfdlb.h"
#include <nvtx3/nvToolsExt.h>
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
    int refl_x, refl_y;  // 1: reflecting wall at the low end of the axis (ghost refreshed every step)
};

// NVTX range over a host call (profilers show where the library's work
// starts and ends; costs nothing without one attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// FP64 grids below this many cells (4 rows of 128 cells per SM) run the
// direct kernel under MRT_KERNEL_AUTO.
constexpr long kSmallFp64Cells = 152L * 128 * 4;
// Grids up to this many cells run the split kernel (and its multi-step
// launch) under MRT_KERNEL_AUTO.  Measured per step: FP64 400 x 4 5.0 us and
// 1300 x 4 7.1 us against 11.3 us for the direct kernel, but 2048 x 8 12.7
// against 12.3; FP32 400 x 4 2.4 us against 4.1 us (the launch period of
// this part), 1300 x 4 6.2 against 4.1.
constexpr long kSplitFp64Cells = 8192;
constexpr long kSplitFp32Cells = 2048;

// Flag word bits written by the kernels.
constexpr unsigned FLAG_UNSTABLE = 1u;  // rho or P not positive, or not finite
constexpr unsigned FLAG_TIMEOUT = 2u;   // a bounded wait ran out

struct StepArgsBase {
    Layout L;
    int per_x, per_y;        // 1 where the axis is periodic (kernel refreshes ghosts)
    int rows_per_cta;        // TMA kernel: rows per CTA chunk (per work item with a queue)
    double* partials;        // 4 doubles per CTA (per warp of each work item with a queue) for totals
    unsigned* flag;
    // work-queue tiles: items are (row band, strip) pairs, numbered row band
    // by row band; next[parity] is this launch's counter, next[parity ^ 1]
    // the one the kernel clears for the following launch
    int strips, nitems, parity;
    unsigned* next;
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
    int queue_rows;  // 0: one static chunk of rows per CTA; else rows per work item
};
constexpr int NUM_TILES = 8;
// tile 0 is "automatic"; 1..7 are explicit.  Tiles 5 and 6 keep row r-1 of
// the y-moving planes in registers so more of the ring is in flight.  Tiles
// 6 and 7 are tiles 5 and 4 with a work queue: one wave of resident CTAs
// takes (row band, strip) items of queue_rows rows from an atomic counter,
// row band by row band, so the items in flight form a compact block (at
// 4096^2 with 8-row items: about 150 rows across the full width) whose
// shared boundary rows and halo columns are still in L2 and whose rows of
// each plane are one contiguous range of memory.  Measured at 4096^2 FP32,
// tile 6 runs best with 8-row items (0.95 of the copy peak; 16 rows 0.91,
// 4 rows 0.88) and tile 7 with 32.
inline TileCfg tile_cfg(int tile) {
    switch (tile) {
        case 1: return {6, 0, 4, "ring6-stg-4cta", 0};
        case 2: return {4, 1, 4, "ring4-tma-4cta", 0};
        case 3: return {6, 1, 3, "ring6-tma-3cta", 0};
        case 4: return {5, 1, 3, "ring5-tma-3cta", 0};
        case 5: return {4, 1, 4, "ring4-tma-4cta-ywin", 0};
        case 6: return {4, 1, 4, "ring4-tma-4cta-ywin-queue8", 8};
        default: return {5, 1, 3, "ring5-tma-3cta-queue32", 32};
    }
}
// Tile 0 picks the work-queue tile for grids with at least two items per
// resident CTA, else the static tile of the precision.
constexpr int kQueueTile = 6;
constexpr int kStaticTileF32 = 4;
constexpr int kStaticTileF64 = 1;
// The unsplit operator runs on every tile but 2 and 3; its queue tile is 6
// (row r-1's diagonal x neighbours then come from registers).
constexpr int kQueueTileXT = 6;
inline bool tile_supports_xt(int tile) { return tile != 2 && tile != 3; }
// Rows per work item of a queue tile (0 for a static tile).  The unsplit
// operator's tile 6 takes 10-row items: at 4096^2 FP32 it ran at 0.885,
// 0.916, 0.935, 0.935 and 0.920 of the measured copy peak with 6, 8, 10, 12
// and 16 rows, where the method's operator peaks at 8 (0.950, 0.967, 0.956,
// 0.936, 0.917): its longer cell update amortises an item's two boundary
// rows over more rows before the block in flight grows too wide for L2.
constexpr int kQueueRowsXT = 10;
inline int queue_rows(int tile, bool xt) {
    const int r = tile_cfg(tile).queue_rows;
    return (xt && tile == kQueueTileXT && r > 0) ? kQueueRowsXT : r;
}

template <class T>
inline size_t tma_smem_bytes(int tile) {
    const TileCfg c = tile_cfg(tile);
    const int stages = sizeof(T) == 8 ? (c.stages > 4 ? 4 : c.stages) : c.stages;
    return stages * tma_slot_bytes<T>() + (c.tstore ? 2 * tma_out_slot_bytes<T>() : 0) + 64;
}

// Launchers (step_kernels.cu).  grid_y = number of row chunks for the TMA
// kernel.  Return the launch status.
// xt: the unsplit operator (MRT_ADV_LW2D; TMA tiles 1, 4, 5, 6 and 7).
template <class T>
cudaError_t launch_step_tma(int tile, bool xt, const CUtensorMap* map_in, const CUtensorMap* map_out,
                            const StepArgs<T>& a, int grid_x, int grid_y, bool totals, cudaStream_t st);
template <class T>
cudaError_t launch_step_direct(const StepArgs<T>& a, bool xt, bool totals, cudaStream_t st);
template <class T>
cudaError_t tma_occupancy(int tile, bool xt, int* blocks_per_sm);
template <class T>
void direct_grid(const Layout& L, dim3* grid, dim3* block);
// Four warps per 32-cell row segment, one per velocity group (small grids);
// one totals partial per block.
template <class T>
cudaError_t launch_step_split(const StepArgs<T>& a, bool xt, bool totals, cudaStream_t st);
void split_grid(const Layout& L, dim3* grid, dim3* block);
// All nsteps of a call in one cooperative launch of split tiles (small
// grids): step s reads buf0 for even s, buf1 for odd s; the last step
// writes totals partials (one per tile) if totals; done holds one
// completed-step count per tile and must be zero at launch.  blocks: at most
// split_persist_blocks (every block resident).
template <class T>
cudaError_t split_persist_blocks(bool xt, int* blocks);
template <class T>
cudaError_t launch_step_split_persist(const StepArgs<T>& a, bool xt, T* buf0, T* buf1, int nsteps, bool totals,
                                      unsigned* done, int blocks, cudaStream_t st);


// Reverse-sweep arguments (adjoint_kernels.cu).
template <class T>
struct AdjArgs {
    Layout L;
    int per_x, per_y;
    const T* lam_in;       // dL/df^{n+1}, padded layout; fixed ghosts hold 0
    const T* f;            // f^n, padded layout (centre values only)
    T* lam_out;            // dL/df^n
    double* gxb;           // fixed x-ghost adjoints [16][2][ny] (unused if periodic)
    double* gyb;           // fixed y-ghost adjoints [16][2][nx]
    double* gpart;         // rate partials [slots][12], accumulated (TMA kernel: one slot per item)
    Coef<T> k;
    unsigned* flag;        // FLAG_TIMEOUT when a bounded wait ran out (TMA kernel)
};

template <class T>
void adjoint_grid(const Layout& L, dim3* grid, dim3* block);
// xt: the unsplit operator (its fixed-ghost adjoints then come from
// launch_ghost_gather_xt, run after each reverse step).
template <class T>
cudaError_t launch_adjoint_step(const AdjArgs<T>& a, bool xt, cudaStream_t st);
template <class T>
cudaError_t launch_ghost_gather_xt(const AdjArgs<T>& a, cudaStream_t st);
template <class T>
cudaError_t launch_lam_from_drho(const Layout& L, const double* drho, T* lam, cudaStream_t st);
template <class T>
cudaError_t launch_ghost_adjoint(const Layout& L, int fix_x, int fix_y, const double* gxb, const double* gyb,
                                 T* lam, cudaStream_t st);
template <class T>
cudaError_t launch_init_adjoint(const Layout& L, const InitCoef& ic, const Coef<T>& kc, const T* lam,
                                const double* rho, const double* ux, const double* uy, const double* Tf,
                                double* g_rho, double* g_ux, double* g_uy, double* g_T, cudaStream_t st);
cudaError_t launch_sum_partials(const double* gpart, int nparts, double* out, cudaStream_t st);
template <class T>
cudaError_t adjoint_tma_setup(bool xt, int* blocks_per_sm);
template <class T>
cudaError_t launch_adjoint_tma(const CUtensorMap* map_lam, const CUtensorMap* map_f, const CUtensorMap* map_out,
                               const AdjArgs<T>& a, bool xt, int grid_x, int grid_y, int rows_per_cta,
                               cudaStream_t st);

}  // namespace mrt
