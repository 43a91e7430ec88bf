// host_state.h - the grid and reverse-mode tape objects
// shared by the host-side translation units of the C ABI (kernels do not
// see them).
#pragma once
#include "internal.h"

// ---------------------------------------------------------------------------
// Grid object shared by the API translation units.
// ---------------------------------------------------------------------------

// Checkpoint tape of a recorded forward run (mrt_adjoint_record).
struct mrt_tape {
    long nsteps = 0;
    int K = 0;                  // steps between checkpoints
    int nck = 0;                // checkpoints: f at steps 0, K, 2K, ...
    size_t state_bytes = 0;     // one padded buffer
    void* ck = nullptr;         // nck buffers
    void* seg = nullptr;        // K - 1 buffers: states 1 .. K-1 of a recomputed segment
                                // (state 0 is read from its checkpoint buffer)
    CUtensorMap* seg_in = nullptr;   // load maps of the segment states, index 1 .. K-1
    CUtensorMap* seg_out = nullptr;  // store maps of the segment states, index 1 .. K-1
    CUtensorMap* ck_in = nullptr;    // load maps of the checkpoint buffers
    void* lam[2] = {nullptr, nullptr};
    double* gxb = nullptr;
    double* gyb = nullptr;
    double* gpart = nullptr;
    int nparts = 0;
    double* scratch = nullptr;  // 8 fields of nx*ny doubles + 12 sums
    // TMA reverse step: maps of the two adjoint buffers and its launch shape
    CUtensorMap lam_in[2], lam_out[2];
    int adj_tma = 0, adj_gx = 0, adj_gy = 0, adj_rows = 0;
};
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct mrt_grid {
    mrt_params p;
    int fp64;
    int xt = 0;                      // unsplit operator (MRT_ADV_LW2D)
    size_t elem;
    mrt::Layout L;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    unsigned* flag = nullptr;        // device flag word
    double* partials = nullptr;      // 2 buffers of max_parts x 4 doubles (block / warp partials)
    int max_parts = 0;
    // Totals slots of kTotalsSlot doubles: 4 totals, a copy of the flag word
    // and the sequence stamp of the step they belong to.  Slots 0 and 1: the
    // side-stream reductions; slot 2: reductions inside a caller's captured
    // graph; slot 3: the newer of slot tlast and slot 2, picked for a reader.
    static constexpr int kTotalsSlot = 6;
    static constexpr int kCapSlot = 2, kPickSlot = 3;
    double* totals_dev = nullptr;
    // The totals reduction and its read-back run on a side stream: a step
    // that reduces totals writes its partials into buffer tnext and goes on;
    // the side stream waits for it (ev_step), sums the partials into
    // totals_dev buffer tnext (ev_red), while the next steps already run.
    // A later totals step writing the same partials buffer waits for ev_red.
    cudaStream_t tstream = nullptr;
    cudaEvent_t ev_step[2] = {}, ev_red[2] = {};
    cudaEvent_t ev_tail = nullptr;   // the grid's stream tail, for readers on the side stream
    bool red_pending[2] = {false, false};
    int tnext = 0;                   // buffer of the next totals reduction
    // Graphs of two plain steps, by (cur, queue parity) at their start
    // (mrt_step replays them for all but the last step of a call).
    cudaGraphExec_t pair_exec[2][2] = {};
    int tlast = 0;                   // buffer holding the latest totals
    double* block_sums = nullptr;    // first-pass sums of the totals reduction
    // A reduction captured into a caller's graph has partials, first-pass
    // sums and totals slot of its own, so a replay never shares scratch with
    // a side-stream reduction still in flight.  Once a grid has been
    // captured, every totals-producing step first writes a sequence stamp
    // (seq[0] counts, seq[1 + slot] holds the stamp of that slot's partials)
    // on the grid's stream, and the readers take the slot with the newer one.
    double* cap_partials = nullptr;
    double* cap_block_sums = nullptr;
    unsigned long long* seq = nullptr;  // device: counter + 3 stamps
    bool cap_used = false;
    double* host_stage = nullptr;    // pinned host copy of totals_dev (one small DMA per read)
    static constexpr int kTotalsEvents = 8;
    cudaEvent_t tev[kTotalsEvents] = {};  // completion markers of asynchronous totals copies
    long tickets = 0;                // asynchronous totals copies issued
    bool totals_fresh = false;
    double* macro_tmp = nullptr;     // 4 fields, for host upload at creation and host readout
    // Host uploads and readouts of the four fields run in row chunks on a
    // copy stream, each chunk's copy overlapping the next (or previous)
    // chunk's initialisation or readout kernel on the grid's stream.
    cudaStream_t xstream = nullptr;
    cudaEvent_t ev_x = nullptr;
    long steps = 0;
    int kernel = MRT_KERNEL_DIRECT;  // in use
    CUtensorMap maps[2];       // loads: whole padded rows, box with halo
    CUtensorMap maps_out[2];   // stores: x extent ends before the right ghost
    int tile = 0;
    int tma_grid_x = 0, tma_grid_y = 0, rows_per_cta = 0;
    int strips = 0, nitems = 0;      // work-queue tiles: strips and (row band, strip) items
    int parts = 0;                   // block partials a totals step writes
    unsigned* qnext = nullptr;       // work-queue tiles: two launch counters
    // split kernel: completed-step count per tile for the multi-step launch,
    // and the number of blocks that launch uses (0: not available)
    unsigned* tile_done = nullptr;
    int persist_blocks = 0;
    int qpar = 0;                    // which counter the next launch uses
    mrt::Coef<double> kd;
    mrt::Coef<float> kf;
    double b;
    mrt_tape* tape = nullptr;
};


// Encode the load and store tensor maps of one padded buffer.
mrt_status mrt_encode_maps(const mrt_grid* g, void* buf, CUtensorMap* in, CUtensorMap* out);
void mrt_tape_free(mrt_tape* t);

template <class T>
mrt_status step_between(mrt_grid* g, const void* in, void* out, const CUtensorMap* map_in,
                        const CUtensorMap* map_out, bool totals);
// Recompute f = f^eq(rho, u, T) into buffer 0 (and both buffers' ghosts),
// as at creation; inputs on the device if on_device.
mrt_status mrt_reinit(mrt_grid* g, const double* rho, const double* ux, const double* uy, const double* T,
                      int on_device);
mrt_status mrt_fail(mrt_status s, const char* fmt, ...);
// mrt_step without the split kernel's multi-step launch: every step its own
// launch, as the reverse sweep recomputes its segments, so recorded and
// recomputed states are the same bits.
mrt_status mrt_step_single_launches(mrt_grid* g, long nsteps);
