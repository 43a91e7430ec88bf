// batch.cu - many independent grids advanced together: every time step is
// one launch that covers all instances' work items (instance x 128-column
// strip x chunk of rows), and a pair of steps is captured once in a CUDA
// graph that mrt_batch_step replays.  Each instance is an ordinary grid
// (created by mrt_create, so initialisation, ghosts, tensor maps, readout and
// health are the single-grid ones); the batch adds
//   - a __constant__ table of the instances' step constants (the
//     relaxation rates, b, and Lax-Wendroff weights differ per instance),
//   - a device table of instance descriptors and their tensor maps,
//   - a work list (instance x strip x chunk of rows; longest first, then
//     instance by instance and row band by row band) that one wave of
//     resident CTAs takes items from through an atomic counter.
// Kernel boundaries order the steps, so no device-side grid barrier exists.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "host_state.h"
#include "step_strip.cuh"

using namespace mrt;

namespace {

constexpr int kCoefSlots = 256;                     // instances across all live batches (per device)
__constant__ Coef<float> c_batch_coef[kCoefSlots];  // 54 floats each: 55 KB
static_assert(sizeof(Coef<float>) == 54 * sizeof(float), "the FP32 step constants fill the constant table");

std::mutex g_slot_mu;
bool g_slot_used[kCoefSlots] = {};

struct BatchInst {
    Layout L;
    int per_x, per_y;
    float* f[2];
    unsigned* flag;
    int cslot;
    int pad;
    const CUtensorMap* maps;  // [load0, load1, store0, store1]
};

struct Item {
    int inst, x0, y0, nrows;
};

// One step of every instance.  Each CTA takes work items in list order
// from the step's counter (next[parity]); the index of its next item is
// fetched while the current one is processed, into the other of two shared
// slots (the barriers of an item separate a slot's read from its next
// write).  The CTA-level ring of the strip loop carries over from item to
// item.  The kernel also clears the other parity's counter for the next
// step, which stream order runs after this one.
template <int NS, bool TSTORE, bool YWIN, int MINB>
__global__ void __launch_bounds__(TMA_W, MINB) batch_step_kernel(const BatchInst* __restrict__ insts,
                                                                 const Item* __restrict__ items, int nitems,
                                                                 unsigned* __restrict__ next, int parity) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_item[2];
    if (blockIdx.x == 0 && threadIdx.x == 0) next[parity ^ 1] = 0u;
    if (threadIdx.x == 0) s_item[0] = (int)atomicAdd(&next[parity], 1u);
    __syncthreads();
    int cur = s_item[0];
    if (cur >= nitems) return;
    StripRing<float> R = strip_ring_init<float, NS, TSTORE>(smem_raw);
    for (int k = 1; cur < nitems; ++k) {
        if (threadIdx.x == 0) s_item[k & 1] = (int)atomicAdd(&next[parity], 1u);
        const Item w = items[cur];
        const BatchInst& I = insts[w.inst];
        const Layout L = I.L;
        const CUtensorMap* mi = I.maps + parity;
        const CUtensorMap* mo = I.maps + 2 + (parity ^ 1);
        bool bad = false;
        if (!strip_chunk<float, false, NS, TSTORE, YWIN>(R, mi, mo, L, I.per_x, I.per_y, I.f[parity ^ 1],
                                                         c_batch_coef[I.cslot], w.x0, w.y0, w.nrows, bad,
                                                         (Acc<float>*)nullptr)) {
            strip_drain<float, NS>(R, I.flag);
            return;
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(I.flag, FLAG_UNSTABLE);
        cur = s_item[k & 1];
    }
}

template <int NS, bool TSTORE, bool YWIN, int MINB>
struct BatchKernel {
    static size_t smem() {
        return NS * tma_slot_bytes<float>() + (TSTORE ? 2 * tma_out_slot_bytes<float>() : 0) + 64;
    }
    static cudaError_t setup(int* occ) {
        cudaError_t e = cudaFuncSetAttribute(batch_step_kernel<NS, TSTORE, YWIN, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_step_kernel<NS, TSTORE, YWIN, MINB>, TMA_W,
                                                             smem());
    }
    static cudaError_t launch(int grid, const BatchInst* insts, const Item* items, int nitems, unsigned* next,
                              int parity, cudaStream_t st) {
        batch_step_kernel<NS, TSTORE, YWIN, MINB><<<grid, TMA_W, smem(), st>>>(insts, items, nitems, next, parity);
        return cudaGetLastError();
    }
};

template <class Fn>
cudaError_t with_batch_tile(int tile, Fn&& fn) {
    switch (tile) {
        case 2: return fn(BatchKernel<4, true, false, 4>());
        case 4: return fn(BatchKernel<5, true, false, 3>());
        case 5: return fn(BatchKernel<4, true, true, 4>());
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

struct mrt_batch {
    int n = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<mrt_grid*> grids;
    std::vector<int> slots;
    BatchInst* d_insts = nullptr;
    CUtensorMap* d_maps = nullptr;
    Item* d_items = nullptr;
    unsigned* d_next = nullptr;  // per-parity work counters
    int tile = 4, rows_per_item = 32, grid = 0, nitems = 0;
    cudaGraphExec_t exec = nullptr;
    long steps = 0;
};

static void batch_release(mrt_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (mrt_grid* g : b->grids) mrt_destroy(g);
    cudaFree(b->d_insts);
    cudaFree(b->d_maps);
    cudaFree(b->d_items);
    cudaFree(b->d_next);
    {
        std::lock_guard<std::mutex> lock(g_slot_mu);
        for (int s : b->slots) g_slot_used[s] = false;
    }
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Work list: every strip of every instance cut into items of up to
// rows_per_item rows, longest first (ties in instance and strip order).  The
// CTAs of a step take items from this list through an atomic counter, so
// the balance does not rest on a cost model: a row of a narrow ragged strip
// or of a short instance costs about as much as a full one (each row is a
// ring step with a CTA barrier) while moving far fewer bytes.
static mrt_status build_work(mrt_batch* b) {
    std::vector<Item> items;
    for (int i = 0; i < b->n; ++i) {
        const Layout& L = b->grids[i]->L;
        for (int x0 = 0; x0 < L.nx; x0 += TMA_W)
            for (int y0 = 0; y0 < L.ny; y0 += b->rows_per_item)
                items.push_back({i, x0, y0, std::min(b->rows_per_item, L.ny - y0)});
    }
    // longest first; among equal heights instance by instance and, inside an
    // instance, row band by row band across all its strips, so that the items
    // in flight at any moment form a compact block of one or a few instances
    // whose shared boundary rows and halo columns are still in L2
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& c) {
        if (a.nrows != c.nrows) return a.nrows > c.nrows;
        if (a.inst != c.inst) return a.inst < c.inst;
        if (a.y0 != c.y0) return a.y0 < c.y0;
        return a.x0 < c.x0;
    });
    b->nitems = (int)items.size();
    cudaFree(b->d_items);
    b->d_items = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_items, sizeof(Item) * items.size())) != cudaSuccess)
        return mrt_fail(MRT_ENOMEM, "batch work list: %s", cudaGetErrorString(e));
    // on the batch's own (non-blocking) stream, so its kernels are ordered
    // after the copies
    if ((e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice,
                             b->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_next, 0, 2 * sizeof(unsigned), b->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        return mrt_fail(MRT_ECUDA, "batch work list: %s", cudaGetErrorString(e));
    return MRT_OK;
}

static mrt_status build_graph(mrt_batch* b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "capture: %s", cudaGetErrorString(e));
    for (int parity = 0; parity < 2; ++parity) {
        e = with_batch_tile(b->tile, [&](auto k) {
            return k.launch(b->grid, b->d_insts, b->d_items, b->nitems, b->d_next, parity, b->stream);
        });
        if (e != cudaSuccess) break;
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return mrt_fail(MRT_ECUDA, "capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return MRT_OK;
}

extern "C" mrt_status mrt_batch_tune(mrt_batch* b, int tile, int rows_per_item) {
    if (!b) return mrt_fail(MRT_EINVAL, "batch is NULL");
    if (tile != 2 && tile != 4 && tile != 5) return mrt_fail(MRT_EINVAL, "batch tile must be 2, 4 or 5");
    if (rows_per_item < 1) return mrt_fail(MRT_EINVAL, "rows_per_item must be >= 1");
    int occ = 0, sms = 0;
    cudaError_t e = with_batch_tile(tile, [&](auto k) { return k.setup(&occ); });
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "batch occupancy: %s", cudaGetErrorString(e));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    cudaStreamSynchronize(b->stream);
    b->tile = tile;
    b->rows_per_item = rows_per_item;
    b->grid = std::max(1, sms * std::max(occ, 1));
    mrt_status st = build_work(b);
    if (st != MRT_OK) return st;
    return build_graph(b);
}

extern "C" mrt_status mrt_batch_create(int n, const mrt_params* params, const double* const* rho,
                                       const double* const* ux, const double* const* uy, const double* const* T,
                                       int fields_on_device, mrt_batch** out) {
    if (!out || !params || !rho || !ux || !uy || !T) return mrt_fail(MRT_EINVAL, "null argument");
    if (n < 1 || n > kCoefSlots) return mrt_fail(MRT_EINVAL, "batch size must be 1..%d", kCoefSlots);
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (params[i].precision != MRT_FP32) return mrt_fail(MRT_EINVAL, "batched instances are FP32 (instance %d)", i);
        if (params[i].advection != MRT_ADV_LW)
            return mrt_fail(MRT_EINVAL, "batched instances take the axis-by-axis operator (instance %d)", i);
    }
    mrt_batch* b = new (std::nothrow) mrt_batch();
    if (!b) return mrt_fail(MRT_ENOMEM, "host allocation failed");
    b->n = n;
    cudaGetDevice(&b->device);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { batch_release(b); return mrt_fail(MRT_ECUDA, "stream: %s", cudaGetErrorString(e)); }
    {
        std::lock_guard<std::mutex> lock(g_slot_mu);
        for (int s = 0; s < kCoefSlots && (int)b->slots.size() < n; ++s)
            if (!g_slot_used[s]) { g_slot_used[s] = true; b->slots.push_back(s); }
    }
    if ((int)b->slots.size() < n) {
        batch_release(b);
        return mrt_fail(MRT_ENOMEM, "constant table full: %d instances fit across all live batches", kCoefSlots);
    }
    b->grids.assign(n, nullptr);
    std::vector<BatchInst> hi(n);
    std::vector<CUtensorMap> maps(4 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        mrt_params p = params[i];
        p.kernel = MRT_KERNEL_TMA;
        p.tile = 4;
        mrt_status st = mrt_create(&p, rho[i], ux[i], uy[i], T[i], fields_on_device, b->stream, &b->grids[i]);
        if (st != MRT_OK) { batch_release(b); return st; }
        mrt_grid* g = b->grids[i];
        if ((e = cudaMemcpyToSymbolAsync(c_batch_coef, &g->kf, sizeof(Coef<float>), sizeof(Coef<float>) * b->slots[i],
                                         cudaMemcpyHostToDevice, b->stream)) != cudaSuccess) {
            batch_release(b);
            return mrt_fail(MRT_ECUDA, "coefficients: %s", cudaGetErrorString(e));
        }
        hi[i].L = g->L;
        hi[i].per_x = g->p.bc_x == MRT_BC_PERIODIC;
        hi[i].per_y = g->p.bc_y == MRT_BC_PERIODIC;
        hi[i].f[0] = static_cast<float*>(g->f[0]);
        hi[i].f[1] = static_cast<float*>(g->f[1]);
        hi[i].flag = g->flag;
        hi[i].cslot = b->slots[i];
        maps[4 * i + 0] = g->maps[0];
        maps[4 * i + 1] = g->maps[1];
        maps[4 * i + 2] = g->maps_out[0];
        maps[4 * i + 3] = g->maps_out[1];
    }
    if ((e = cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * maps.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_insts, sizeof(BatchInst) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_next, 2 * sizeof(unsigned))) != cudaSuccess) {
        batch_release(b);
        return mrt_fail(MRT_ENOMEM, "batch tables: %s", cudaGetErrorString(e));
    }
    for (int i = 0; i < n; ++i) hi[i].maps = b->d_maps + 4 * i;
    if ((e = cudaMemcpyAsync(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                             b->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->d_insts, hi.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, b->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(b->stream)) != cudaSuccess) {
        batch_release(b);
        return mrt_fail(MRT_ECUDA, "batch tables: %s", cudaGetErrorString(e));
    }
    mrt_status st = mrt_batch_tune(b, 4, 32);
    if (st != MRT_OK) { batch_release(b); return st; }
    *out = b;
    return MRT_OK;
}

extern "C" mrt_status mrt_batch_step(mrt_batch* b, long nsteps) {
    NvtxRange range("mrt_batch_step");
    if (!b) return mrt_fail(MRT_EINVAL, "batch is NULL");
    if (nsteps < 0) return mrt_fail(MRT_EINVAL, "nsteps must be >= 0");
    long done = 0;
    int cur = b->grids[0]->cur;  // all instances share the buffer parity
    auto single = [&](int parity) -> mrt_status {
        cudaError_t e = with_batch_tile(b->tile, [&](auto k) {
            return k.launch(b->grid, b->d_insts, b->d_items, b->nitems, b->d_next, parity, b->stream);
        });
        if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "batch step: %s", cudaGetErrorString(e));
        return MRT_OK;
    };
    if (cur == 1 && nsteps > 0) {
        mrt_status st = single(1);
        if (st != MRT_OK) return st;
        cur = 0;
        done = 1;
    }
    for (; done + 2 <= nsteps; done += 2) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    }
    if (done < nsteps) {
        mrt_status st = single(0);
        if (st != MRT_OK) return st;
        cur = 1;
        done += 1;
    }
    for (mrt_grid* g : b->grids) {
        g->cur = cur;
        g->steps += nsteps;
        g->totals_fresh = false;
    }
    b->steps += nsteps;
    return MRT_OK;
}

extern "C" mrt_status mrt_batch_grid(mrt_batch* b, int i, mrt_grid** g) {
    if (!b || !g) return mrt_fail(MRT_EINVAL, "null argument");
    if (i < 0 || i >= b->n) return mrt_fail(MRT_EINVAL, "instance %d out of range", i);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "sync: %s", cudaGetErrorString(e));
    *g = b->grids[i];
    return MRT_OK;
}

extern "C" mrt_status mrt_batch_info(const mrt_batch* b, int* n, int* tile, int* rows_per_item, int* ctas,
                                     int* items) {
    if (!b) return mrt_fail(MRT_EINVAL, "batch is NULL");
    if (n) *n = b->n;
    if (tile) *tile = b->tile;
    if (rows_per_item) *rows_per_item = b->rows_per_item;
    if (ctas) *ctas = b->grid;
    if (items) *items = b->nitems;
    return MRT_OK;
}

extern "C" mrt_status mrt_batch_stream(const mrt_batch* b, void** stream) {
    if (!b || !stream) return mrt_fail(MRT_EINVAL, "null argument");
    *stream = (void*)b->stream;
    return MRT_OK;
}

extern "C" mrt_status mrt_batch_sync(mrt_batch* b) {
    if (!b) return mrt_fail(MRT_EINVAL, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "sync: %s", cudaGetErrorString(e));
    return MRT_OK;
}

extern "C" void mrt_batch_destroy(mrt_batch* b) { batch_release(b); }
