// diag.cu - diagnostics of the library itself (no counterpart in the paper):
//
//  * mrt_debug_padding: every row of a grid's padded buffers has columns that
//    no kernel may write - left of the left ghost column and right of the
//    right one (the TMA store maps end at the last data column, the ghost
//    stores are single columns).  They are zero from creation on, so a
//    nonzero word there is an out-of-bounds write: a guard band, in place of
//    a memory checker.
//  * mrt_debug_wait_timeout: one thread runs the kernels' bounded mbarrier
//    wait on a barrier that nothing completes, another the multi-step
//    launch's bounded wait on a tile counter that nothing raises, so both
//    waits run out (after their 2 s limit) and set the timeout flag, which
//    mrt_health reports as MRT_ETIMEOUT.  It exercises the failure path of
//    every TMA kernel and of the multi-step launch without a fault, a trap
//    or an unbounded wait.
//  * mrt_debug_fma_rate: the device's fused multiply-add throughput in FP32
//    or FP64, the arithmetic roof against which the FP64 step (bound by the
//    FP64 pipe on this part) is measured.
#include "host_state.h"
#include "tma.cuh"

using namespace mrt;

namespace {

template <class T>
__global__ void padding_kernel(Layout L, const T* __restrict__ f, unsigned long long* count) {
    const int left = L.G - 1;                                   // columns 0 .. G-2
    const int right = (int)(L.pitch - (L.G + L.nx + 1));       // columns G+nx+1 .. pitch-1
    const int per_row = left + right;
    const long rows = 16L * (L.ny + 2);
    unsigned long long c = 0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < rows * per_row;
         t += (long)gridDim.x * blockDim.x) {
        const long r = t / per_row;
        const int k = (int)(t % per_row);
        const int col = k < left ? k : L.G + L.nx + 1 + (k - left);
        const int plane = (int)(r / (L.ny + 2)), row = (int)(r % (L.ny + 2));
        if (f[plane * L.plane + (long)row * L.pitch + col] != (T)0) ++c;
    }
    if (c) atomicAdd(count, c);
}

__global__ void wait_timeout_kernel(unsigned* flag, const unsigned* never) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar, 1);
        tma::fence_barrier_init();
        // nothing arrives on the barrier: the bounded wait gives up
        if (!tma::mbar_wait_bounded(&bar, 0u)) atomicOr(flag, FLAG_TIMEOUT);
    }
    if (threadIdx.x == 32) {
        // nothing raises the counter: the multi-step launch's bounded wait
        // on a neighbour tile gives up
        if (!tma::wait_at_least(never, 1u)) atomicOr(flag, FLAG_TIMEOUT);
    }
}

// Independent multiply-add chains a <- a * b + c per thread (b = c = 1/2:
// every chain converges to 1 and stays a normal number, so no denormal or
// overflow path is timed).  kChains chains give each warp enough
// independent instructions to cover the pipe latency; the sum is stored only
// if it equals a value it cannot reach, which keeps every chain live.
constexpr int kFmaMaxThreads = 1024;
constexpr int kFmaChains = 8;
constexpr int kFmaUnroll = 16;
template <class T>
__global__ void __launch_bounds__(kFmaMaxThreads) fma_kernel(long iters, int active_lanes, T b, T c, T* out) {
    if ((int)(threadIdx.x & 31) >= active_lanes) return;
    T a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = (T)(threadIdx.x + 1) * (T)(k + 1) * (T)1e-3;
    for (long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kFmaUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += a[k];
    if (s == (T)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// A kernel that does nothing but exist, for the launch period.
__global__ void empty_kernel(int* sink) {
    if (sink && threadIdx.x == 1u << 30) *sink = 0;
}

}  // namespace

extern "C" mrt_status mrt_debug_fma_rate(int precision, long iters, int blocks_per_sm, int threads_per_block,
                                         int active_lanes, double* flops_per_s, double* ms) {
    if (!flops_per_s || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || threads_per_block < 32 ||
        threads_per_block > kFmaMaxThreads || threads_per_block % 32 || blocks_per_sm * threads_per_block > 2048 ||
        active_lanes < 1 || active_lanes > 32 || (precision != MRT_FP32 && precision != MRT_FP64))
        return mrt_fail(MRT_EINVAL, "need precision MRT_FP32 or MRT_FP64, iters >= 1, 1 <= blocks_per_sm <= 8, "
                                    "threads_per_block a multiple of 32 in 32..1024 with at most 2048 threads per "
                                    "SM, 1 <= active_lanes <= 32, flops_per_s");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * blocks_per_sm;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void* out = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMallocAsync(&out, (size_t)blocks * threads_per_block * 8, st);
    float el = 0.f;
    if (e == cudaSuccess) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
            e = cudaEventRecord(e0, st);
            if (precision == MRT_FP64)
                fma_kernel<double><<<blocks, threads_per_block, 0, st>>>(iters, active_lanes, 0.5, 0.5,
                                                                         static_cast<double*>(out));
            else
                fma_kernel<float><<<blocks, threads_per_block, 0, st>>>(iters, active_lanes, 0.5f, 0.5f,
                                                                        static_cast<float*>(out));
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&el, e0, e1);
        cudaFreeAsync(out, st);
        cudaStreamSynchronize(st);
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "fma rate: %s", cudaGetErrorString(e));
    const double warps = (double)blocks * (threads_per_block / 32);
    const double flops = 2.0 * kFmaChains * kFmaUnroll * (double)iters * warps * active_lanes;
    *flops_per_s = flops / (el * 1e-3);
    if (ms) *ms = el;
    return MRT_OK;
}

extern "C" mrt_status mrt_debug_launch_period(int nlaunches, int blocks, int threads, double* us_stream,
                                              double* us_graph) {
    if (nlaunches < 2 || nlaunches % 2 || blocks < 1 || threads < 1 || threads > 1024 || !us_stream || !us_graph)
        return mrt_fail(MRT_EINVAL, "need an even nlaunches >= 2, blocks >= 1, 1 <= threads <= 1024, outputs");
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float a = 0.f, b = 0.f;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        empty_kernel<<<blocks, threads, 0, st>>>(nullptr);
        e = cudaEventRecord(e0, st);
        for (int i = 0; i < nlaunches && e == cudaSuccess; ++i) {
            empty_kernel<<<blocks, threads, 0, st>>>(nullptr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, e0, e1);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        empty_kernel<<<blocks, threads, 0, st>>>(nullptr);
        empty_kernel<<<blocks, threads, 0, st>>>(nullptr);
        const cudaError_t ec = cudaStreamEndCapture(st, &graph);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = ec;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int i = 0; i < nlaunches / 2 && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, e0, e1);
    if (st) cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "launch period: %s", cudaGetErrorString(e));
    *us_stream = 1e3 * a / nlaunches;
    *us_graph = 1e3 * b / nlaunches;
    return MRT_OK;
}

extern "C" mrt_status mrt_debug_padding(mrt_grid* g, long* nonzero) {
    if (!g || !nonzero) return mrt_fail(MRT_EINVAL, "null argument");
    unsigned long long* d = nullptr;
    unsigned long long h = 0;
    cudaError_t e = cudaMallocAsync(&d, sizeof h, g->stream);
    if (e != cudaSuccess) return mrt_fail(MRT_ENOMEM, "debug counter: %s", cudaGetErrorString(e));
    cudaMemsetAsync(d, 0, sizeof h, g->stream);
    for (int b = 0; b < 2; ++b) {
        if (g->fp64)
            padding_kernel<double><<<256, 256, 0, g->stream>>>(g->L, static_cast<const double*>(g->f[b]), d);
        else
            padding_kernel<float><<<256, 256, 0, g->stream>>>(g->L, static_cast<const float*>(g->f[b]), d);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cudaFreeAsync(d, g->stream);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "padding check: %s", cudaGetErrorString(e));
    *nonzero = (long)h;
    return MRT_OK;
}

extern "C" mrt_status mrt_debug_wait_timeout(mrt_grid* g) {
    if (!g) return mrt_fail(MRT_EINVAL, "grid is NULL");
    // a zero counter that nothing raises, freed in stream order after the probe
    unsigned* never = nullptr;
    cudaError_t e = cudaMallocAsync(&never, sizeof(unsigned), g->stream);
    if (e != cudaSuccess) return mrt_fail(MRT_ENOMEM, "timeout probe: %s", cudaGetErrorString(e));
    e = cudaMemsetAsync(never, 0, sizeof(unsigned), g->stream);
    if (e == cudaSuccess) {
        wait_timeout_kernel<<<1, 64, 0, g->stream>>>(g->flag, never);
        e = cudaGetLastError();
    }
    cudaFreeAsync(never, g->stream);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "timeout probe: %s", cudaGetErrorString(e));
    return MRT_OK;
}
