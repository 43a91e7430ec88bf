// diag.cu - diagnostics of the library itself (no counterpart in the paper):
//
//  * mrt_debug_padding: every row of a grid's padded buffers has columns that
//    no kernel may write - left of the left ghost column and right of the
//    right one (the TMA store maps end at the last data column, the ghost
//    stores are single columns).  They are zero from creation on, so a
//    nonzero word there is an out-of-bounds write: a guard band, in place of
//    a memory checker.
//  * mrt_debug_wait_timeout: one thread runs the kernels' bounded mbarrier
//    wait on a barrier that nothing completes, so the wait runs out (after
//    its 2 s limit) and sets the timeout flag, which mrt_health reports as
//    MRT_ETIMEOUT.  It exercises the failure path of every TMA kernel without
//    a fault, a trap or an unbounded wait.
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

__global__ void wait_timeout_kernel(unsigned* flag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar, 1);
        tma::fence_barrier_init();
        // nothing arrives on the barrier: the bounded wait gives up
        if (!tma::mbar_wait_bounded(&bar, 0u)) atomicOr(flag, FLAG_TIMEOUT);
    }
}

}  // namespace

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
    wait_timeout_kernel<<<1, 32, 0, g->stream>>>(g->flag);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "timeout probe: %s", cudaGetErrorString(e));
    return MRT_OK;
}
