// noalloc.cu - conserved totals of a caller-provided state without any
// allocation by the library.
//
// mrt_conserved_totals() keeps its block partials in memory that mrt_create()
// allocated.  Some callers cannot allocate device memory when they need the
// totals: a host framework that owns the whole device-memory budget through
// its own pool (a cudaMalloc behind its back can fail or break its
// accounting), and monitoring loops that must not stall on the allocator
// (cudaMalloc and cudaFree can synchronise the device).  For them this entry
// point keeps its scratch in a fixed array in the library's own device
// memory instead.
//
// The scratch array is a file-scope __device__ variable: every GPU that
// loads the library holds it (kMaxParts * 4 doubles = 128 KB) until the
// process exits.  Host code cannot use the array's name as a device address,
// so the address is obtained once per device with cudaGetSymbolAddress()
// while that device is current, and passed to the kernels.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/mrtfdlb.h"
#include "internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 64;
constexpr long kCellsPerBlock = (long)kThreads * kCellsPerThread;   // 16384
constexpr int kMaxParts = 4096;                                      // blocks
constexpr long kMaxCells = kCellsPerBlock * kMaxParts;               // 8192 x 8192
constexpr int kMaxDevices = 64;

// Block partials (rho, jx, jy, e) of the most recent call, shared by all calls.
static __device__ __align__(256) double g_scratch[kMaxParts * 4];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};


// Conserved moments of one cell of a dense [16][n] state, in FP64.
template <class T>
__device__ __forceinline__ void cell_moments(const T* __restrict__ f, long n, long c, double q[4]) {
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = (double)f[i * n + c];
    double S[4], Dx[4], Dy[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double* a = v + 4 * g;
        S[g] = (a[0] + a[2]) + (a[1] + a[3]);
        const double d02 = a[0] - a[2], d13 = a[1] - a[3];
        Dx[g] = g < 2 ? d02 : d02 - d13;
        Dy[g] = g < 2 ? d13 : d02 + d13;
    }
    q[0] = (S[0] + S[1]) + (S[2] + S[3]);
    q[1] = mrt::kU(0) * Dx[0] + mrt::kU(1) * Dx[1] + mrt::kU(2) * Dx[2] + mrt::kU(3) * Dx[3];
    q[2] = mrt::kU(0) * Dy[0] + mrt::kU(1) * Dy[1] + mrt::kU(2) * Dy[2] + mrt::kU(3) * Dy[3];
    q[3] = mrt::kW(0) * S[0] + mrt::kW(1) * S[1] + mrt::kW(2) * S[2] + mrt::kW(3) * S[3];
}

// Block b sums cells [b * kCellsPerBlock, (b+1) * kCellsPerBlock) and writes
// its four sums to scratch[4b .. 4b+3]; every slot it reads later is written
// by this call, so nothing needs clearing.
template <class T>
__global__ void __launch_bounds__(kThreads) partial_kernel(const T* __restrict__ f, long n,
                                                           double* __restrict__ scratch) {
    __shared__ double red[kThreads / 32][4];
    const long begin = (long)blockIdx.x * kCellsPerBlock;
    const long end = begin + kCellsPerBlock < n ? begin + kCellsPerBlock : n;
    double acc[4] = {0, 0, 0, 0};
    for (long c = begin + threadIdx.x; c < end; c += kThreads) {
        double q[4];
        cell_moments<T>(f, n, c, q);
        for (int k = 0; k < 4; ++k) acc[k] += q[k];
    }
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 4; ++k) red[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) {
            double s = 0;
            for (int w = 0; w < kThreads / 32; ++w) s += red[w][k];
            scratch[4 * blockIdx.x + k] = s;
        }
}

// Fixed-order sum of the first nparts partials, times scale = dx*dx (square
// cells: the entry point takes one cell size), into out[4].
__global__ void __launch_bounds__(kThreads) final_kernel(const double* __restrict__ scratch, int nparts,
                                                         double scale, double* __restrict__ out) {
    __shared__ double red[kThreads][4];
    double acc[4] = {0, 0, 0, 0};
    for (int p = threadIdx.x; p < nparts; p += kThreads)
        for (int k = 0; k < 4; ++k) acc[k] += scratch[4 * p + k];
    for (int k = 0; k < 4; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 4; ++k) red[threadIdx.x][k] += red[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) out[k] = red[0][k] * scale;
}

// Device address of g_scratch on the current device, looked up once.
mrt_status scratch_address(double** ptr) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        mrt::set_last_error("cudaGetDevice: %s", cudaGetErrorString(e));
        return MRT_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        mrt::set_last_error("device ordinal %d out of range", dev);
        return MRT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            mrt::set_last_error("cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return MRT_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *ptr = g_scratch_addr[dev];
    return MRT_OK;
}

}  // namespace

extern "C" mrt_status mrt_conserved_totals_static(const void* f, int precision, int nx, int ny, double dx,
                                                  double* out, void* stream) {
    if (!f || !out) {
        mrt::set_last_error("f and out must be device pointers, got NULL");
        return MRT_EINVAL;
    }
    if (nx < 1 || ny < 1 || !(dx > 0) || !std::isfinite(dx)) {
        mrt::set_last_error("need nx, ny >= 1 and finite dx > 0");
        return MRT_EINVAL;
    }
    if (precision != MRT_FP32 && precision != MRT_FP64) {
        mrt::set_last_error("precision must be MRT_FP32 or MRT_FP64");
        return MRT_EINVAL;
    }
    const long n = (long)nx * (long)ny;
    if (n > kMaxCells) {
        mrt::set_last_error("%d x %d = %ld cells exceeds the fixed scratch capacity of %ld cells", nx, ny, n, kMaxCells);
        return MRT_EINVAL;
    }
    double* scratch = nullptr;
    mrt_status st = scratch_address(&scratch);
    if (st != MRT_OK) return st;
    const int parts = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == MRT_FP32)
        partial_kernel<float><<<parts, kThreads, 0, s>>>(static_cast<const float*>(f), n, scratch);
    else
        partial_kernel<double><<<parts, kThreads, 0, s>>>(static_cast<const double*>(f), n, scratch);
    final_kernel<<<1, kThreads, 0, s>>>(scratch, parts, dx * dx, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mrt::set_last_error("launch: %s", cudaGetErrorString(e));
        return MRT_ECUDA;
    }
    return MRT_OK;
}
