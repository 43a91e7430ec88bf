// adjoint_api.cu - reverse mode through a recorded run (C ABI):
//   mrt_adjoint_record    f^0 = f^eq(fields), nsteps forward steps, f kept at
//                         every ckpt_every-th step
//   mrt_adjoint_backward  from dL/drho_N: segment by segment (last first) the
//                         states are recomputed from their checkpoint and the
//                         reverse step runs back through them; then the fixed
//                         ghosts' and the initial map's adjoints give
//                         dL/d(rho, u, T) at t = 0, and the per-block rate
//                         partials give dL/ds_k
//   mrt_adjoint_step      one reverse step on caller-provided states
#include <algorithm>
#include <cstring>
#include <new>

#include "host_state.h"

using namespace mrt;

#define A_TRY(call)                                                                                    \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return mrt_fail(e_ == cudaErrorMemoryAllocation ? MRT_ENOMEM : MRT_ECUDA, "%s: %s", #call, \
                            cudaGetErrorString(e_));                                                   \
    } while (0)

mrt_status mrt_refresh_periodic_ghosts(mrt_grid* g, void* buf);

void mrt_tape_free(mrt_tape* t) {
    if (!t) return;
    cudaFree(t->ck);
    cudaFree(t->seg);
    cudaFree(t->lam[0]);
    cudaFree(t->lam[1]);
    cudaFree(t->gxb);
    cudaFree(t->gyb);
    cudaFree(t->gpart);
    cudaFree(t->scratch);
    delete[] t->seg_in;
    delete[] t->seg_out;
    delete[] t->ck_in;
    delete t;
}

static char* buf_at(void* base, size_t bytes, long i) { return static_cast<char*>(base) + bytes * (size_t)i; }

extern "C" mrt_status mrt_adjoint_record(mrt_grid* g, const double* rho0, const double* ux0, const double* uy0,
                                         const double* T0, int on_device, long nsteps, int ckpt_every) {
    NvtxRange range("mrt_adjoint_record");
    if (!g) return mrt_fail(MRT_EINVAL, "grid is NULL");
    if (nsteps < 1) return mrt_fail(MRT_EINVAL, "nsteps must be >= 1");
    if (ckpt_every < 1) return mrt_fail(MRT_EINVAL, "ckpt_every must be >= 1");
    if (!rho0 || !ux0 || !uy0 || !T0) return mrt_fail(MRT_EINVAL, "null field pointer");
    mrt_tape_free(g->tape);
    g->tape = nullptr;
    mrt_tape* t = new (std::nothrow) mrt_tape();
    if (!t) return mrt_fail(MRT_ENOMEM, "host allocation failed");
    g->tape = t;
    const long n = (long)g->L.nx * g->L.ny;
    t->nsteps = nsteps;
    t->K = (int)(ckpt_every < nsteps ? ckpt_every : nsteps);
    t->nck = (int)((nsteps + t->K - 1) / t->K);
    t->state_bytes = 16 * (size_t)g->L.plane * g->elem;
    dim3 agrid, ablock;
    if (g->fp64) adjoint_grid<double>(g->L, &agrid, &ablock); else adjoint_grid<float>(g->L, &agrid, &ablock);
    t->nparts = (int)(agrid.x * agrid.y);
    if (g->kernel == MRT_KERNEL_TMA) {
        // TMA reverse step: its own occupancy decides the row chunks
        int occ = 0, sms = 0;
        cudaError_t e = g->fp64 ? adjoint_tma_setup<double>(g->xt, &occ) : adjoint_tma_setup<float>(g->xt, &occ);
        if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "adjoint occupancy: %s", cudaGetErrorString(e));
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        if (occ < 1) occ = 1;
        const int strips = (g->L.nx + TMA_W - 1) / TMA_W;
        // as many row chunks as fit in one wave of resident CTAs
        long chunks = ((long)sms * occ) / strips;
        if (chunks < 1) chunks = 1;
        t->adj_rows = (int)((g->L.ny + chunks - 1) / chunks);
        if (t->adj_rows < 1) t->adj_rows = 1;
        t->adj_gx = strips;
        t->adj_gy = (g->L.ny + t->adj_rows - 1) / t->adj_rows;
        t->adj_tma = 1;
        // only the TMA reverse step runs: one rate-partial slot per CTA
        t->nparts = t->adj_gx * t->adj_gy;
    }
    A_TRY(cudaMalloc(&t->ck, t->state_bytes * (size_t)t->nck));
    A_TRY(cudaMalloc(&t->seg, t->state_bytes * (size_t)std::max(t->K - 1, 1)));
    A_TRY(cudaMalloc(&t->lam[0], t->state_bytes));
    A_TRY(cudaMalloc(&t->lam[1], t->state_bytes));
    A_TRY(cudaMalloc(&t->gxb, sizeof(double) * 32 * (size_t)g->L.ny));
    A_TRY(cudaMalloc(&t->gyb, sizeof(double) * 32 * (size_t)g->L.nx));
    A_TRY(cudaMalloc(&t->gpart, sizeof(double) * 12 * (size_t)t->nparts));
    A_TRY(cudaMalloc(&t->scratch, sizeof(double) * (9 * (size_t)n + 16)));
    // the initial fields stay on the device for the initial map's adjoint
    double* f0 = t->scratch;
    const double* src[4] = {rho0, ux0, uy0, T0};
    for (int q = 0; q < 4; ++q)
        A_TRY(cudaMemcpyAsync(f0 + q * n, src[q], sizeof(double) * n,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    mrt_status st = mrt_reinit(g, f0, f0 + n, f0 + 2 * n, f0 + 3 * n, 1);
    if (st != MRT_OK) return st;
    if (g->kernel == MRT_KERNEL_TMA) {
        t->seg_in = new (std::nothrow) CUtensorMap[t->K];
        t->seg_out = new (std::nothrow) CUtensorMap[t->K];
        t->ck_in = new (std::nothrow) CUtensorMap[t->nck];
        if (!t->seg_in || !t->seg_out || !t->ck_in) return mrt_fail(MRT_ENOMEM, "host allocation failed");
        for (int j = 1; j < t->K; ++j) {
            st = mrt_encode_maps(g, buf_at(t->seg, t->state_bytes, j - 1), &t->seg_in[j], &t->seg_out[j]);
            if (st != MRT_OK) return st;
        }
        for (int c = 0; c < t->nck; ++c) {
            CUtensorMap unused;
            st = mrt_encode_maps(g, buf_at(t->ck, t->state_bytes, c), &t->ck_in[c], &unused);
            if (st != MRT_OK) return st;
        }
    }
    // every segment buffer carries the fixed-equilibrium ghosts of f^0 (on
    // periodic axes the recompute steps write every ghost they later read,
    // and segment buffer 0 is a full checkpoint copy)
    if (g->p.bc_x != MRT_BC_PERIODIC || g->p.bc_y != MRT_BC_PERIODIC)
        for (int j = 0; j + 1 < t->K; ++j)
            A_TRY(cudaMemcpyAsync(buf_at(t->seg, t->state_bytes, j), g->f[g->cur], t->state_bytes,
                                  cudaMemcpyDeviceToDevice, g->stream));
    if (t->adj_tma)
        for (int b = 0; b < 2; ++b) {
            st = mrt_encode_maps(g, t->lam[b], &t->lam_in[b], &t->lam_out[b]);
            if (st != MRT_OK) return st;
        }
    // adjoint buffers: zero everywhere, so fixed ghosts read as zero
    A_TRY(cudaMemsetAsync(t->lam[0], 0, t->state_bytes, g->stream));
    A_TRY(cudaMemsetAsync(t->lam[1], 0, t->state_bytes, g->stream));
    // forward run with checkpoints
    for (int c = 0; c < t->nck; ++c) {
        A_TRY(cudaMemcpyAsync(buf_at(t->ck, t->state_bytes, c), g->f[g->cur], t->state_bytes,
                              cudaMemcpyDeviceToDevice, g->stream));
        const long len = std::min<long>(t->K, nsteps - (long)c * t->K);
        st = mrt_step_single_launches(g, len);
        if (st != MRT_OK) return st;
    }
    return MRT_OK;
}

template <class T>
static mrt_status backward_impl(mrt_grid* g, const double* drho, double* outs[4], double g_s[16], int on_device) {
    mrt_tape* t = g->tape;
    const long n = (long)g->L.nx * g->L.ny;
    double* f0 = t->scratch;
    double* dev_drho = t->scratch + 4 * n;
    double* gout = t->scratch + 5 * n;  // 4 fields; sums after them
    double* sums = t->scratch + 9 * n;
    A_TRY(cudaMemcpyAsync(dev_drho, drho, sizeof(double) * n,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    // dL/df^N_i = dL/drho_N for every i (rho = sum_i f_i)
    A_TRY(cudaMemsetAsync(t->lam[0], 0, t->state_bytes, g->stream));
    A_TRY(cudaMemsetAsync(t->lam[1], 0, t->state_bytes, g->stream));
    A_TRY(launch_lam_from_drho<T>(g->L, dev_drho, static_cast<T*>(t->lam[0]), g->stream));
    mrt_status st = mrt_refresh_periodic_ghosts(g, t->lam[0]);
    if (st != MRT_OK) return st;
    A_TRY(cudaMemsetAsync(t->gxb, 0, sizeof(double) * 32 * (size_t)g->L.ny, g->stream));
    A_TRY(cudaMemsetAsync(t->gyb, 0, sizeof(double) * 32 * (size_t)g->L.nx, g->stream));
    A_TRY(cudaMemsetAsync(t->gpart, 0, sizeof(double) * 12 * (size_t)t->nparts, g->stream));

    AdjArgs<T> a;
    a.L = g->L;
    a.per_x = g->p.bc_x == MRT_BC_PERIODIC;
    a.per_y = g->p.bc_y == MRT_BC_PERIODIC;
    a.gxb = t->gxb;
    a.gyb = t->gyb;
    a.gpart = t->gpart;
    if constexpr (sizeof(T) == 8) a.k = g->kd; else a.k = g->kf;
    a.flag = g->flag;
    int cur = 0;
    for (int c = t->nck - 1; c >= 0; --c) {
        const long s0 = (long)c * t->K;
        const int len = (int)std::min<long>(t->K, t->nsteps - s0);
        // state j of the segment: the checkpoint itself for j = 0 (read only,
        // never copied), a recomputed buffer for j >= 1
        auto state = [&](int j) -> char* {
            return j == 0 ? buf_at(t->ck, t->state_bytes, c) : buf_at(t->seg, t->state_bytes, j - 1);
        };
        auto load_map = [&](int j) -> const CUtensorMap* {
            if (!t->seg_in) return nullptr;
            return j == 0 ? &t->ck_in[c] : &t->seg_in[j];
        };
        for (int j = 0; j + 1 < len; ++j) {
            st = step_between<T>(g, state(j), state(j + 1), load_map(j), t->seg_out ? &t->seg_out[j + 1] : nullptr,
                                 false);
            if (st != MRT_OK) return st;
        }
        for (int j = len - 1; j >= 0; --j) {
            a.lam_in = static_cast<const T*>(t->lam[cur]);
            a.f = reinterpret_cast<const T*>(state(j));
            a.lam_out = static_cast<T*>(t->lam[cur ^ 1]);
            if (t->adj_tma)
                A_TRY(launch_adjoint_tma<T>(&t->lam_in[cur], load_map(j), &t->lam_out[cur ^ 1], a, g->xt, t->adj_gx,
                                            t->adj_gy, t->adj_rows, g->stream));
            else
                A_TRY(launch_adjoint_step<T>(a, g->xt, g->stream));
            if (g->xt) A_TRY(launch_ghost_gather_xt<T>(a, g->stream));
            cur ^= 1;
        }
    }
    A_TRY(launch_ghost_adjoint<T>(g->L, !a.per_x, !a.per_y, t->gxb, t->gyb, static_cast<T*>(t->lam[cur]),
                                  g->stream));
    InitCoef ic;
    if (mrt_init_coef_build(g->b, &ic) != 0) return mrt_fail(MRT_ECUDA, "model blocks singular");
    Coef<T> kc;
    if constexpr (sizeof(T) == 8) kc = g->kd; else kc = g->kf;
    A_TRY(launch_init_adjoint<T>(g->L, ic, kc, static_cast<const T*>(t->lam[cur]), f0, f0 + n, f0 + 2 * n,
                                 f0 + 3 * n, gout, gout + n, gout + 2 * n, gout + 3 * n, g->stream));
    A_TRY(launch_sum_partials(t->gpart, t->nparts, sums, g->stream));
    for (int q = 0; q < 4; ++q)
        if (outs[q])
            A_TRY(cudaMemcpyAsync(outs[q], gout + q * n, sizeof(double) * n,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    double hs[12];
    unsigned flag = 0;
    A_TRY(cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, g->stream));
    A_TRY(cudaMemcpyAsync(&flag, g->flag, sizeof flag, cudaMemcpyDeviceToHost, g->stream));
    A_TRY(cudaStreamSynchronize(g->stream));
    if (flag & FLAG_TIMEOUT) return mrt_fail(MRT_ETIMEOUT, "a device-side wait ran out");
    if (g_s) {
        for (int k = 0; k < 4; ++k) g_s[k] = 0.0;  // conserved moments: no dependence
        for (int k = 0; k < 12; ++k) g_s[4 + k] = hs[k] * g->p.dt;  // sigma_k = s_k dt
    }
    return MRT_OK;
}

extern "C" mrt_status mrt_adjoint_backward(mrt_grid* g, const double* dL_drhoN, int on_device, double* g_rho0,
                                           double* g_ux0, double* g_uy0, double* g_T0, double g_s[16]) {
    NvtxRange range("mrt_adjoint_backward");
    if (!g) return mrt_fail(MRT_EINVAL, "grid is NULL");
    if (!g->tape) return mrt_fail(MRT_EINVAL, "no recorded run: call mrt_adjoint_record first");
    if (!dL_drhoN) return mrt_fail(MRT_EINVAL, "dL_drhoN is NULL");
    double* outs[4] = {g_rho0, g_ux0, g_uy0, g_T0};
    return g->fp64 ? backward_impl<double>(g, dL_drhoN, outs, g_s, on_device)
                   : backward_impl<float>(g, dL_drhoN, outs, g_s, on_device);
}

template <class T>
static mrt_status adjoint_step_impl(mrt_grid* g, const void* f, const void* lam_next, void* lam, int on_device,
                                    double g_s[16]) {
    const size_t sb = 16 * (size_t)g->L.plane * g->elem;
    dim3 agrid, ablock;
    adjoint_grid<T>(g->L, &agrid, &ablock);
    const int nparts = (int)(agrid.x * agrid.y);
    void *bf = nullptr, *bl = nullptr, *bo = nullptr;
    double *gxb = nullptr, *gyb = nullptr, *gpart = nullptr, *sums = nullptr;
    mrt_status st = MRT_OK;
    auto cleanup = [&]() {
        cudaStreamSynchronize(g->stream);
        cudaFree(bf); cudaFree(bl); cudaFree(bo); cudaFree(gxb); cudaFree(gyb); cudaFree(gpart); cudaFree(sums);
    };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&bf, sb)) || (e = cudaMalloc(&bl, sb)) || (e = cudaMalloc(&bo, sb)) ||
        (e = cudaMalloc(&gxb, sizeof(double) * 32 * (size_t)g->L.ny)) ||
        (e = cudaMalloc(&gyb, sizeof(double) * 32 * (size_t)g->L.nx)) ||
        (e = cudaMalloc(&gpart, sizeof(double) * 12 * (size_t)nparts)) || (e = cudaMalloc(&sums, sizeof(double) * 12))) {
        cleanup();
        return mrt_fail(MRT_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    const size_t rowb = (size_t)g->L.nx * g->elem, dp = (size_t)g->L.pitch * g->elem;
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaMemsetAsync(bl, 0, sb, g->stream);
    cudaMemsetAsync(gxb, 0, sizeof(double) * 32 * (size_t)g->L.ny, g->stream);
    cudaMemsetAsync(gyb, 0, sizeof(double) * 32 * (size_t)g->L.nx, g->stream);
    cudaMemsetAsync(gpart, 0, sizeof(double) * 12 * (size_t)nparts, g->stream);
    for (int i = 0; i < 16 && e == cudaSuccess; ++i) {
        const size_t off = ((size_t)i * g->L.plane + g->L.pitch + g->L.G) * g->elem;
        const size_t uoff = (size_t)i * g->L.nx * g->L.ny * g->elem;
        e = cudaMemcpy2DAsync(static_cast<char*>(bf) + off, dp, static_cast<const char*>(f) + uoff, rowb, rowb,
                              g->L.ny, kin, g->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(static_cast<char*>(bl) + off, dp, static_cast<const char*>(lam_next) + uoff, rowb,
                                  rowb, g->L.ny, kin, g->stream);
    }
    if (e != cudaSuccess) { cleanup(); return mrt_fail(MRT_ECUDA, "copy in: %s", cudaGetErrorString(e)); }
    st = mrt_refresh_periodic_ghosts(g, bl);
    if (st != MRT_OK) { cleanup(); return st; }
    AdjArgs<T> a;
    a.L = g->L;
    a.per_x = g->p.bc_x == MRT_BC_PERIODIC;
    a.per_y = g->p.bc_y == MRT_BC_PERIODIC;
    a.lam_in = static_cast<const T*>(bl);
    a.f = static_cast<const T*>(bf);
    a.lam_out = static_cast<T*>(bo);
    a.gxb = gxb;
    a.gyb = gyb;
    a.gpart = gpart;
    if constexpr (sizeof(T) == 8) a.k = g->kd; else a.k = g->kf;
    a.flag = g->flag;
    if ((e = launch_adjoint_step<T>(a, g->xt, g->stream)) == cudaSuccess && g->xt)
        e = launch_ghost_gather_xt<T>(a, g->stream);
    if (e == cudaSuccess) e = launch_sum_partials(gpart, nparts, sums, g->stream);
    for (int i = 0; i < 16 && e == cudaSuccess; ++i) {
        const size_t off = ((size_t)i * g->L.plane + g->L.pitch + g->L.G) * g->elem;
        const size_t uoff = (size_t)i * g->L.nx * g->L.ny * g->elem;
        e = cudaMemcpy2DAsync(static_cast<char*>(lam) + uoff, rowb, static_cast<char*>(bo) + off, dp, rowb, g->L.ny,
                              kout, g->stream);
    }
    double hs[12] = {0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, g->stream);
    cleanup();
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "adjoint step: %s", cudaGetErrorString(e));
    if (g_s)
        for (int k = 0; k < 12; ++k) g_s[4 + k] += hs[k] * g->p.dt;
    return MRT_OK;
}

extern "C" mrt_status mrt_adjoint_step(mrt_grid* g, const void* f, const void* lam_next, void* lam, int on_device,
                                       double g_s[16]) {
    if (!g) return mrt_fail(MRT_EINVAL, "grid is NULL");
    if (!f || !lam_next || !lam) return mrt_fail(MRT_EINVAL, "null state pointer");
    return g->fp64 ? adjoint_step_impl<double>(g, f, lam_next, lam, on_device, g_s)
                   : adjoint_step_impl<float>(g, f, lam_next, lam, on_device, g_s);
}
