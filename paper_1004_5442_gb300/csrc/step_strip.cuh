// step_strip.cuh - the strip machinery shared by the single-grid and the
// batched step kernels: a ring of TMA-loaded rows in shared memory, the
// per-row cell update, row stores (TMA for whole strips, per thread for a
// ragged strip), periodic ghost refresh, and the bounded-wait bookkeeping.
#pragma once
#include <cstdint>

#include "internal.h"
#include "tma.cuh"

namespace mrt {

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

// CTA-wide FP64 sum of 4 values; thread 0 writes them to dst[0..3].  Lanes
// and warps follow the linear thread index, so 2-D blocks (the direct
// kernel's 32 x BY) reduce correctly.
__device__ __forceinline__ void block_sum4(double v[4], double* dst) {
    __shared__ double red[32][4];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0)
        for (int q = 0; q < 4; ++q) red[warp][q] = v[q];
    __syncthreads();
    if (t == 0) {
        for (int q = 0; q < 4; ++q) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += red[w][q];
            dst[q] = s;
        }
    }
}

// Warp-wide sum of the 4 running totals in a fixed order; lane 8q writes
// moment q to dst[q] as a double.  The first two butterfly levels also
// transpose: across lanes 16 apart a lane keeps two of the four sums and
// hands over the other two, across lanes 8 apart one of its two, and the
// last three levels sum the single value a lane then holds (6 pair
// additions and 12 shuffles per warp instead of 20 and 40).  FP32
// accumulators are combined as (hi, lo) pairs with error-free FP32
// additions (Knuth's TwoSum), which keeps their double-float accuracy
// without FP64 arithmetic: one SM of this part retires only two FP64 lanes
// per clock.
__device__ __forceinline__ void dd_add(float& hi, float& lo, float h2, float l2) {
    const float s = hi + h2;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (h2 - bb);
    lo = lo + l2 + e;
    hi = s + lo;  // renormalise (fast two-sum, |s| >= |lo|)
    lo = lo - (hi - s);
}
__device__ __forceinline__ void warp_sum4(Acc<float> acc[4], double* dst) {
    const unsigned all = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool up16 = lane & 16, up8 = lane & 8;
    float h0 = up16 ? acc[2].hi : acc[0].hi, l0 = up16 ? acc[2].lo : acc[0].lo;
    float h1 = up16 ? acc[3].hi : acc[1].hi, l1 = up16 ? acc[3].lo : acc[1].lo;
    const float g0 = up16 ? acc[0].hi : acc[2].hi, m0 = up16 ? acc[0].lo : acc[2].lo;
    const float g1 = up16 ? acc[1].hi : acc[3].hi, m1 = up16 ? acc[1].lo : acc[3].lo;
    dd_add(h0, l0, __shfl_xor_sync(all, g0, 16), __shfl_xor_sync(all, m0, 16));
    dd_add(h1, l1, __shfl_xor_sync(all, g1, 16), __shfl_xor_sync(all, m1, 16));
    float hi = up8 ? h1 : h0, lo = up8 ? l1 : l0;
    const float gh = up8 ? h0 : h1, gl = up8 ? l0 : l1;
    dd_add(hi, lo, __shfl_xor_sync(all, gh, 8), __shfl_xor_sync(all, gl, 8));
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) dd_add(hi, lo, __shfl_xor_sync(all, hi, o), __shfl_xor_sync(all, lo, o));
    if ((lane & 7) == 0) dst[lane >> 3] = (double)hi + (double)lo;
}
__device__ __forceinline__ void warp_sum4(Acc<double> acc[4], double* dst) {
    const unsigned all = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool up16 = lane & 16, up8 = lane & 8;
    double v0 = up16 ? acc[2].hi : acc[0].hi, v1 = up16 ? acc[3].hi : acc[1].hi;
    v0 += __shfl_xor_sync(all, up16 ? acc[0].hi : acc[2].hi, 16);
    v1 += __shfl_xor_sync(all, up16 ? acc[1].hi : acc[3].hi, 16);
    double v = up8 ? v1 : v0;
    v += __shfl_xor_sync(all, up8 ? v0 : v1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(all, v, o);
    if ((lane & 7) == 0) dst[lane >> 3] = v;
}

template <class T>
__device__ __forceinline__ bool healthy(T rho, T P) {
    // false for NaN, non-positive or infinite values
    return rho > (T)0 && P > (T)0 && rho < (T)INFINITY && P < (T)INFINITY;
}

// Store a cell's 16 outputs and the ghost copies the next step reads: on
// periodic axes column G-1 repeats x = nx-1, column G+nx x = 0, row 0
// y = ny-1, row ny+1 y = 0; behind a reflecting wall (low end) column G-1
// holds x = 0 and row 0 holds y = 0 with each velocity mirrored.
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
    if (L.refl_x && x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) out[i * L.plane + row + L.G - 1] = v[mirror_plane(i, 0)];
    }
    if (L.refl_y && y == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) out[i * L.plane + col] = v[mirror_plane(i, 1)];
    }
}

// Unsplit operator only: the corner ghosts that the step itself refreshes
// (both axes periodic or reflecting), written by the cell whose ghost-column
// copy they repeat along y.  A corner holds what the ghost-row rule gives
// when applied to the ghost column: the wrapped row on a periodic y axis,
// row 0 of the column with mirrored velocities behind a reflecting y wall.
// Corners beyond a fixed end never change (set at creation).  v(i) is the
// cell's output of plane i; planes [i0, i1) are written (a velocity and its
// mirror images share a group of four).
template <class T, class V>
__device__ __forceinline__ void store_corners(T* __restrict__ out, const Layout& L, int per_x, int per_y, int x,
                                              int y, const V& v, int i0 = 0, int i1 = NV) {
    long col = -1;
    bool mx = false;
    if (per_x) col = x == 0 ? L.G + L.nx : (x == L.nx - 1 ? L.G - 1 : -1);
    else if (L.refl_x && x == 0) { col = L.G - 1; mx = true; }
    if (col < 0) return;
    long row = -1;
    bool my = false;
    if (per_y) row = y == 0 ? L.ny + 1 : (y == L.ny - 1 ? 0 : -1);
    else if (L.refl_y && y == 0) { row = 0; my = true; }
    if (row < 0) return;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i < i0 || i >= i1) continue;
        const int j = mx ? (my ? mirror_plane(mirror_plane(i, 1), 0) : mirror_plane(i, 0))
                         : (my ? mirror_plane(i, 1) : i);
        out[i * L.plane + row * L.pitch + col] = v(j);
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

// Shared-memory ring of a strip kernel and its row bookkeeping.  Row indices
// are global over all the work items a CTA processes, so each ring slot's
// mbarrier phases follow one another without re-initialisation.
template <class T>
struct StripRing {
    T* ring;          // NS slots of NV x BOXW
    T* outbuf;        // 2 output rows of NV x TMA_W
    uint64_t* full;   // NS mbarriers
    int base;         // global index of local row 0 of the current item
    int issued;       // thread 0: global rows issued
    int waited;       // thread 0: global rows seen complete (contiguous)
};

// One work item of a strip kernel: columns [x0, x0+TMA_W) and rows
// [y0, y0+nrows) of the field described by L, read through map_in and
// written to out (map_out for whole-strip TMA row stores).  Returns false if
// a bounded wait ran out (the caller drains and flags).
// XT: the unsplit operator (diagonal neighbours).  Row r+1 at x +- 1 comes
// from the ring; row r-1 at x +- 1 from the ring, or with YWIN from
// registers: the diagonal planes' x neighbours of row r, which the cell
// update reads anyway, are kept for the next row.
template <class T, bool TOTALS, int NS, bool TSTORE, bool YWIN, bool XT = false, class CoefT>
__device__ __forceinline__ bool strip_chunk(StripRing<T>& R, const CUtensorMap* map_in, const CUtensorMap* map_out,
                                            const Layout& L, int per_x, int per_y, T* __restrict__ out,
                                            const CoefT& k, int x0, int y0, int nrows, bool& bad, Acc<T>* acc) {
    constexpr bool XW = XT && YWIN;  // diagonal corners of row r-1 in registers
    constexpr int HALO = tma_halo<T>();
    constexpr int BOXW = tma_boxw<T>();
    constexpr uint32_t SLOT_BYTES = (uint32_t)tma_slot_bytes<T>();
    const int tid = threadIdx.x;
    const int nload = nrows + 2;           // local rows 0..nrows+1 = padded rows y0..y0+nrows+1
    const int x = x0 + tid;
    const bool active = x < L.nx;
    const int tma_x = L.G + x0 - HALO;     // 16-byte aligned start column of the load box
    // Row stores by TMA only for whole strips: a TMA store that ends inside a
    // 16-byte chunk can write that whole chunk, which for a ragged last strip
    // holds the right ghost column.  The ragged strip copies its staged row
    // out per thread instead.
    const bool tstore = TSTORE && (x0 + TMA_W <= L.nx);
    T* ring = R.ring;
    uint64_t* full = R.full;
    const int base = R.base;
    auto slot_of = [&](int l) { return (base + l) % NS; };
    auto issue = [&](int l) {
        const int sl = slot_of(l);
        mbar_arrive_expect_tx(&full[sl], SLOT_BYTES);
        tma_load_3d(ring + (size_t)sl * NV * BOXW, map_in, &full[sl], tma_x, y0 + l, 0);
        R.issued = base + l + 1;
    };
    auto wait_row = [&](int l) -> bool {
        const int gl = base + l;
        const bool ok = mbar_wait_bounded(&full[gl % NS], (uint32_t)((gl / NS) & 1));
        if (tid == 0 && ok && gl == R.waited) R.waited = gl + 1;
        return ok;
    };

    if (tid == 0) {
        const int first = min(NS, nload);
        for (int l = 0; l < first; ++l) issue(l);
    }
    bool ok = wait_row(0);
    ok = wait_row(1) && ok;
    if (!YWIN) ok = wait_row(2) && ok;
    const int col = tid + HALO;
    T ym[NV], fc[NV];  // YWIN: rows r-1 (y-moving planes) and r at this column
    T dm[8], dp[8];    // XW: row r-1 at x-1 / x+1 of the diagonal planes 8..15
    T nm[8], np[8];    // XW: row r at x-1 / x+1, captured for the next row
    if (YWIN && ok) {
        const T* s0 = ring + (size_t)slot_of(0) * NV * BOXW;
        const T* s1 = ring + (size_t)slot_of(1) * NV * BOXW;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            if (moves_y<YWIN>(i)) ym[i] = s0[i * BOXW + col];
            fc[i] = s1[i * BOXW + col];
            if (XW && i >= 8) {
                dm[i - 8] = s0[i * BOXW + col - 1];
                dp[i - 8] = s0[i * BOXW + col + 1];
            }
        }
    }
    if (__syncthreads_or(!ok)) return false;
    if (YWIN && tid == 0 && NS < nload) issue(NS);  // row 0 now lives in registers

    // TOTALS: the conserved moments are linear in f, so each thread sums its
    // column's 16 outputs over runs of at most kFoldRows rows in plain
    // arithmetic and folds the moments of those sums into acc (error-free
    // for FP32) at the end of each run: 16 additions per cell instead of
    // the moments and four error-free additions.
    constexpr int kFoldRows = 8;
    T fs[TOTALS ? NV : 1];
    if (TOTALS) {
#pragma unroll
        for (int i = 0; i < NV; ++i) fs[i] = (T)0;
    }

#pragma unroll 2
    for (int r = 1; r <= nrows; ++r) {
        const int y = y0 + r - 1;
        // Out slots alternate on the global row count (base + r), not on r:
        // across an item boundary the first row then uses the slot whose
        // last store the previous row already waited for (bulk_wait_read
        // below), whatever the previous item's height.
        T* ob = R.outbuf + (size_t)((base + r) & 1) * NV * TMA_W;
        if (YWIN) {
            ok = wait_row(r + 1);  // a failed wait is acted on at the barrier below
        }
        if (active && ok) {
            const T* sm = ring + (size_t)slot_of(r - 1) * NV * BOXW;
            const T* sc = ring + (size_t)slot_of(r) * NV * BOXW;
            const T* sp = ring + (size_t)slot_of(r + 1) * NV * BOXW;
            T yp[NV];
            if (YWIN) {
#pragma unroll
                for (int i = 0; i < NV; ++i) yp[i] = sp[i * BOXW + col];
            }
            auto F = [&](int i, int pos) -> T {
                switch (pos) {
                    case C: return YWIN ? fc[i] : sc[i * BOXW + col];
                    case XM: {
                        const T v = sc[i * BOXW + col - 1];
                        if (XW && i >= 8) nm[i - 8] = v;
                        return v;
                    }
                    case XP: {
                        const T v = sc[i * BOXW + col + 1];
                        if (XW && i >= 8) np[i - 8] = v;
                        return v;
                    }
                    case YM: return YWIN ? ym[i] : sm[i * BOXW + col];
                    case YP: return YWIN ? yp[i] : sp[i * BOXW + col];
                    case XPYP: return sp[i * BOXW + col + 1];
                    case XPYM: return XW ? dp[i - 8] : sm[i * BOXW + col + 1];
                    case XMYP: return sp[i * BOXW + col - 1];
                    default: return XW ? dm[i - 8] : sm[i * BOXW + col - 1];
                }
            };
            T o[NV];
            T rho, P;
            cell_update<T, XT>(F, k, o, rho, P);
            if (YWIN) {
#pragma unroll
                for (int i = 0; i < NV; ++i) {
                    if (moves_y<YWIN>(i)) ym[i] = fc[i];
                    fc[i] = yp[i];
                }
            }
            if (XW) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    dm[j] = nm[j];
                    dp[j] = np[j];
                }
            }
            bad |= !(rho > (T)0) | !(P > (T)0);
            if (TSTORE) {
#pragma unroll
                for (int i = 0; i < NV; ++i) ob[i * TMA_W + tid] = o[i];
            } else {
                store_cell<T>(out, L, per_x, per_y, x, y, o);
                if (XT) store_corners<T>(out, L, per_x, per_y, x, y, [&](int j) { return o[j]; });
            }
            if (TOTALS) {
#pragma unroll
                for (int i = 0; i < NV; ++i) fs[i] += o[i];
            }
        }
        if (TOTALS && (r % kFoldRows == 0 || r == nrows)) {
            T q0, q1, q2, q3;
            conserved_moments<T>(fs, q0, q1, q2, q3);
            acc[0].add(q0); acc[1].add(q1); acc[2].add(q2); acc[3].add(q3);
#pragma unroll
            for (int i = 0; i < NV; ++i) fs[i] = (T)0;
        }
        if (tstore) {
            fence_async_shared();                // make this thread's row visible to the TMA engine
            if (tid == 0) bulk_wait_read_all();  // the store from the other out slot has read it
        }
        if (!YWIN) ok = (r + 2 < nload) ? wait_row(r + 2) : true;
        // every thread is done with the slot released below, and the out row
        // is complete
        if (__syncthreads_or(!ok)) return false;
        if (tid == 0) {
            if (tstore) {
                tma_store_3d(map_out, ob, L.G + x0, y + 1, 0);
                if (per_y && y == 0) tma_store_3d(map_out, ob, L.G + x0, L.ny + 1, 0);
                if (per_y && y == L.ny - 1) tma_store_3d(map_out, ob, L.G + x0, 0, 0);
                bulk_commit();
            }
            // without YWIN row r-1 is the oldest row still read; with it, row r
            const int l = YWIN ? r + NS : r - 1 + NS;
            if (l < nload) issue(l);
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
                    out[i * L.plane + c0] = v;
                    if (per_y && y == 0) out[i * L.plane + (long)(L.ny + 1) * L.pitch + L.G + x] = v;
                    if (per_y && y == L.ny - 1) out[i * L.plane + L.G + x] = v;
                }
            }
            if (per_x && (x == 0 || x == L.nx - 1)) {
                // periodic ghost columns are single values: plain stores
                const long gc = (long)(y + 1) * L.pitch + (x == 0 ? L.G + L.nx : L.G - 1);
#pragma unroll 4
                for (int i = 0; i < NV; ++i) out[i * L.plane + gc] = ob[i * TMA_W + tid];
            }
            if (L.refl_x && x == 0) {
                // reflecting wall: the mirrored cell behind it
                const long gc = (long)(y + 1) * L.pitch + L.G - 1;
#pragma unroll 4
                for (int i = 0; i < NV; ++i) out[i * L.plane + gc] = ob[mirror_plane(i, 0) * TMA_W + tid];
            }
            if (L.refl_y && y == 0 && active) {
                // reflecting wall: ghost row 0 is row 0 with mirrored planes
#pragma unroll 4
                for (int i = 0; i < NV; ++i) out[i * L.plane + L.G + x] = ob[mirror_plane(i, 1) * TMA_W + tid];
            }
            if (XT && active) store_corners<T>(out, L, per_x, per_y, x, y, [&](int j) { return ob[j * TMA_W + tid]; });
        }
    }
    if (tstore && tid == 0) bulk_wait_all();
    R.base += nload;
    return true;
}

// After a failed wait: thread 0 waits (bounded) for its loads still in
// flight and for its stores, then flags the timeout.
template <class T, int NS>
__device__ __forceinline__ void strip_drain(StripRing<T>& R, unsigned* flag) {
    if (threadIdx.x == 0) {
        for (int gl = R.waited; gl < R.issued; ++gl) mbar_wait_bounded(&R.full[gl % NS], (uint32_t)((gl / NS) & 1));
        bulk_wait_all();
        atomicOr(flag, FLAG_TIMEOUT);
    }
}

template <class T, int NS, bool TSTORE>
__device__ __forceinline__ StripRing<T> strip_ring_init(unsigned char* smem_raw) {
    constexpr uint32_t SLOT_BYTES = (uint32_t)tma_slot_bytes<T>();
    constexpr uint32_t OUT_BYTES = TSTORE ? (uint32_t)tma_out_slot_bytes<T>() : 0u;
    StripRing<T> R;
    R.ring = reinterpret_cast<T*>(smem_raw);
    R.outbuf = reinterpret_cast<T*>(smem_raw + NS * SLOT_BYTES);
    R.full = reinterpret_cast<uint64_t*>(smem_raw + NS * SLOT_BYTES + 2 * OUT_BYTES);
    R.base = 0;
    R.issued = 0;
    R.waited = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&R.full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    return R;
}


}  // namespace mrt
