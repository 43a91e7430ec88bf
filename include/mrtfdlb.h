/*
 * mrtfdlb.h - C ABI of the GB300 (sm_103a) library for the two-dimensional
 * 16-velocity (D2V16) thermal multiple-relaxation-time finite-difference
 * lattice Boltzmann method of Chen, Xu, Zhang, Li and Succi (arXiv:1004.5442).
 *
 * Method, per time step dt and for every cell (Eq. 3 of the paper):
 *   fhat   = M f                     moments; rows m_1..m_16 (Appendix)
 *   Delta_k = s_k (fhat_k - fhat^eq_k) relaxation with a diagonal S;
 *                                    fhat^eq from rho, j, e (Appendix), with
 *                                    P = rho T, e = b rho T + j^2/rho, R = 1
 *   Omega   = -M^-1 Delta            back to velocity space
 *   f^{n+1} = f + Adv(f) + dt Omega  forward Euler in time; Adv is the
 *                                    Lax-Wendroff operator applied along x and
 *                                    along y (Sect. "Construction of
 *                                    energy-conserving MRT LB model")
 * gamma = (b+2)/b; the velocity set is the D2V16 table of the same section
 * with eta_i = 5/2 on the four unit-speed velocities.
 *
 * Conventions shared by every entry point:
 *   - Fields are row-major [ny][nx], x fastest, cell centres at
 *     ((i+1/2)dx, (j+1/2)dx); dy = dx.
 *   - Distribution arrays exchanged with the caller are [16][ny][nx] in the
 *     grid's precision (float for MRT_FP32, double for MRT_FP64); the
 *     velocity index order is (1,0),(0,1),(-1,0),(0,-1) times 1 and 6, then
 *     (1,1),(-1,1),(-1,-1),(1,-1) times sqrt(2) and 3/sqrt(2).
 *   - The library owns all device state of a grid; the caller owns every
 *     array passed in or out.  Pointers flagged "on device" are CUDA device
 *     pointers of the current device; otherwise host pointers.
 *   - Every call returns an mrt_status; nothing aborts or throws across the
 *     ABI.  mrt_last_error() gives a one-line reason for the last failure of
 *     the calling thread.
 *   - A grid is bound to the device that was current at mrt_create and to the
 *     stream given there; calls that launch work are asynchronous on that
 *     stream, calls that return data to the host synchronise it.  A grid
 *     handle is not thread-safe.
 */
#ifndef MRTFDLB_H
#define MRTFDLB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mrt_status {
    MRT_OK = 0,
    MRT_EINVAL = 1,     /* invalid argument (sizes, rates, states, null) */
    MRT_ENOMEM = 2,     /* device or host allocation failed */
    MRT_ECUDA = 3,      /* a CUDA runtime or driver call failed */
    MRT_EUNSTABLE = 4,  /* the health flag tripped: rho or P non-positive or not finite */
    MRT_ETIMEOUT = 5    /* a bounded device-side wait ran out */
} mrt_status;

typedef enum mrt_precision { MRT_FP32 = 0, MRT_FP64 = 1 } mrt_precision;

/* Boundary treatment of one axis.  MRT_BC_FIXED_EQ: one ghost cell beyond
 * each end holds, for the whole run, the initial f of the adjacent domain
 * cell, i.e. f^eq = M^-1 fhat^eq of its initial state (Sect. (b): boundary
 * nodes set to f^eq).  MRT_BC_REFLECT_FIXED: a reflecting wall at the low
 * end (Sect. (d): the normal velocity is the reverse of the one at the
 * mirror-image interior point) - its ghost holds, at every step, the
 * adjacent cell's f with each velocity mirrored across the wall - and a
 * fixed-equilibrium inflow at the high end. */
typedef enum mrt_bc { MRT_BC_PERIODIC = 0, MRT_BC_FIXED_EQ = 1, MRT_BC_REFLECT_FIXED = 2 } mrt_bc;

/* Step kernel selection: MRT_KERNEL_TMA is the TMA-staged strip kernel,
 * MRT_KERNEL_DIRECT the one-thread-per-cell kernel that reads its stencil
 * straight from global memory, MRT_KERNEL_SPLIT the kernel for small grids
 * that gives each 32-cell row segment four warps, one per velocity group
 * (the cell update's phases split across them, so four times as many warps
 * share the latency of one cell update); an mrt_step of two or more steps on
 * such a grid runs them all in one cooperative launch in which each tile
 * waits (bounded) for its neighbour tiles' previous step instead of a kernel
 * boundary.  MRT_KERNEL_AUTO picks the split kernel for grids of at most
 * 8,192 cells (FP64) or 2,048 cells (FP32), the direct kernel for other FP64
 * grids of fewer than 77,824 cells (its small blocks spread the FP64
 * arithmetic over more SMs), and the TMA kernel otherwise.  All run the same
 * cell arithmetic; results agree to rounding. */
typedef enum mrt_kernel { MRT_KERNEL_AUTO = 0, MRT_KERNEL_TMA = 1, MRT_KERNEL_DIRECT = 2, MRT_KERNEL_SPLIT = 3 }
    mrt_kernel;

/* Space discretisation of the advection term v_ia d_a f_i (Sect.
 * "Construction of energy-conserving MRT LB model": Lax-Wendroff in space,
 * forward Euler in time).  MRT_ADV_LW: the Lax-Wendroff operator applied
 * axis by axis, per axis -(c/2)(f_+ - f_-) + (c^2/2)(f_+ - 2 f + f_-),
 * c = v_a dt/dx (the method's default reading).  MRT_ADV_LW2D: the unsplit
 * two-dimensional Lax-Wendroff operator, which adds to each diagonal
 * velocity the mixed term (c_x c_y / 4)(f_{x+1,y+1} - f_{x+1,y-1} -
 * f_{x-1,y+1} + f_{x-1,y-1}) of the second-order Taylor expansion in time
 * (second order in time for those velocities; the split form is first order
 * there).  Beyond two fixed ends the corner ghost holds the corner cell's
 * initial f.  MRT_ADV_LW2D runs on the direct kernel and on TMA tiles 0, 1,
 * 4, 5, 6 and 7 (tiles 2 and 3 give MRT_EINVAL), forward and in reverse
 * mode; batches take MRT_ADV_LW only. */
typedef enum mrt_advection { MRT_ADV_LW = 0, MRT_ADV_LW2D = 1 } mrt_advection;

typedef struct mrt_params {
    int nx, ny;         /* cells; each >= 3 */
    double dx;          /* cell size (dy = dx), > 0 */
    double dt;          /* time step, > 0 */
    double gamma;       /* specific-heat ratio, > 1; b = 2/(gamma-1) */
    double Pr;          /* > 0: s_8 = s_9 = Pr * s_6 (Pr = s_8/s_6 from Eqs. 12b,d);
                           <= 0: s_8, s_9 taken from s[] as given */
    double s[16];       /* relaxation rates s_1..s_16 in 1/time, finite, >= 0;
                           s_1..s_4 act on conserved moments and have no effect */
    int bc_x, bc_y;     /* mrt_bc per axis */
    int precision;      /* mrt_precision of the stored f and of the arithmetic */
    int kernel;         /* mrt_kernel */
    int tile;           /* TMA kernel variant: 0 = tile 6 when the grid gives
                           every resident CTA at least two 8-row items, else
                           tile 4 (FP32) or 1 (FP64);
                           1..5 = ring depth / store path / CTAs-per-SM choices
                           with one static chunk of rows per CTA; 6, 7 = the
                           variants of 5 and 4 whose CTAs take 8- or 32-row
                           work items (10-row on tile 6 with MRT_ADV_LW2D)
                           from an atomic counter; other values give
                           MRT_EINVAL.  Results do not depend on it. */
    int advection;      /* mrt_advection; 0 (MRT_ADV_LW) for the method's
                           axis-by-axis Lax-Wendroff operator */
} mrt_params;

typedef struct mrt_grid mrt_grid;

/* Create a grid and set f = f^eq(rho, u, T) in every cell (Sect. (b):
 * f^eq = M^-1 fhat^eq, formed in FP64 for FP64 grids; for FP32 grids in
 * double-float arithmetic, about 44 bits, whose FP32 rounding is that of
 * the FP64 value except within about 2^-44 of a rounding boundary).
 * rho, ux, uy, T are [ny][nx] doubles, on the device if fields_on_device,
 * else on the host; host fields are uploaded through a device buffer of
 * 4 nx ny doubles that the grid keeps for mrt_get_macro's host readout.
 * stream is a cudaStream_t (NULL = legacy default stream).  Errors: MRT_EINVAL for nx or ny < 3, dx, dt <= 0,
 * gamma <= 1, a negative or non-finite rate, a null pointer, and for an
 * initial state with rho <= 0, T <= 0 or a non-finite value (checked on the
 * device); MRT_ENOMEM; MRT_ECUDA.  Synchronises the stream once. */
mrt_status mrt_create(const mrt_params *params, const double *rho, const double *ux,
                      const double *uy, const double *T, int fields_on_device,
                      void *stream, mrt_grid **out);

/* Advance nsteps >= 0 time steps (Eq. 3, forward Euler + Lax-Wendroff).
 * Asynchronous.  The conserved totals of the final state are reduced in the
 * same pass (FP64 block partials) and kept for mrt_conserved_totals.  All
 * but the last step of a call are replayed from CUDA graphs of two steps,
 * captured on the first call that needs them (a grid keeps up to four);
 * the results do not depend on it.
 * While the grid's stream is being captured into a caller's CUDA graph, the
 * call instead launches every step directly and reduces the totals on that
 * stream.  Such a graph repeats the captured kernels on the same buffers:
 * replayed on the grid's stream, each replay advances the state by nsteps
 * steps if nsteps is even (the state is back in the buffer it started from;
 * an odd count is not replayable).  Replays may alternate with direct calls
 * of even step counts, which leave the buffers and work counters where a
 * replay expects them.  A captured graph reduces its totals into a slot of
 * its own (scratch it shares with no side-stream reduction), and from the
 * first capture on each totals-producing step stamps its place in the
 * grid's stream order, so the totals readers return those of the latest
 * step, replayed or direct.  The grid's step count advances at capture
 * only.  The totals readers return MRT_EINVAL inside a capture. */
mrt_status mrt_step(mrt_grid *g, long nsteps);

/* Macroscopic fields of the current state: rho = fhat_1, j = (fhat_2,
 * fhat_3), u = j/rho, and T from the closure stated with Eq. 12 (P = rho R T,
 * e = fhat_4 = b rho R T + j^2/rho, R = 1 as in Sect. "Numerical Simulation
 * and Analysis"): T = (e - j^2/rho)/(b rho).  Outputs are [ny][nx] doubles, on the
 * device if dst_on_device (asynchronous on the grid's stream), else on the
 * host (synchronises; through the grid's device buffer of 4 nx ny doubles,
 * allocated by the first host readout unless host fields created the grid).
 * Any output pointer may be NULL to skip it. */
mrt_status mrt_get_macro(mrt_grid *g, double *rho, double *ux, double *uy, double *T,
                         int dst_on_device);

/* Conserved totals sum_cells (rho, j_x, j_y, e) * dx * dy of the current
 * state: the moments fhat_1..4 that the collision leaves unchanged
 * (fhat_k = fhat^eq_k for k <= 4, Sect. "Construction of energy-conserving
 * MRT LB model" and the Appendix rows m_1..m_4), so on a periodic grid they
 * are invariants of the step.  Accumulated in FP64 with a fixed summation
 * order (deterministic).
 * out[4] is host memory; synchronises the grid's stream.  Returns
 * MRT_EUNSTABLE if the health flag has tripped (out is still written). */
mrt_status mrt_conserved_totals(mrt_grid *g, double out[4]);

/* The same totals without waiting.  The library reduces the totals of a
 * step on a side stream of the grid, so the grid's stream goes on with the
 * next steps meanwhile; this call enqueues, behind that reduction, a copy of
 * the current state's totals and health flag word into dst[5], caller-owned
 * page-locked host memory (cudaMallocHost / cudaHostAlloc /
 * cudaHostRegister; pageable memory makes the copy synchronous), and
 * returns at once with *ticket identifying the copy.  dst[0..3] are the
 * totals; dst[4] is the flag word as a double (0: healthy; bit 0: a step
 * met non-positive or non-finite rho or pressure; bit 1: a device-side
 * wait ran out).  dst is valid once mrt_totals_wait(g, *ticket) returns
 * MRT_OK, or once a later mrt_conserved_totals or mrt_destroy returns (a
 * synchronisation of the grid's stream alone does not cover the side
 * stream's copy), and must stay allocated until then.  Steps enqueued
 * after the call do not disturb the copy, so a caller can launch step n+1
 * before it waits for the totals of step n and keep the GPU busy.
 * Errors: MRT_EINVAL (NULL argument, or the grid's stream is being
 * captured), MRT_ECUDA. */
mrt_status mrt_conserved_totals_async(mrt_grid *g, double *dst, long *ticket);
/* Wait until the copy of a ticket has landed.  The grid keeps the last 8
 * tickets' completion markers; waiting on an older ticket waits for a
 * later copy instead (correct, possibly longer).  Errors: MRT_EINVAL
 * (NULL grid, or a ticket that was never issued), MRT_ECUDA. */
mrt_status mrt_totals_wait(mrt_grid *g, long ticket);

/* Copy the raw state f [16][ny][nx] (grid precision) out of / into the grid;
 * for checkpoint/resume and tests.  Host copies synchronise. */
mrt_status mrt_get_f(mrt_grid *g, void *f, int on_device);
mrt_status mrt_set_f(mrt_grid *g, const void *f, int on_device);

/* Save the grid's state to a file and restore it (the paper has no
 * counterpart; for checkpoint and resume of long runs).  The file holds a
 * header (grid size, precision, advection operator, boundary kinds, dx,
 * dt, gamma, the 16 rates as stepped, the step count, the padded layout and
 * an FNV-1a checksum of the payload) and the current distribution buffer in
 * the library's padded layout, fixed-equilibrium ghosts included, so a
 * resumed run continues bit for bit whatever fields the loading grid was
 * created from.  mrt_load requires a grid of the same size, precision,
 * operator, boundary kinds, dx, dt, gamma and rates; it restores the state
 * and the step count (mrt_info), not the health flag or a recorded
 * reverse-mode run.  Both synchronise the grid's stream and stage the state
 * in host memory.  Errors: MRT_EINVAL (NULL argument; a file that cannot be
 * opened, is not a checkpoint of this library, is truncated, fails its
 * checksum or does not match the grid, with the reason in mrt_last_error),
 * MRT_ENOMEM (host staging), MRT_ECUDA. */
mrt_status mrt_save(mrt_grid *g, const char *path);
mrt_status mrt_load(mrt_grid *g, const char *path);

/* Synchronise the grid's stream and report the health flag: MRT_OK,
 * MRT_EUNSTABLE (non-positive or non-finite rho or pressure met by a step),
 * MRT_ETIMEOUT (a device-side wait ran out) or MRT_ECUDA. */
mrt_status mrt_health(mrt_grid *g);

/* Information about a grid: steps taken so far, the element pitch and plane
 * stride of its padded device layout, the step kernel and TMA tile variant
 * in use (any pointer may be NULL). */
mrt_status mrt_info(const mrt_grid *g, long *steps, long *pitch, long *plane_stride,
                    int *kernel_in_use, int *tile_in_use);

/* Reverse mode (adjoint) of the method, for gradients of a loss L(rho_N) of
 * the density after N steps with respect to the initial fields and the 16
 * relaxation rates.  The transpose of one step (Eq. 3, forward Euler +
 * Lax-Wendroff) is, per cell, with lam = dL/df^{n+1} and mu = M^-T lam:
 *   dL/df^n     = lam + Adv^T(lam) - M^T (I - J)^T S mu,
 *   dL/dsigma_k += -mu_k (fhat_k - fhat^eq_k)      (sigma_k = s_k dt),
 * where J = d fhat^eq / d fhat (Appendix equilibria, non-zero only through
 * rho, j, e) and Adv^T is the Lax-Wendroff stencil with c -> -c (the
 * unsplit operator's mixed term is its own transpose).  Fixed
 * ghosts hold the initial f of their cells, so their adjoints are added to
 * dL/df^0 there; f^0 = M^-1 fhat^eq(rho, u, T) is differentiated last.
 *
 * mrt_adjoint_record: sets f = f^eq(rho0, ux0, uy0, T0) (fields [ny][nx]
 * doubles, on the device if on_device), runs nsteps >= 1 steps keeping f
 * every ckpt_every >= 1 steps on the device (memory: ceil(nsteps/ckpt_every)
 * checkpoints + max(ckpt_every - 1, 1) recomputed segment states + 2 adjoint
 * states), and leaves f^N in the grid.  Synchronises once.  With
 * MRT_ADV_LW2D the reverse sweep transposes the unsplit operator.
 *
 * mrt_adjoint_backward: after a record, from dL/drho_N ([ny][nx] doubles)
 * writes dL/drho_0, dL/dux_0, dL/duy_0, dL/dT_0 ([ny][nx] doubles; any may
 * be NULL) and g_s[16] = dL/ds_1..16 (host; g_s[0..3] = 0: those rates act
 * on conserved moments).  Each segment of ckpt_every steps is recomputed
 * from its checkpoint before its reverse sweep.  Gradients are with respect
 * to the 16 rates as used (after the Pr rule of mrt_params).  The first
 * state of a segment is read from its checkpoint in place.  Synchronises.
 *
 * mrt_adjoint_step: one reverse step on caller states f^n and lam_next =
 * dL/df^{n+1} ([16][ny][nx], grid precision), writing lam = dL/df^n and
 * adding dL/ds_k of this step to g_s (fixed-ghost adjoints are not
 * returned).  Allocates its own temporaries; synchronises.
 * Errors: MRT_EINVAL (null pointers, bad counts, backward before record),
 * MRT_ENOMEM, MRT_ECUDA, MRT_ETIMEOUT (backward: a bounded device-side wait
 * of the reverse step ran out). */
mrt_status mrt_adjoint_record(mrt_grid *g, const double *rho0, const double *ux0, const double *uy0,
                              const double *T0, int on_device, long nsteps, int ckpt_every);
mrt_status mrt_adjoint_backward(mrt_grid *g, const double *dL_drhoN, int on_device, double *g_rho0,
                                double *g_ux0, double *g_uy0, double *g_T0, double g_s[16]);
mrt_status mrt_adjoint_step(mrt_grid *g, const void *f, const void *lam_next, void *lam, int on_device,
                            double g_s[16]);

/* Conserved totals sum_cells (rho, j_x, j_y, e) * dx * dy of a state held by
 * the caller on the device, computed without any allocation by the library.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory at the moment they need the totals, such as
 * code inside a framework that owns the device-memory budget through its own
 * pool (an allocation behind its back can fail or break its accounting), or
 * monitoring loops that must not stall on the allocator (cudaMalloc and
 * cudaFree can synchronise the device).
 *   f       device pointer, dense [16][ny][nx] (the layout of mrt_get_f, not
 *           the grid's padded layout), float for MRT_FP32, double for
 *           MRT_FP64; read only.
 *   out     device pointer to 4 doubles owned by the caller; written
 *           asynchronously on `stream` (a cudaStream_t, NULL = legacy stream).
 * Scratch: a fixed 128 KB array in the library's device memory, present on
 * every GPU that loads the library until the process exits.  It limits
 * nx * ny to 67,108,864 cells (8192 x 8192); larger sizes return MRT_EINVAL.
 * The first call on a device looks the array's device address up with
 * cudaGetSymbolAddress while that device is current.  No cudaMalloc,
 * cudaFree or other allocating call is made.  Every call uses the same array: calls whose kernels can run
 * at the same time on the GPU (unordered streams) race and return wrong
 * totals, so order them.  Each call writes every scratch slot it reads, so
 * what an earlier call left behind does not matter.
 * Errors: MRT_EINVAL (NULL f or out, nx or ny < 1, dx not finite and > 0,
 * bad precision, too many cells), MRT_ECUDA. */
mrt_status mrt_conserved_totals_static(const void *f, int precision, int nx, int ny, double dx,
                                       double *out, void *stream);

/* Batched independent grids (many instances of uneven size, gamma, Pr and
 * rates advanced together).  Every time step is one kernel launch covering
 * all instances' work items (instance x 128-column strip x chunk of rows),
 * which one wave of resident CTAs takes, longest first, from an atomic
 * counter; two consecutive steps
 * are captured once in a CUDA graph and replayed.  Each instance is an
 * ordinary FP32 grid with the TMA step kernel; its handle (mrt_batch_grid)
 * serves for readout (mrt_get_macro, mrt_get_f, mrt_conserved_totals,
 * mrt_health) but must not be stepped, re-initialised or destroyed by
 * itself.  Batch work runs on a stream the batch owns; the readout calls
 * synchronise it.  The per-instance step constants live in a table of 256
 * slots per device shared by all live batches.
 *
 * mrt_batch_create: n in 1..256 instances; params[i] as for mrt_create
 * (precision must be MRT_FP32; kernel and tile are overridden), fields
 * rho[i], ux[i], uy[i], T[i] ([ny_i][nx_i] doubles, on the device if
 * fields_on_device).  Errors: MRT_EINVAL, MRT_ENOMEM (also when the
 * constant table is full), MRT_ECUDA.
 * mrt_batch_step: advance every instance nsteps >= 0 steps (asynchronous).
 * mrt_batch_tune: choose the kernel variant (tile 2, 4 or 5, as in
 * mrt_params) and the rows per work item (>= 1; 32 with tile 4 at
 * creation); rebuilds the work list and the graph.  Results do not depend
 * on the choice.
 * mrt_batch_grid: handle of instance i (synchronises the batch stream).
 * mrt_batch_info: instances, tile, rows per item, CTAs and work items.
 * mrt_batch_sync: wait for the batch's work.
 * mrt_batch_stream: the batch's cudaStream_t (owned by the batch; valid
 * until mrt_batch_destroy), for events or waits a caller records on it. */
typedef struct mrt_batch mrt_batch;
mrt_status mrt_batch_create(int n, const mrt_params *params, const double *const *rho,
                            const double *const *ux, const double *const *uy, const double *const *T,
                            int fields_on_device, mrt_batch **out);
mrt_status mrt_batch_step(mrt_batch *b, long nsteps);
mrt_status mrt_batch_tune(mrt_batch *b, int tile, int rows_per_item);
mrt_status mrt_batch_grid(mrt_batch *b, int i, mrt_grid **g);
mrt_status mrt_batch_info(const mrt_batch *b, int *n, int *tile, int *rows_per_item, int *ctas,
                          int *items);
mrt_status mrt_batch_sync(mrt_batch *b);
mrt_status mrt_batch_stream(const mrt_batch *b, void **stream);
void mrt_batch_destroy(mrt_batch *b);

/* Diagnostics of the library itself (no counterpart in the paper).
 *
 * mrt_debug_padding: *nonzero = the number of nonzero words in the columns
 * of the grid's two padded buffers that no kernel may write (left of the
 * left ghost column, right of the right one; zero from creation on): a guard
 * band that counts out-of-bounds writes.  Synchronises the grid's stream.
 * mrt_debug_wait_timeout: launches one thread that waits, with the bounded
 * wait of the TMA kernels, on a barrier nothing completes, and one that
 * waits, with the bounded wait of the split kernel's multi-step launch, on
 * a tile counter nothing raises; after the waits' 2 s limit the grid's
 * timeout flag is set, so the next mrt_health returns MRT_ETIMEOUT (the
 * grid stays flagged).  Allocates the counter (stream-ordered).
 * Asynchronous on the grid's stream.
 * Errors: MRT_EINVAL (null pointers), MRT_ENOMEM, MRT_ECUDA. */
mrt_status mrt_debug_padding(mrt_grid *g, long *nonzero);
mrt_status mrt_debug_wait_timeout(mrt_grid *g);

/* mrt_debug_fma_rate: fused multiply-add throughput of the current device in
 * FP32 or FP64 (precision = mrt_precision), the arithmetic roof of the
 * steps that are bound by the FP64 pipe.  One launch of blocks_per_sm (1..8)
 * blocks of threads_per_block threads (a multiple of 32, at most 1024, at
 * most 2048 per SM) per SM, in which the first active_lanes (1..32) lanes of
 * every warp run 8 independent chains a <- a * 1/2 + 1/2 of 16 * iters
 * multiply-adds each (the other lanes return at once), is timed with CUDA
 * events after one untimed launch of the same shape; *flops_per_s =
 * 2 * multiply-adds / time, *ms (may be NULL) the timed launch's duration.
 * Allocates a small output buffer (stream-ordered) and synchronises.
 * Errors: MRT_EINVAL (an argument out of range, NULL flops_per_s),
 * MRT_ECUDA.
 *
 * mrt_debug_launch_period: the time per launch of a kernel that does
 * nothing, with blocks x threads threads, over nlaunches (even, >= 2)
 * launches in a row on one stream (*us_stream) and as nlaunches/2 replays
 * of a two-launch CUDA graph (*us_graph), CUDA events after one untimed
 * launch; the floor under any step of a small grid.  Synchronises.
 * Errors: MRT_EINVAL, MRT_ECUDA. */
mrt_status mrt_debug_fma_rate(int precision, long iters, int blocks_per_sm, int threads_per_block,
                              int active_lanes, double *flops_per_s, double *ms);
mrt_status mrt_debug_launch_period(int nlaunches, int blocks, int threads, double *us_stream,
                                   double *us_graph);

/* Release every device resource of the grid (synchronises its streams). */
void mrt_destroy(mrt_grid *g);

const char *mrt_status_str(mrt_status s);
const char *mrt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MRTFDLB_H */
