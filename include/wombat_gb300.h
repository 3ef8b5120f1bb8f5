/*
 * wombat_gb300.h -- C ABI of the GB300 (sm_103a) WENO-Wombat MHD hot path.
 *
 * The library advances the ideal-MHD equations (Donnert et al. 2018,
 * "Towards Exascale Simulations of the ICM Dynamo with WENO-Wombat",
 * Sec. 2.1) on periodic Cartesian grids:
 *   - fifth-order characteristic WENO flux sweeps along x, y, z (Sec. 2.1,
 *     eq. FWENO with the interpolant phi_N and the Jiang-Shu weights; the
 *     "rotated" sweeps of Sec. 2.2),
 *   - local Lax-Friedrichs splitting per characteristic field (Sec. 2.1),
 *   - constrained transport of the face-centred magnetic field on a
 *     staggered mesh (Sec. 2.1),
 *   - SSP-RK3 stages (or the classic four-stage RK4 of Sec. 2.1),
 *   - a CFL time step and FP64 conserved totals.
 *
 * Conventions (all entry points):
 *   - Every function returns a wb_status; no exception or abort crosses the
 *     ABI.  On failure wb_last_error() returns a message for the calling
 *     thread.
 *   - Host arrays belong to the caller and are copied; device memory is
 *     allocated and owned by the library (released by wb_destroy).
 *   - Work is ordered on the CUDA stream given at wb_init_grid.  Functions
 *     marked "synchronises" wait for that stream before returning.
 *   - Cell arrays use the layout [patch][8][nz][ny][nx] (x fastest), fields
 *     (rho, mx, my, mz, Bx, By, Bz, E), E = p/(gamma-1) + rho|v|^2/2 +
 *     |B|^2/2 (magnetic permeability absorbed).  Face arrays use
 *     [patch][3][nz][ny][nx]: component 0 is b_x on the face (i-1/2, j, k),
 *     1 is b_y on (i, j-1/2, k), 2 is b_z on (i, j, k-1/2).  Each patch is
 *     periodic in every direction, unless wb_grid_desc.links joins patches
 *     into a larger world.  The cell-centred B is always the mean of
 *     the two faces: the B entries of a cell array passed in are ignored and
 *     those returned are recomputed from the faces.
 *   - Values are FP64 at the ABI in every precision mode.
 */
#ifndef WOMBAT_GB300_H
#define WOMBAT_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wb_grid wb_grid;   /* opaque, owned by the library */

typedef enum {
    WB_OK = 0,
    WB_EINVAL = -1,       /* bad argument (null pointer, size, mode)          */
    WB_ECUDA = -2,        /* a CUDA runtime call or kernel launch failed      */
    WB_ENOMEM = -3,       /* device or pinned host allocation failed          */
    WB_ENONFINITE = -4,   /* NaN/Inf or non-positive rho or p in the state    */
    WB_ETIMEOUT = -5,     /* a bounded device wait gave up                    */
    WB_EINTERNAL = -6     /* internal consistency check failed                */
} wb_status;

typedef enum {
    WB_FP64 = 0,          /* whole path in FP64                               */
    WB_FP32 = 1,          /* state and sweeps in FP32; FP64 in the eigenvector
                             normalisation near degenerate points, the CFL
                             reduction and the conserved totals              */
    WB_FP32_LEARNED = 2   /* as WB_FP32, with the nonlinear weights of phi_N
                             from the learned networks (wb_set_mlp) wherever
                             the detectors do not fire                       */
} wb_precision;

typedef enum {
    WB_SSPRK3 = 0,        /* three-stage SSP Runge-Kutta (Shu-Osher form)     */
    WB_RK4 = 1            /* classic four-stage RK4 (Sec. 2.1)               */
} wb_integrator;

typedef struct {
    int npatch;           /* number of patches, 1 <= npatch < 2^24            */
    const int *dims;      /* host, npatch*3 interior sizes (nx, ny, nz), each
                             in [1, 4096]; copied                            */
    double dx, dy, dz;    /* cell sizes (> 0), shared by all patches         */
    double gamma;         /* ratio of specific heats (> 1), e.g. 5/3         */
    int ghost;            /* stencil half-width + 1; must be 3 (WENO5)        */
    int precision;        /* wb_precision                                    */
    int integrator;       /* wb_integrator                                   */
    int emf_mode;         /* 0: edge EMF = 1/2 sum of the 4 face EMFs - 1/4
                             sum of the 4 cell values of -v x B (reduces to
                             the 1-D upwind flux for grid-aligned flow);
                             1: plain mean of the 4 face EMFs               */
    int weights;          /* 0: Jiang-Shu nonlinear weights (Sec. 2.1);
                             1: WENO-Z weights (the alternative Sec. 2.1
                             names); not with WB_FP32_LEARNED              */
    const int *links;     /* NULL: every patch is periodic on itself.
                             Otherwise host, npatch*27 patch indices, copied:
                             links[27 p + 9 (oz+1) + 3 (oy+1) + (ox+1)] is
                             the patch that continues patch p in direction
                             (ox, oy, oz) in {-1,0,1}^3, so patches tile a
                             larger world and read their neighbours' cells
                             in place where Sec. 2.2 fills ghost zones.
                             Checked: entries in [0, npatch), centre entry
                             p, reciprocal, diagonal entries the composition
                             of single-axis moves, equal extents along the
                             axes a link does not cross, and at least 3 cells
                             on both sides of every crossing between two
                             different patches; else WB_EINVAL.  A patch may
                             link to itself along an axis (periodic there).
                             wb_harvest needs links == NULL.               */
} wb_grid_desc;

typedef struct {
    int npatch;
    long long ncells;     /* total cells over all patches                    */
    int precision, integrator, emf_mode;
    long long device_bytes; /* device memory held by the grid                */
    double time;          /* simulated time advanced so far (device dt sum)  */
    long long steps;      /* steps taken                                     */
} wb_grid_info;

/* Create a grid and upload the initial state.
 * d: descriptor (Sec. 2.2 patches of a periodic world grid).  U0: host,
 * cell array as above (B entries ignored).  b0: host, face array; its face
 * divergence is preserved by the constrained transport.  cuda_stream: a
 * cudaStream_t to order all work on, or NULL for a stream the library
 * creates.  out: receives the grid.  Synchronises.
 * Errors: WB_EINVAL for a null pointer, npatch < 1 or >= 2^24, a patch
 * extent outside [1, 4096] or a patch of 2^31 cells or more,
 * ghost != 3, an unknown mode, WENO-Z with learned weights,
 * non-positive dx/dy/dz or gamma <= 1, or an inconsistent link table;
 * WB_ENOMEM; WB_ECUDA. */
int wb_init_grid(const wb_grid_desc *d, const double *U0, const double *b0,
                 void *cuda_stream, wb_grid **out);

/* Replace the state with host arrays of the wb_init_grid layout.  Ordered on
 * the grid's stream.  Page-locked arrays mapped at the same address on the
 * grid's device (cudaHostAlloc memory, e.g. pinned torch tensors) are read
 * in place by the import kernel over the host link, with no staging copy;
 * they must stay valid until the next synchronising call.  Pageable arrays
 * are copied through a device staging buffer and read before the call
 * returns.  The same holds for every state entry point below. */
int wb_set_state(wb_grid *g, const double *U, const double *b);

/* The same in FP32 host arrays, for grids that hold FP32 (WB_FP32,
 * WB_FP32_LEARNED): half the bytes to move, no rounding (the state is FP32).
 * Errors: WB_EINVAL (null argument, an FP64 grid), WB_ECUDA. */
int wb_set_state_f32(wb_grid *g, const float *U, const float *b);

/* Advance nsteps steps of fixed size dt > 0 (Sec. 2.1 scheme; SSP-RK3 or
 * RK4 per the descriptor).  Asynchronous on the grid's stream. */
int wb_step(wb_grid *g, double dt, int nsteps);

/* Advance nsteps steps, each with dt = cfl / max_cells sum_d (|v_d| +
 * c_f,d) / dx_d taken on the device from the step's start state (no host
 * round trip).  0 < cfl.  Asynchronous; a non-finite state is reported by
 * the next synchronising call. */
int wb_step_cfl(wb_grid *g, double cfl, int nsteps);

/* dt = cfl / max_cells sum_d (|v_d| + c_f,d)/dx_d for the current state,
 * FP64 max reduction.  Synchronises.  WB_ENONFINITE if any cell holds
 * NaN/Inf or rho <= 0 or p <= 0. */
int wb_cfl_dt(wb_grid *g, double cfl, double *dt_out);

/* out[q] = sum over all cells of all patches of U_q * dx*dy*dz for the 8
 * cell fields (B = face mean), deterministic FP64 reduction.  Synchronises.
 * Also reports a non-finite state seen by an earlier asynchronous step. */
int wb_conserved_totals(wb_grid *g, double out[8]);

/* Per-step totals: with on != 0 every step (wb_step, wb_step_cfl) also
 * takes the conserved totals of its start state, on a second stream beside
 * the CFL kernel and the first Runge-Kutta stages (joined before the last
 * stage overwrites the state), so they cost little step time.  Synchronises
 * when the setting changes.  Errors: WB_EINVAL, WB_ECUDA. */
int wb_set_step_totals(wb_grid *g, int on);

/* The per-step totals of the last step taken (the state at that step's
 * start; layout as wb_conserved_totals).  Synchronises.  Errors: WB_EINVAL
 * (null argument, per-step totals off), WB_ENONFINITE as wb_cfl_dt. */
int wb_step_totals(wb_grid *g, double out[8]);

/* Face divergence of the magnetic field, the invariant of the constrained
 * transport (Sec. 2.1): out[0] = max over cells of |(bx(i+1)-bx(i))/dx +
 * (by(j+1)-by(j))/dy + (bz(k+1)-bz(k))/dz| (neighbouring faces across patch
 * links or periodic wrap), out[1] = max |b| over the faces, both in FP64.
 * Synchronises.  Errors: WB_EINVAL (null argument), WB_ECUDA. */
int wb_div_b(wb_grid *g, double out[2]);

/* Copy the state to host arrays of the wb_init_grid layout (FP64).
 * Either pointer may be NULL to skip it.  Mapped page-locked arrays are
 * written in place by the export kernel.  Synchronises. */
int wb_get_state(wb_grid *g, double *U_out, double *b_out);

/* wb_get_state in FP32 host arrays for grids that hold FP32 (exact).
 * Synchronises.  Errors: WB_EINVAL (null grid, an FP64 grid), WB_ECUDA,
 * WB_ENONFINITE as wb_get_state. */
int wb_get_state_f32(wb_grid *g, float *U_out, float *b_out);

/* Wait for the grid's stream; reports a non-finite state seen by an earlier
 * asynchronous CFL step. */
int wb_sync(wb_grid *g);

/* Diagnostic: run the sweep along `axis` (0 x, 1 y, 2 z) on the current
 * state and copy its numerical fluxes (Sec. 2.1 eq. FWENO, rotated back to
 * the global frame) to the host.  F_out: host, [7][ncells] FP64 in the
 * cell layout of wb_get_state (patch-major), entry c holding the flux
 * through the lower face of cell c along `axis`; components (rho, mx, my,
 * mz, E, B_t1, B_t2) with (t1, t2) = (y, z), (z, x), (x, y) for axis 0, 1,
 * 2.  Does not change the state.  Synchronises. */
int wb_face_fluxes(wb_grid *g, int axis, double *F_out);

/* Autotuner of the sweep tiles.  A sweep tile is TA interfaces along the
 * axis times 128/TA pencils (one per thread of a block); each axis has
 * WB_NTILE_SHAPE shapes (default first).  At wb_init_grid every patch gets
 * the shape that needs the fewest thread slots for its sizes (a cost model:
 * ragged tiles at patch edges idle threads) and the table is ordered by
 * shape, so that each shape runs as its own launch of one tile per block.
 * The same table unordered runs as one persistent launch per axis whose
 * blocks take tiles of any shape from a work counter (the WENO-Z sweeps
 * always run that way).  wb_autotune measures, for
 * each axis, one sweep of the current state with WB_NTILE_CANDIDATE tables
 * (CUDA events, mean of the second and third of three launches): the
 * cost-model table, each fixed shape everywhere, and the cost-model table
 * ordered by shape (a launch per shape, one tile per block), and keeps the
 * fastest.  ms_out (host, 3 * WB_NTILE_CANDIDATE, may be NULL): the times,
 * per axis [model, shape 0, shape 1, shape 2, model by shape].  Not for
 * WB_FP32_LEARNED grids.  Synchronises. */
#define WB_NTILE_SHAPE 3
#define WB_NTILE_CANDIDATE (WB_NTILE_SHAPE + 2)
int wb_autotune(wb_grid *g, double *ms_out);

/* Installs wb_autotune's candidate table `candidate` (0 <= candidate <
 * WB_NTILE_CANDIDATE, the order of ms_out) on all three axes without timing
 * it; WB_EINVAL outside that range or on a WB_FP32_LEARNED grid.  Every
 * candidate gives the same fluxes: the tiles only regroup the interfaces.
 * Synchronises. */
int wb_set_tiles(wb_grid *g, int candidate);

/* Kernel classes timed by wb_step_profiled. */
enum {
    WB_K_SWEEP_X = 0,     /* x-sweep flux kernel (Sec. 2.1 eq. FWENO)         */
    WB_K_SWEEP_Y = 1,
    WB_K_SWEEP_Z = 2,
    WB_K_UPDATE = 3,      /* flux difference + face -curl E + RK combine      */
    WB_K_CFL = 4,         /* CFL max reduction                                */
    WB_K_DT = 5,          /* dt from the reduced speed                        */
    WB_K_TOTALS = 6,      /* conserved totals (two kernels)                   */
    WB_K_EMF = 7,         /* edge EMFs of constrained transport               */
    WB_NKERNEL = 8
};

/* Measurement helper: advance nsteps CFL steps exactly as wb_step_cfl does,
 * but launch the kernels one by one (no graph) with a CUDA event pair
 * recorded on the grid's stream around every launch; with_totals != 0 adds
 * the conserved-totals reduction after every step.  kernel_ms[k] (host,
 * WB_NKERNEL entries) receives the summed device time of class k,
 * launches[k] its number of launches, *total_ms the device time from the
 * first to the last event.  Synchronises. */
int wb_step_profiled(wb_grid *g, double cfl, int nsteps, int with_totals,
                     double *kernel_ms, int *launches, double *total_ms);

/* Measurement helper, not part of the paper's method: FP32 (precision =
 * WB_FP32) or FP64 (WB_FP64) fused multiply-add throughput of the current
 * device in TFLOP/s, from a kernel of independent FMA chains timed with
 * CUDA events (2 flops per FMA).  Synchronises the device. */
int wb_alu_peak(int precision, double *tflops);

int wb_get_info(wb_grid *g, wb_grid_info *info);

/* Free all device memory of the grid (synchronises first).  NULL is a no-op. */
int wb_destroy(wb_grid *g);

/* Message of the last failing call on this thread ("" if none). */
const char *wb_last_error(void);

/* Conserved totals for callers that cannot allocate device memory.
 *
 * Some callers cannot call cudaMalloc: code that runs under another
 * component's device memory pool (a framework that owns the device's memory
 * and forbids allocations it does not make), or a time-critical loop where
 * the implicit device synchronisation of cudaMalloc/cudaFree is not
 * acceptable.  This entry point computes the same deterministic FP64 sums as
 * wb_conserved_totals, but on a state held in the caller's device memory and
 * without allocating anything: its per-block partial sums live in a
 * file-scope device array of WB_NOALLOC_PARTIALS x 8 doubles (64 KiB), which
 * every GPU that loads the library holds until the process exits.  The paper
 * has no counterpart; it is an interface convenience.
 *
 * state: device, 8 arrays of ncells values, array f at state + f*ncells, in
 *   the order rho, mx, my, mz, E, bx, by, bz (bx/by/bz on the lower faces of
 *   periodic patches, so that their sums equal the sums of the cell means);
 *   element type double for precision WB_FP64, float for WB_FP32.
 * ncells: 1 .. WB_NOALLOC_MAX_CELLS; larger values return WB_EINVAL with a
 *   message.
 * dV: cell volume the sums are multiplied by.
 * out: device, 8 doubles: totals of (rho, mx, my, mz, Bx, By, Bz, E) * dV.
 * cuda_stream: cudaStream_t to order the work on (NULL: the default stream).
 * Asynchronous: out is valid once the stream has been synchronised.
 * Each call looks up the scratch array's device address (cudaGetSymbolAddress)
 * with the current device, so a cudaDeviceReset between calls leaves no
 * stale address; while cuda_stream is being captured the address found by
 * the last call outside capture on that device is used instead, so make the
 * first call on a device (and the first after a cudaDeviceReset) before any
 * stream capture: otherwise WB_EINVAL.  Every call shares the one scratch array, so
 * calls that overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.  Each call rewrites every partial
 * slot it reads, so nothing needs clearing between calls.
 * Errors: WB_EINVAL (null pointer, unknown precision, ncells out of range),
 * WB_ECUDA. */
#define WB_NOALLOC_PARTIALS 1024
#define WB_NOALLOC_MAX_CELLS (1LL << 34)
int wb_conserved_totals_noalloc(const void *state, int precision, long long ncells,
                                double dV, double *out, void *cuda_stream);

/* ---- learned WENO weights ------------------------------------------------
 * One network per characteristic field s = 0..6 (waves u-cf, u-ca, u-cs, u,
 * u+cs, u+ca, u+cf): 6 -> 32 -> 32 -> 3 with GELU (tanh form) and softmax,
 * predicting the weights (w0, w1, w2) that phi_N (Sec. 2.1) uses in place of
 * the Jiang-Shu weights.  Parameters: WB_MLP_NFIELD blocks of WB_MLP_NPARAM
 * floats, each W1 (32x6 row-major), b1, W2 (32x32), b2, W3 (3x32), b3.
 * Training records: WB_MLP_RECORD floats each: field, x[6] (normalised
 * stencil), q[3] (normalised third-order candidate fluxes), T (normalised
 * target reconstruction), flag (non-zero: excluded from training).  The
 * paper has no learned component; this follows the readings recorded with
 * the design notes. */
#define WB_MLP_NFIELD 7
#define WB_MLP_NPARAM 1379
#define WB_MLP_RECORD 12

/* Mean loss per field (loss_out[7]) and its gradient (grad_out[7*1379])
 * over all unflagged records (host arrays), computed on the GPU by the
 * library's forward and backward kernels; loss per record
 * (sum_k w_k q_k - T)^2 + lam * sum_k d_k log(d_k / w_k), d = (0.1,0.6,0.3).
 * Deterministic.  Synchronises. */
int wb_mlp_loss_grad(const float *records, long long n, const float *params,
                     double lam, double *loss_out, float *grad_out);

/* Adam training of all seven networks: `steps` steps, `batch` records per
 * field per step drawn by a counter-based generator from `seed`; params
 * (host, in/out) starts from the given values; loss_history (host,
 * steps*7, may be NULL) receives each step's minibatch loss per field.
 * Synchronises. */
int wb_mlp_train(const float *records, long long n, float *params, int steps,
                 int batch, double lr, double lam, unsigned long long seed,
                 float *loss_history);

/* Training records from the solver's own state: for n sampled interfaces
 * (the lower faces along `axis` of the cells `cells[t]`, host, local indices
 * of patch 0 of an FP64 grid), WB_MLP_NFIELD x 2 records each (field-major,
 * '+' side then '-' side) written to records_out (host, n*14*12 floats).
 * hU, hF (host, n*7 doubles): the exact face reconstructions of the rotated
 * conservative 7-vector (rho, m_n, m_t1, m_t2, B_t1, B_t2, E) and of its
 * physical flux at each sampled face; they give the targets T through the
 * same left eigenvectors and Lax-Friedrichs speeds the sweep uses.
 * kappa, pjump: detector thresholds (records where a detector fires carry
 * flag 1).  Synchronises.  Errors: WB_EINVAL (not FP64, bad axis/sizes). */
int wb_harvest(wb_grid *g, int axis, const long long *cells, long long n,
               const double *hU, const double *hF, double kappa, double pjump,
               float *records_out);

/* The rotated conservative 7-vector X = (rho, m_n, m_t1, m_t2, B_t1, B_t2, E)
 * of every cell of patch 0 of a periodic FP64 grid, and its physical ideal-
 * MHD flux F along `axis` (0 x, 1 y, 2 z; n = axis, t1 = axis+1, t2 =
 * axis+2 mod 3), with the cell field the mean of the cell's two faces
 * (Sec. 2.1: the flux of the state the sweep projects).  X_out, F_out:
 * host, 7 * nx*ny*nz doubles each, field-major, x fastest.  The training
 * pipeline reconstructs the exact face values hU, hF of wb_harvest from
 * them.  Synchronises.  Errors: WB_EINVAL (not FP64, linked grid, bad axis),
 * WB_ECUDA. */
int wb_cell_state_flux(wb_grid *g, int axis, double *X_out, double *F_out);

/* Install the learned-weight networks on a WB_FP32_LEARNED grid (required
 * before its first step).  params: host, WB_MLP_NFIELD * WB_MLP_NPARAM
 * floats (copied, rounded to BF16 for the tensor cores).  kappa: jump
 * detector threshold (the largest of the four differences phi_N reads
 * against kappa times the mean of the other three); pjump: pressure
 * detector (max p > (1 + pjump) min p over the six stencil cells).  Where a
 * detector fires the Jiang-Shu weights are used.  Synchronises. */
int wb_set_mlp(wb_grid *g, const float *params, double kappa, double pjump);

/* Smoothness gate of a WB_FP32_LEARNED grid: the networks' weights are used
 * for a field and side only where its smoothness indicators IS_0..2 (those
 * of the Jiang-Shu weights, Sec. 2.1, on the four differences phi_N reads)
 * spread by more than the ratio `smooth`, (eps + max IS) > smooth (eps +
 * min IS), eps = 1e-6: near critical points of the solution, where the
 * Jiang-Shu weights lose accuracy.  Where the stencil is smoother than that
 * the Jiang-Shu weights (within O(dx^2) of the linear weights there) are
 * kept, so that the network's BF16 rounding does not cap the order of the
 * scheme on smooth flow.  Default 1.03 (the indicators of a field differing
 * by more than 3 %); smooth = 0: the networks wherever no detector fires.
 * Errors: WB_EINVAL (not a learned grid, smooth < 0 or not finite). */
int wb_set_mlp_gate(wb_grid *g, double smooth);

/* Detector log of a WB_FP32_LEARNED grid: out[0] = weight decisions that
 * kept the Jiang-Shu weights (a detector fired, or the smoothness gate of
 * wb_set_mlp_gate held the network back), out[1] = all weight decisions
 * (7 characteristic fields x 2 sides per interface and sweep), counted on
 * the device over every learned sweep since the grid was made or last
 * reset; reset != 0 zeroes the counters afterwards.  Synchronises.
 * Errors: WB_EINVAL (null argument, not a learned grid). */
int wb_learned_stats(wb_grid *g, long long out[2], int reset);

/* Library version string. */
const char *wb_version(void);

#ifdef __cplusplus
}
#endif
#endif
