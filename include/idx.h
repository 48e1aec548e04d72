/*
 * idx.h -- C ABI of the B300 (sm_103a) ideal-MHD Runge-Kutta stage library (libidx.so).
 *
 * One simulation ("sim") is one Cartesian box of ideal MHD (periodic, or with outflow or
 * reflecting boundaries per direction) advanced by the Godunov scheme of the IDEFIX paper
 * (Lesur et al. 2023):
 *   Eqs. (1)-(4)  ideal-MHD conservation laws (units without 4*pi),
 *   Eq. (5)       finite-volume update of cell averages,
 *   Sec. 2.3      PLM reconstruction of the primitives with the van Leer limiter, or the
 *                 compact third-order LimO3 (Cada & Torrilhon 2009);
 *                 HLLD Riemann solver (Miyoshi & Kusano 2005), pressure in the flux;
 *                 HLL or Rusanov selectable,
 *   Sec. 2.4      constrained transport of face-centred B with the E^c edge EMF
 *                 (Gardiner & Stone 2005), Eq. (6); or its vector-potential form,
 *                 Eqs. (7)-(8): an edge potential A stepped with -E, B = curl A,
 *   Sec. 2.7      Runge-Kutta stages U_s = w_s U* + w0_s U_0 (Eq. 9, Table 1: RK2 w = 1, 0;
 *                 1/2, 1/2 -- the default; RK3 w = 1, 0; 1/4, 3/4; 2/3, 1/3) and the CFL
 *                 step dt = sigma / max_V sum_d c_max,d / dl_d (Eq. 10).
 *
 * Layout (every field): double[nz][ny][nx], x fastest, periodic in x, y and z unless
 * idx_grid.bc says otherwise.  The 8 state fields, in this order: rho, mx, my, mz, E
 * (cell averages), then Bx, By, Bz (face averages: Bx[k][j][i] on the x-face at i-1/2,
 * By[k][j][i] on the y-face at j-1/2, Bz[k][j][i] on the z-face at k-1/2).  Along a
 * non-periodic direction the normal field has one more face: Bx is double[nz][ny][nx+1]
 * when x is not periodic (face i = nx is the upper boundary face), and likewise for By, Bz.
 * A direction with a single cell is not integrated (nz == 1 is the 2D case).
 *
 * Time step: the first cycle after idx_set_state / idx_set_primitive takes its dt
 * from a signal-speed pass on the new state; every later cycle takes
 * dt = cfl / inv, where inv is the larger of the two stages' values of
 * max over cells of sum_d max(c at the two d-faces) / dl_d of the previous cycle,
 * with c = max(|S_L|, |S_R|) of the HLLD outer speeds.
 *
 * Return codes: 0 on success, a negative IDX_E* code otherwise (idx_strerror()).
 * Ownership: the library owns all device memory of a sim (allocated in idx_create,
 * freed in idx_destroy); callers own every buffer they pass in, and set/get copy.
 * Threading: a sim is not thread-safe; distinct sims are independent.  All work of
 * a sim runs on its stream (the caller's, or one the library creates).
 */
#ifndef IDX_H
#define IDX_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IDX_OK 0
#define IDX_EINVAL (-1)    /* bad sizes, gamma <= 1, cfl outside (0,1), NULL, unsupported solver */
#define IDX_ENOMEM (-2)    /* device allocation failed                                        */
#define IDX_ENONPHYS (-3)  /* rho <= 0, P <= 0 or non-finite found on the device             */
#define IDX_ECUDA (-4)     /* a CUDA runtime call failed                                      */
#define IDX_ETIMEOUT (-5)  /* a bounded wait expired                                          */

typedef enum {
  IDX_BC_PERIODIC = 0,    /* the default                                                   */
  IDX_BC_OUTFLOW = 1,     /* zero gradient: ghost cells copy the nearest interior cell (the
                             paper's outflow boundary, Sec. 4.1)                           */
  IDX_BC_REFLECTING = 2   /* mirror image about the boundary face with the normal velocity and
                             the normal field reversed (a rigid, perfectly conducting wall) */
} idx_bc;

typedef struct {
  int nx, ny, nz;      /* cells per direction, each >= 1, nx*ny*nz < 2^31 */
  double lx, ly, lz;   /* box [0,lx) x [0,ly) x [0,lz); cell size l/n      */
  int bc[3];           /* boundary kind per direction (idx_bc); a direction with one cell is
                          not integrated and takes none.  A non-periodic direction needs at
                          least 2 cells; it is stepped with 2 ghost cells per side that are
                          refilled from the interior before every stage. */
} idx_grid;

typedef enum {
  IDX_FP64 = 0,       /* every step in FP64                                                  */
  IDX_FP32_BULK = 1   /* reconstruction, HLLD and EMFs in FP32; primitive recovery, the
                         conserved/face-B accumulation and the dt reduction in FP64          */
} idx_precision;

typedef enum {
  IDX_INDUCTION_FIELD = 0,     /* step the face field with the curl of the edge EMFs (Eq. 6)  */
  IDX_INDUCTION_POTENTIAL = 1  /* step an edge vector potential with -E and set the face field
                                  to Bref + curl A every stage (Eqs. 7-8).  Equal to the field
                                  form in exact arithmetic; the discrete divergence of B then
                                  stays at the rounding of one curl instead of accumulating.
                                  Costs 72 B per cell (RK3: 96 B) for Bref and the potentials. */
} idx_induction;

typedef struct {
  int recon;       /* reconstruction of the primitives (Sec. 2.3): 1 = PLM with the van Leer
                      limiter; 3 = LimO3, face value w + phi(t) dw / 2 toward each face with
                      phi(t) = max(0, min(P3, max(-t/2, min(2t, P3, 3/2)))), P3 = (2 + t)/3,
                      t the ratio of the difference behind the cell to the one toward the
                      face (no switch to P3 near smooth extrema).  Both read two cells on
                      each side of a face.                                                  */
  int riemann;     /* Riemann solver (Sec. 2.3): 4 = HLLD, 2 = HLL, 1 = Rusanov (Lax-
                      Friedrichs).  All use the HLLD outer speed estimates for the CFL dt. */
  int emf;         /* 2 = E^c (Sec. 2.4); the only value accepted                          */
  int rk_order;    /* 2 = RK2 or 3 = RK3 (Table 1; RK3 adds a 64 B/cell state buffer)   */
  double cfl;      /* sigma of Eq. (10), 0 < cfl < 1                                       */
  int precision;   /* idx_precision                                                         */
  int induction;   /* idx_induction                                                         */
} idx_solver;

typedef struct idx_sim idx_sim; /* opaque */

/* Create a sim: validates the arguments, allocates its device buffers on the current
 * CUDA device.  stream: a cudaStream_t to run on, or NULL for a library-owned stream.
 * The state is undefined until idx_set_state / idx_set_primitive. */
int idx_create(const idx_grid* grid, double gamma, const idx_solver* solver, void* stream,
               idx_sim** out);

/* Copy in the conserved state (8 fields in the order and layout above).  on_device != 0:
 * the pointers are device memory, else host memory.  Resets t = 0 and the step count and
 * runs the signal-speed pass that fixes the first dt.  Synchronises the sim's stream.
 * IDX_ENONPHYS if the state has rho <= 0, P <= 0 or a non-finite value. */
int idx_set_state(idx_sim* sim, const double* const fields[8], int on_device);

/* Same, from primitives: rho, vx, vy, vz, P (cell centres) and Bx, By, Bz (faces).
 * E = P/(gamma-1) + rho|v|^2/2 + |B_c|^2/2 with B_c the mean of the two faces that
 * bound the cell (the inverse of the primitive recovery). */
int idx_set_primitive(idx_sim* sim, const double* const fields[8], int on_device);

/* Same, with the field given by an edge vector potential (Sec. 2.4, Eq. 8): fields =
 * rho, vx, vy, vz, P (cell centres), then Ax, Ay, Az on the cell edges -- Ax[k][j][i] on
 * the x-edge at (i, j-1/2, k-1/2), Ay at (i-1/2, j, k-1/2), Az at (i-1/2, j-1/2, k)
 * (along a direction with one cell the half offset is void) -- and bmean the uniform
 * part of the field, which a periodic A cannot carry.  The face field is bmean +
 * curl A (circulation over each face / its area; differences along a direction with one
 * cell are dropped), so its discrete divergence vanishes to rounding.  Then as
 * idx_set_primitive.  In the vector-potential form A is kept and Bref = bmean; in the
 * field form A only shapes the initial field.  IDX_EINVAL for NULL or non-finite bmean,
 * and on a grid with a non-periodic direction (the vector-potential form, too, takes
 * periodic grids only: idx_create refuses the combination). */
int idx_set_potential(idx_sim* sim, const double* const fields[8], const double bmean[3],
                      int on_device);

/* Copy out the edge potential of a vector-potential sim (layout of idx_set_potential).
 * After idx_set_state / idx_set_primitive the potential starts at 0 with Bref = the
 * given face field (the gauge A = -integral of E dt from then on).  IDX_EINVAL for a
 * field-form sim.  Synchronises; reports a pending device error. */
int idx_get_potential(const idx_sim* sim, double* const A[3], int on_device);

/* Copy out the conserved state.  Synchronises the sim's stream; reports a pending
 * device error (IDX_ENONPHYS) of earlier asynchronous steps. */
int idx_get_state(const idx_sim* sim, double* const fields[8], int on_device);

/* One RK cycle (its two or three stages with the same dt).  Asynchronous when dt_taken is NULL
 * (errors surface at the next synchronising call); otherwise waits and writes dt. */
int idx_step(idx_sim* sim, double* dt_taken);

/* Cycles until t == t_end; the last dt is clamped to t_end - t and t is then set to
 * t_end exactly.  nsteps (nullable) receives the cycles taken by this call. */
int idx_advance(idx_sim* sim, double t_end, int64_t* nsteps);

/* Current time and the dt the next cycle will take (before any clamp).  Synchronises. */
int idx_time(const idx_sim* sim, double* t, double* next_dt);

/* Cycles taken since the last idx_set_state / idx_set_primitive.  Synchronises. */
int idx_step_count(const idx_sim* sim, int64_t* nsteps);

/* Device bytes idx_create allocates for this grid and precision with RK2 (FP64 432 B per
 * cell, FP32 bulk 304 B per cell on a periodic grid -- 24 B of it the stage-1 face fields
 * of the carried-primitive stages -- and 280 B on a padded one, plus alignment; RK3 adds
 * 64 B per cell and drops those 24 B); no device call.  For admission control. */
int idx_footprint(const idx_grid* grid, int precision, uint64_t* bytes);

/* Device bytes idx_create allocates for this grid and any valid solver (RK order and
 * induction form included); no device call.  IDX_EINVAL for an invalid solver. */
int idx_footprint_solver(const idx_grid* grid, const idx_solver* solver, uint64_t* bytes);

/* Flat index k*ny*nx + j*nx + i of the first (lowest-index) cell found non-physical by
 * the last failing call, or -1. */
int idx_last_error_cell(const idx_sim* sim, int64_t* cell);

/* Time-stepping state of a sim beside its fields, for restart dumps (Sec. 3.3: a dump
 * holds the raw data needed to continue a run).  inv_dt is the inverse CFL time carried
 * from the last cycle, the larger of its stages' max over cells of sum_d c_max,d / dl_d
 * (Eq. 10); the next cycle takes dt = cfl / inv_dt.  Restart: idx_get_state +
 * idx_get_clock on the running sim; idx_create + idx_set_state + idx_set_clock on the new
 * one.  The field-form run then continues bit for bit as if it had not stopped (same
 * device, grid, solver and sweep shapes).  A vector-potential sim restarts its gauge at
 * the given face field (idx_set_state), so it continues to rounding only. */
typedef struct {
  double t;        /* simulated time                                    */
  double inv_dt;   /* carried inverse CFL time (> 0)                    */
  int64_t nsteps;  /* cycles taken since the state was first set        */
} idx_clock;

/* Read the clock.  Synchronises; reports a pending device error. */
int idx_get_clock(const idx_sim* sim, idx_clock* clock);

/* Replace the clock of a sim whose state is set (after idx_set_state, which resets t and
 * the count and fixes inv_dt by a signal-speed pass).  IDX_EINVAL for a non-finite t, an
 * inv_dt that is not a finite positive value, or a negative count.  Synchronises. */
int idx_set_clock(idx_sim* sim, const idx_clock* clock);

/* Device time per launch of each kernel of the stage, averaged over the 2 * reps stages
 * of `reps` cycles launched kernel by kernel with CUDA events between them on the sim's
 * stream: ms[0] primitive recovery, [1] x sweep (PLM + HLLD), [2] y sweep, [3] z sweep,
 * [4] E^c edge EMFs, [5] update (0 for a direction that is not integrated).  With the fused
 * FP32-bulk stage (idx_stage_kernels) ms[5] is the fused kernel and ms[1..4] are 0; with
 * the carried-primitive stages ms[0] is 0 and ms[5] is the update that also forms the next
 * stage's primitives.  The
 * cycles are real: the sim advances by `reps` cycles.  A measurement aid, not part of the
 * method. */
int idx_kernel_times(idx_sim* sim, int reps, double ms[6]);

/* Sweep shape per direction chosen by the autotuner, which runs before a sim's first
 * idx_step / idx_advance (grids of at least 32768 cells; smaller ones march 2 faces per
 * thread, LimO3 16; results are cached per grid, precision and device for the process).
 * A marching sweep too small to give two 256-thread blocks per SM runs smaller blocks
 * (down to 32 threads), so that a small grid spreads over the SMs.  Shapes:
 *   2, 4, 8, 16, 32   one thread marches that many faces of a pencil (loads from HBM);
 *   -1                x only: one warp per 32 cells of an x-row, neighbours by shuffle;
 *   -2                x only: a block stages 32 x-faces of 8 rows (plus periodic halos)
 *                     into shared memory with bulk tensor copies (TMA), one face per
 *                     thread; needs nx % 32 == 0 and ny % 8 == 0;
 *   116, 132          y or z only: a block stages a tile of 32 x-cells by 16 / 32 faces
 *                     (plus a 2-cell periodic halo) into shared memory with bulk tensor
 *                     copies (TMA) and marches it there; needs nx % 32 == 0 and n_d a
 *                     multiple of the tile length;
 *   0                 a direction that is not integrated.
 * With LimO3 (idx_solver.recon = 3) only 16, 32 and the staged y/z tiles 116, 132 are used.
 * Every shape does the same arithmetic per face; results differ between shapes at most by
 * rounding (the compiler may contract products into FMAs differently in each kernel
 * instantiation). */
int idx_sweep_shapes(const idx_sim* sim, int shapes[3]);

/* Fix the sweep shapes (values as above; ignored for a direction that is not integrated)
 * instead of autotuning them.  IDX_EINVAL if a shape is unknown or does not fit the grid
 * (with LimO3, anything but 16, 32, 116 or 132).
 * A measurement and testing aid, not part of the method; call it before stepping. */
int idx_set_sweep_shapes(idx_sim* sim, const int shapes[3]);

/* The FP32-bulk stage as one fused kernel: for every-direction-integrated PLM field-form
 * grids with nx % 32 == 0 and ny % 8 == 0, a CTA stages 32 x 8 tiles of the primitives
 * (with their 2-cell periodic halo) plane by plane into shared memory by bulk tensor
 * copies, forms the x/y/z Riemann fluxes, the E^c EMFs and the update of its cells there,
 * and writes only the new state; the primitive recovery stays a kernel of its own.
 * mode: 0 automatic (the carried-primitive stages where they fit, else the split kernels),
 * 1 the split kernels (primitives, three sweeps, E^c, update), 2 the fused kernel, 3 the
 * carried-primitive stages (IDX_EINVAL for 2 or 3 where they do not fit).  The fused and
 * split kernels do the same arithmetic per face, edge and cell in the same order.
 * The carried-primitive stages (FP32 bulk, RK2, field form, periodic grid) run the three
 * sweeps and E^c as the split kernels do, but each update also recovers the primitives of
 * the state it forms (its cells' upper face fields formed there too), so no stage has a
 * primitive kernel, and the RK2 combine of Eq. 9 is carried as the half sum
 * S = (U^n + U*)/2 = U^n + (dt/2) L(U^n): stage 1 writes S and the face fields of U*,
 * stage 2 forms U^{n+1} = S + (dt/2) L(U*) from S alone.  This changes FP64 rounding order
 * only.  A state that another path changed (a batch's work-list kernels, the split
 * kernels) gets its primitives recovered before the next carried cycle.  A non-physical
 * cell found at the end of a cycle becomes the error of the next cycle, as with the split
 * kernels, whose primitive recovery finds it there.
 * A measurement and testing aid; call it before stepping. */
int idx_set_stage_kernels(idx_sim* sim, int mode);

/* *in_use = the stage kernels the sim runs: 1 split, 2 fused, 3 carried primitives. */
int idx_stage_kernels(const idx_sim* sim, int* in_use);

/* Free the sim and its device memory (and its stream, if the library made it). */
void idx_destroy(idx_sim* sim);

const char* idx_strerror(int code);

/* The bounded mbarrier wait of the TMA-staged sweeps (every device wait of the library is
 * bounded: on expiry the block records IDX_ETIMEOUT in the sim's control block and
 * leaves), run alone in one block of a test kernel on `stream` (NULL: the default
 * stream).  The block announces announce_bytes of transaction bytes on its barrier and
 * issues no copy, so with announce_bytes > 0 the wait expires after limit_ms and the call
 * returns IDX_ETIMEOUT; with 0 the barrier completes at once and it returns IDX_OK.  No
 * copy is ever in flight.  limit_ms in (0, 1000], announce_bytes < 2^20, else IDX_EINVAL.
 * Synchronises the stream.  A testing aid, not part of the method. */
int idx_probe_bounded_wait(void* stream, uint32_t announce_bytes, double limit_ms);

/* Measured throughput of the current device's arithmetic pipes, in operations per
 * second: rates[0] FP64 fused multiply-add, [1] FP64 divide, [2] FP64 square root,
 * [3] FP32 fused multiply-add, [4] FP32 divide, [5] FP32 square root.  Each comes
 * from a short kernel of independent operations timed with CUDA events (a few ms).
 * Not part of the method: it supplies the denominators of the ALU roofline. */
int idx_pipe_rates(double rates[6]);

/* ---- Batched stepping (many independent boxes advanced together) --------------------
 * A batch advances a set of sims together: per RK2 stage each kernel type is launched
 * once over a device work-list of all members, and every member keeps its own grid,
 * state, CFL dt (Eq. 10) and end time.  The arithmetic per cell is that of idx_step (up to
 * the compiler's choice of FMA contractions in each kernel instantiation), so a sim gives
 * the same result, to rounding, alone and in a batch.  The work-list is read at run time, so
 * sims join and leave between steps without re-capturing the batch's CUDA graph.  The
 * sweep shapes are autotuned on the batch when its membership first changes.
 * Members of at least 2^18 cells, and members with RK3, LimO3, the vector-potential form or
 * non-periodic boundaries, run their own (single-sim) kernels inside the batch's cycle; the
 * smaller periodic RK2 PLM field-form members share the work-list kernels.
 * Members must share the batch's precision and device; a member must not be stepped by
 * idx_step/idx_advance, nor read with idx_get_state/idx_time, until idx_batch_poll or
 * idx_batch_remove has synchronised the batch. */
typedef struct idx_batch idx_batch; /* opaque */

/* precision: idx_precision; stream: a cudaStream_t, or NULL for a library-owned one. */
int idx_batch_create(int precision, void* stream, idx_batch** out);

/* Add a sim whose state is set; it will advance until its time reaches t_end (the last dt
 * clamped, as in idx_advance).  Pass t_end = INFINITY for an open-ended member. */
int idx_batch_add(idx_batch* batch, idx_sim* sim, double t_end);

/* Remove a member (waits for the batch's work); it goes back to unclamped idx_step. */
int idx_batch_remove(idx_batch* batch, idx_sim* sim);

/* Enqueue ncycles batched cycles (asynchronous); finished members idle. */
int idx_batch_step(idx_batch* batch, int ncycles);

/* Synchronise the batch and list the members that reached their end time or failed
 * (up to cap of them in finished[]); n_finished and n_active are nullable. */
int idx_batch_poll(idx_batch* batch, idx_sim** finished, int cap, int* n_finished,
                   int* n_active);

/* Sweep shapes chosen by the batch's autotuner (as idx_sweep_shapes). */
int idx_batch_shapes(const idx_batch* batch, int shapes[3]);

/* Fix the batch's sweep shapes instead of autotuning them (values as idx_sweep_shapes; a
 * staged shape 116 / 132 applies to the members whose grids fit its tiles, the others
 * march 16 faces per thread).  IDX_EINVAL for an unknown shape.  A measurement and
 * testing aid, not part of the method. */
int idx_batch_set_shapes(idx_batch* batch, const int shapes[3]);

void idx_batch_destroy(idx_batch* batch);

/* ---- Allocation-free cycle (no counterpart in the paper) -------------------------
 * Some callers cannot call cudaMalloc: code running inside another framework's
 * device-memory pool, under a sandbox or device budget that forbids new device
 * allocations, or on a latency-bound path that must not pay for one.  For them,
 * idx_step_noalloc advances caller-owned device state by one FP64 RK2 cycle (the same
 * kernels as idx_step) without allocating anything: its scratch -- the stage-1 state,
 * primitives, face fluxes, edge EMFs and a control block -- lives in one fixed-size
 * device array inside the library (IDX_NOALLOC_SCRATCH_BYTES), which every GPU that
 * loads the library holds until the process exits.
 *
 *   grid, gamma, cfl  as for idx_create (precision is FP64); periodic in every direction
 *                     (IDX_EINVAL otherwise).
 *   state             8 device pointers on the current device, layout as above, updated
 *                     in place.
 *   inv_dt            host double, in/out: the inverse CFL time carried between calls.
 *                     Pass a value <= 0 on the first call: a signal-speed pass on the
 *                     input state then fixes the first dt, as after idx_set_state.  On
 *                     return it holds the bound for the next call.
 *   dt_taken          nullable host double: the cycle's dt.
 *   stream            cudaStream_t to run on, or NULL for the default stream.
 *
 * Limits and behaviour:
 *   - at most IDX_NOALLOC_MAX_CELLS cells; a larger grid returns IDX_ETOOLARGE;
 *   - the first call on a device looks up the array's device address, with that device
 *     current, and later calls reuse it; the lookup is kept per device and CUDA context
 *     (a context that another framework makes current has its own copy of the array and
 *     gets its own lookup).  Do not call it after a cudaDeviceReset in the same process:
 *     a cached address belongs to the context that the reset destroyed;
 *   - the call reads back dt and the error flag and waits for its stream, which a graph
 *     capture cannot record: never issue it on a stream that is capturing (IDX_EINVAL);
 *   - every call shares the one array, which keeps the last call's contents (the call
 *     clears what must start at zero): calls that overlap on the GPU race, so issue
 *     them one at a time (same stream, or synchronise between streams and devices
 *     sharing a process);
 *   - it returns when its stream has finished the cycle; IDX_ENONPHYS as for idx_step. */
#define IDX_ETOOLARGE (-6)                      /* grid exceeds a fixed-size buffer */
#define IDX_NOALLOC_SCRATCH_BYTES (64u << 20)   /* 64 MiB per GPU                   */
#define IDX_NOALLOC_MAX_CELLS 195072            /* 256 + 43 x align256(8 n) <= 64 MiB */
int idx_step_noalloc(const idx_grid* grid, double gamma, double cfl, double* const state[8],
                     double* inv_dt, double* dt_taken, void* stream);

#ifdef __cplusplus
}
#endif
#endif
