/*
 * mhd.h -- C ABI of libmhd.so, the GB300 (sm_103a) implementation of one time step of the MHD +
 * H/H2 chemistry method of Kulikov, Chernykh & Protasov, "A new code for numerical simulation of
 * MHD astrophysical flows with chemistry" (arXiv:1608.08748).
 *
 * One call of mhd_step() advances the state by one step of the operator-split scheme of Sec. 2:
 *   tau from the CFL rule (Sec. 2.3) -> Eulerian stage, three SSP-RK3 substages (Sec. 2.2) of the
 *   characteristic Riemann solver on piecewise-parabolic data (Sec. 2.1, 2.4, App. A) with Flux-CT
 *   inside each substage (Sec. 2.5, App. C) -> Lagrangian advection stage, three SSP-RK3 substages
 *   (Sec. 2.6) -> H/H2 chemistry (Sec. 2.7, App. D reactions 1-4; 1-8 with H+ and electrons when
 *   MHD_OPT_IONS is on) -> heating/cooling when on (Sec. 2.8) -> regularisation (Sec. 2.9).
 * Every step runs in CUDA kernels of this library; there is no CPU path.
 *
 * Conventions
 *   Grid: nx * ny * nz cells of width dx on every axis.  Fields are C-order arrays [k][j][i]
 *   (x fastest), nx*ny*nz elements each.  Boundaries are periodic unless set to outflow
 *   (zero-gradient) per axis with mhd_set_option.
 *   Code units: the closure has no 4 pi (total pressure p + B^2/2, energy rho eps + rho v^2/2 +
 *   B^2/2, Sec. 2).  With chemistry on, rho is in m_H cm^-3, lengths in pc, velocities in km/s.
 *   Magnetic field: the library stores face-centred b_x(i-1/2,j,k), b_y(i,j-1/2,k),
 *   b_z(i,j,k-1/2) (Sec. 2.5); cell-centred B is the mean of the two faces.
 *   Ownership: the library allocates and owns all device memory of a simulation; buffers passed in
 *   are only read or written during the call and never retained.
 *   Errors: every int-returning call returns MHD_OK (0) or a negative MHD_E* code; mhd_last_error()
 *   returns a message for the last failure on the calling thread.
 *   Threading: one mhd_sim must not be used from two threads at once; distinct sims are
 *   independent.  All work of a sim is issued on its CUDA stream (mhd_set_stream).
 */
#ifndef MHD_H
#define MHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum mhd_status {
  MHD_OK = 0,
  MHD_PENDING = 1,       /* serving: request not finished yet */
  MHD_EINVAL = -1,       /* bad argument or option */
  MHD_ENOMEM = -2,       /* device allocation failed */
  MHD_ECUDA = -3,        /* a CUDA call failed (message in mhd_last_error) */
  MHD_ENONPHYS = -4,     /* rho <= 0, rho eps <= 0 or a non-finite value after a step (Sec. 2 closure);
                            the state is left as the failing step produced it */
  MHD_ETIMEOUT = -5,     /* a bounded wait gave up */
  MHD_ENOTFOUND = -6,    /* serving: unknown request id */
  MHD_ECAPACITY = -7,    /* serving: request can never fit the memory budget */
  MHD_ECANCELED = -8     /* serving: the request was cancelled (mhd_cancel) */
};

enum mhd_option {
  MHD_OPT_BC_X = 1,          /* 0 periodic (default), 1 outflow (zero-gradient ghost cells/faces) */
  MHD_OPT_BC_Y = 2,
  MHD_OPT_BC_Z = 3,
  MHD_OPT_CHEM = 4,          /* 0 off (scalar gamma), 1 H/H2 network of App. D reactions 1-4 with
                                gamma_eff = (5 n_H + 7 n_H2) / (3 n_H + 5 n_H2) (Sec. 4.3) */
  MHD_OPT_PRECISION = 5,     /* 0 FP64 throughout (default); 1 FP32 bulk (reconstruction, fluxes,
                                updates, state) with FP64 CFL reduction, chemistry and sums */
  MHD_OPT_REGUL_MODE = 7,    /* Sec. 2.9: 0 rho eps := max(rho eps, rho E - rho v^2/2 - B^2/2) where
                                the thermal fraction f >= 1e-3 (default); 1 unconditional overwrite;
                                2 the sentence's literal branch order */
  MHD_OPT_CHEM_LSHIELD = 8,  /* shielding length for column densities N = n L, code length units
                                (0: one cell, the default) */
  MHD_OPT_CHEM_BDOP = 9,     /* Doppler parameter b of f_shield in km/s (default 3) */
  MHD_OPT_CHEM_XNORM = 10,   /* N_H2 normaliser of f_shield in cm^-2 (default 5e14) */
  MHD_OPT_CHEM_TAUD = 11,    /* dust optical depth per unit column, cm^2 (default 1e-21) */
  MHD_OPT_GRAPH = 14,        /* 1 (default): replay each step from a captured CUDA graph; 0: launch */
  MHD_OPT_HEATCOOL = 15,     /* 0 off (default); 1 the Sec. 2.8 heating/cooling stage after the
                                chemistry (needs MHD_OPT_CHEM = 1): rho E and rho eps change by
                                tau (Gamma_1 + Gamma_4 - Lambda_2 - Lambda_3) of App. D, FP64, the
                                change limited to at most half of rho eps */
  MHD_OPT_GRAV_G = 16,       /* gravitational constant G in code units (0: no self-gravity, the
                                default; 1.0635e-4 is G in pc, km/s, m_H cm^-3).  Each step first
                                solves the Poisson equation of Sec. 2.10 for the density (27-point
                                scheme in harmonic space, cuFFT, periodic boundaries required) and
                                the Eulerian stage adds -rho grad Phi and -rho v . grad Phi (central
                                differences).  Such a sim steps without graph capture and cannot
                                join a batch. */
  MHD_OPT_IONS = 17,         /* 0 off (default); 1 reactions 5-8 of Sec. 4.3 / App. D with H+ and
                                electrons (needs MHD_OPT_CHEM = 1): one more advected density
                                rho_H+ = n_H+ (code density units; n_e = n_H+, neutral
                                n_H = rho - rho_H2 - rho_H+), gamma_eff counting H, H+ and e as
                                monatomic particles, and the creation k5 n_H + k6 n_H n_e and
                                destruction (k7 n_e + k8 n) n_H+ of H+ by the semi-implicit
                                update of Sec. 2.7 with rates frozen at the stage start, H2
                                first.  With MHD_OPT_HEATCOOL, Gamma_5 - Lambda_6 - Lambda_7 -
                                Lambda_8 join the heating/cooling.  mhd_set_state zeroes rho_H+;
                                mhd_set_ions loads it. */
  MHD_OPT_X_STAGE = 18       /* 0 (default): the FP32-bulk x sweep reads its pencils' cells from
                                global memory; 1: it brings the six window primitives of its rows
                                into shared memory by bulk asynchronous copies where every box's
                                nx is a multiple of 4 (the results are the same bit for bit; on
                                GB300 this measured slower, since the shared memory takes L1
                                capacity from the sweep's other, strided loads).  A batch stages
                                only if all its members ask for it. */
};

enum mhd_dtype { MHD_F64 = 0, MHD_F32 = 1 };

/* Field set for set/get.  All pointers host or all device (on_device), dtype MHD_F64 or MHD_F32.
   mom and B are three arrays each (x, y, z); B is cell-centred.  rho_h2 may be NULL (then zero on
   input, skipped on output).  Host arrays that are page-locked (cudaMallocHost, cudaHostAlloc,
   cudaHostRegister of the whole array) are read and written in place by the load and store
   kernels (over NVLink-C2C on GB300); pageable ones go through a device staging copy. */
typedef struct mhd_fields {
  void* rho;
  void* mom[3];
  void* E;
  void* B[3];
  void* rho_h2;
  int dtype;
  int on_device;
} mhd_fields;

/* FP64 diagnostics (deterministic fixed-tree sums over all cells) */
typedef struct mhd_diag {
  double sum_rho, sum_mom[3], sum_E, sum_b[3]; /* sum_b over the stored faces */
  double max_div_b_h;   /* max over cells of |sum_d (b_d(i_d + 1/2) - b_d(i_d - 1/2))| = h |div b| */
  double t;             /* simulated time */
  double tau_next;      /* tau / CFL of the current state: dx / max denominator (Sec. 2.3) */
  int64_t steps;        /* steps taken since the last set_state */
  int64_t vel_branch;   /* cells that took the velocity branch of the regularisation, cumulative */
  int32_t error_flags;  /* bit 0: non-physical state seen by the last step's checks; bit 1: tau <= 0;
                           bit 2: a bulk copy of the FP32 x sweep's rows into shared memory did not
                           complete within its bounded wait (the kernel left the step; MHD_ECUDA) */
} mhd_diag;

typedef struct mhd_sim mhd_sim;

/* Create a simulation of nx*ny*nz cells of width dx with adiabatic index gamma (used when
   chemistry is off).  Allocates all device memory on the current CUDA device.  NULL on error. */
mhd_sim* mhd_create(int nx, int ny, int nz, double gamma, double dx);
void mhd_destroy(mhd_sim* s);
const char* mhd_last_error(void);

int mhd_set_option(mhd_sim* s, int key, double value);
/* Issue all work on this cudaStream_t (default: a stream the library creates). */
int mhd_set_stream(mhd_sim* s, void* cuda_stream);

/* Load a cell-centred state (Sec. 2 closure).  Faces are built as the mean of the two
   neighbouring cell values; rho eps = rho E - |m|^2 / (2 rho) - |B_cell(faces)|^2 / 2.
   Resets t and the step counter and computes the first tau. */
int mhd_set_state(mhd_sim* s, const mhd_fields* in);
/* Load exact face values (e.g. a divergence-free field): b_d at face i_d - 1/2, float64, C order;
   recomputes rho eps from rho E with the new field. */
int mhd_set_face_B(mhd_sim* s, const double* bx, const double* by, const double* bz, int on_device);
/* Copy the state out into caller buffers (B cell-centred). */
int mhd_get_state(mhd_sim* s, mhd_fields* out);
/* Full state for checkpoint/resume: rho eps and the face fields (float64). */
int mhd_get_full(mhd_sim* s, double* eint, double* bx, double* by, double* bz, int on_device);
int mhd_set_full(mhd_sim* s, const double* eint, const double* bx, const double* by,
                 const double* bz, int on_device);

/* rho_H+ (float64, C order, nx*ny*nz values, host or device per on_device) in and out.  Set after
   mhd_set_state (which zeroes it); recomputes the first tau.  Used by the steps only with
   MHD_OPT_IONS on.  MHD_EINVAL for a null pointer or (set) no loaded state. */
int mhd_set_ions(mhd_sim* s, const double* rho_hp, int on_device);
int mhd_get_ions(mhd_sim* s, double* rho_hp, int on_device);

/* One full step with tau = CFL-limited (Sec. 2.3).  dt_taken may be NULL: then the call only
   enqueues work and does not synchronise.  Every step copies its error flags to a host-mapped word
   when it finishes, so such a call first returns MHD_ENONPHYS (or MHD_EINVAL for tau <= 0) if a
   step that has finished on the device by then flagged a non-physical state; a flagged step still
   in flight surfaces at a later mhd_step or at the next synchronising call (mhd_sync,
   mhd_diagnostics, mhd_step with dt_taken).  With dt_taken != NULL it waits for the step and
   reports MHD_ENONPHYS.  A bulk copy that did not complete in a step's bounded wait is reported the
   same way, as MHD_ECUDA. */
int mhd_step(mhd_sim* s, double cfl, double* dt_taken);
/* Steps until t_end (the last step truncated to t_end) or max_steps. */
int mhd_advance(mhd_sim* s, double cfl, double t_end, int max_steps, int* steps_done);
/* Wait for all queued work of this sim; returns MHD_ENONPHYS if a step flagged it. */
int mhd_sync(mhd_sim* s);
int mhd_diagnostics(mhd_sim* s, mhd_diag* out);

/* One stage alone with a given tau (per-stage parity checks): 1 Eulerian + Flux-CT, 2 Lagrangian,
   3 chemistry, 4 regularisation, 5 heating/cooling (with MHD_OPT_HEATCOOL on). */
int mhd_stage(mhd_sim* s, int which, double tau);

/* The gravitational potential of the current density (Sec. 2.10, MHD_OPT_GRAV_G > 0): nx*ny*nz
   doubles in C order [k][j][i], host or device pointer, owned by the caller.  MHD_EINVAL when
   self-gravity is off, no state is loaded or a boundary is not periodic. */
int mhd_get_potential(mhd_sim* s, double* out);

/* Kernel classes reported by mhd_profile (index into its output arrays). */
enum mhd_kernel_class {
  MHD_K_PRIM = 0,        /* primitives of every cell (Eulerian substage) */
  MHD_K_EULER_FACE = 1,  /* Eulerian face Riemann solve, all three directions */
  MHD_K_EDGES = 2,       /* App. C edge EMFs */
  MHD_K_EULER_UPDATE = 3,/* finite-volume + Flux-CT + RK update */
  MHD_K_LAG_FACE = 4,    /* Lagrangian face fluxes, all three directions */
  MHD_K_LAG_UPDATE = 5,  /* Lagrangian update (first and second substages in a step) */
  MHD_K_POST = 6,        /* the third substage's Lagrangian update with the chemistry, regularisation
                            and CFL of the new state (one kernel in a step; the post stage alone for
                            mhd_stage and after a load) */
  MHD_K_SMALL = 7,       /* single-thread bookkeeping kernels (step begin and end) */
  MHD_K_NCLASSES = 8
};

/* Run `steps` full steps launch by launch (no graph) with a CUDA event pair around every kernel on
   the sim's stream; out_ms[c] = total milliseconds of class c over the steps, out_launches[c] = its
   number of launches.  The steps advance the state like mhd_step.  Arrays have MHD_K_NCLASSES
   entries. */
int mhd_profile(mhd_sim* s, double cfl, int steps, double* out_ms, int64_t* out_launches);
/* Number of kernel launches in one mhd_step (the first update of each stage stores its RK register,
   so no copy kernels). */
int mhd_launches_per_step(mhd_sim* s);

/* ---- Batched execution (many boxes, one launch per kernel class) ------------------------------
   A batch advances several simulations together: every kernel of the step is launched once over
   a table of tiles that covers all their boxes (uneven sizes allowed), and the step is captured in
   one CUDA graph.  Each box keeps its own tau (its own CFL reduction, Sec. 2.3) and its own device
   memory; per-cell arithmetic does not depend on the batch, so a batched box evolves bit for bit
   like the same box stepped alone.  All sims of a batch must have a loaded state, the same
   precision and the same device.  The batch issues work on its own stream: call mhd_batch_sync
   before using a member sim on its own again.  A sim may belong to several batches but must not
   be stepped by two of them at once. */
typedef struct mhd_batch mhd_batch;
mhd_batch* mhd_batch_create(mhd_sim* const* sims, int n);  /* NULL on error (mhd_last_error) */
void mhd_batch_destroy(mhd_batch* b);
/* One step of every member (tau per member from its own state). */
int mhd_batch_step(mhd_batch* b, double cfl);
/* Wait for the batch's work; MHD_ENONPHYS if any member flagged a non-physical state. */
int mhd_batch_sync(mhd_batch* b);
/* Non-blocking: MHD_PENDING while the batch's work is still queued or running, else as
   mhd_batch_sync. */
int mhd_batch_query(mhd_batch* b);
/* Issue the batch's work on a stream of the device's highest (high = 1) or lowest (0, the
   default) priority: where batches of both kinds are in flight, the block scheduler starts the
   high-priority batch's blocks first as SMs free up. */
int mhd_batch_set_priority(mhd_batch* b, int high);
/* Autotune the launch shape (threads per tile, grid size) of every kernel class on this batch by
   timing `reps` full steps per candidate; the members' states are restored afterwards, so tuning
   changes no results.  best_ms (may be NULL) receives the tuned per-step time. */
int mhd_batch_tune(mhd_batch* b, double cfl, int reps, double* best_ms);
/* Launch shape of one kernel class (MHD_K_PRIM .. MHD_K_POST of mhd_profile; MHD_K_SMALL has no
   shape and gives MHD_EINVAL): threads per tile (64, 128, 256 or 512) and grid = grid_mult x SMs
   (0: one block per tile). */
int mhd_batch_get_shape(mhd_batch* b, int kernel_class, int* block, int* grid_mult);
int mhd_batch_set_shape(mhd_batch* b, int kernel_class, int block, int grid_mult);
/* Per-class CUDA-event timings of `steps` batch steps (as mhd_profile). */
int mhd_batch_profile(mhd_batch* b, double cfl, int steps, double* out_ms, int64_t* out_launches);

/* ---- Serving: continuous batching of simulation requests -------------------------------------
   A server owns a scheduler thread.  Requests (a grid, an initial state and a number of steps)
   wait in arrival order; a request is admitted when its device memory (mhd_bytes_needed) fits in
   the remaining HBM budget and fewer than max_active are running.  The admitted requests of one
   precision and size lane (mhd_server_set_bulk_cells) advance together, one step per batched launch
   per kernel class (their work overlaps on the device), each lane on a stream of its own priority
   and as soon as its previous step has finished; a request that has taken its steps is copied back to
   host memory and its device memory released, which admits waiting requests.  A request's result
   is the same as running it alone (bit for bit).  A request whose device memory cannot be had when
   it is admitted (mhd_create fails) ends with that error (MHD_ENOMEM for a failed allocation) and
   gives its budget back; the server carries on.  Every server call is thread-safe. */
typedef struct mhd_server mhd_server;

typedef struct mhd_request {
  int nx, ny, nz;
  double gamma, dx;
  int precision;       /* 0 FP64, 1 FP32 bulk */
  int chem;            /* H/H2 network on */
  int bc[3];           /* per axis: 0 periodic, 1 outflow */
  double cfl;
  int nsteps;          /* steps to take (> 0) */
  mhd_fields state;    /* initial state, host pointers (copied by mhd_submit; not retained) */
} mhd_request;

typedef struct mhd_result {
  int status;          /* MHD_PENDING while queued or running, then MHD_OK or an error */
  int64_t steps_done;
  double t;            /* simulated time reached */
  double t_submit, t_admit, t_done;  /* seconds on the server's monotonic clock */
  int64_t cells;
} mhd_result;

/* hbm_budget_bytes: device memory the admitted requests may use together; max_active >= 1. */
mhd_server* mhd_server_create(size_t hbm_budget_bytes, int max_active);
/* Admission order of waiting requests: MHD_SERVE_FIFO (the default; the oldest waits until it
   fits) or MHD_SERVE_SMALLEST_WORK (among the requests that fit, the fewest cell-updates,
   cells x steps, first).  Results do not depend on the policy, only their latencies. */
enum mhd_serve_policy { MHD_SERVE_FIFO = 0, MHD_SERVE_SMALLEST_WORK = 1 };
int mhd_server_set_policy(mhd_server* srv, int policy);
/* Stops the scheduler after the running step; unfinished requests are dropped. */
void mhd_server_destroy(mhd_server* srv);
/* >= 0: request id; < 0: MHD_EINVAL, or MHD_ECAPACITY if it can never fit the budget. */
int64_t mhd_submit(mhd_server* srv, const mhd_request* req);
/* Non-blocking: MHD_PENDING, MHD_OK (result ready), MHD_ENOTFOUND, or the request's error. */
int mhd_poll(mhd_server* srv, int64_t id, mhd_result* out);
/* Copy a finished request's state into `out` (host pointers; B cell-centred) and release it. */
int mhd_fetch(mhd_server* srv, int64_t id, mhd_fields* out);
/* Wait (up to timeout_s seconds) until every submitted request has finished: MHD_OK or
   MHD_ETIMEOUT. */
int mhd_server_drain(mhd_server* srv, double timeout_s);
/* Cancel a request.  A waiting request leaves the queue at once; a running one is retired at the
   end of the scheduler's current batched step (its device memory released, no result kept).  Its
   status becomes MHD_ECANCELED (mhd_poll, mhd_fetch).  Returns MHD_OK, MHD_ENOTFOUND for an
   unknown id, or MHD_EINVAL if the request has already finished. */
int mhd_cancel(mhd_server* srv, int64_t id);
/* Pause (paused = 1) or resume (0) admission: while paused no waiting request is admitted;
   running requests keep stepping.  For maintenance and draining. */
int mhd_server_pause(mhd_server* srv, int paused);
/* Requests of at least `cells` cells (default 16,777,216, i.e. 256^3) form the bulk lane: they are
   batched apart from the smaller ones and step on a low-priority stream, while the smaller ones
   step on a high-priority stream, each group as soon as its previous step has finished.  A large
   box then shares the GPU with the small requests instead of setting the pace of their steps.
   Applies to requests admitted afterwards.  MHD_EINVAL for cells < 1. */
int mhd_server_set_bulk_cells(mhd_server* srv, int64_t cells);
/* Change the HBM budget.  Waiting requests that can no longer ever fit fail with MHD_ECAPACITY;
   running requests are not disturbed, and a budget below what they use only holds back further
   admissions until they finish.  MHD_EINVAL for a zero budget. */
int mhd_server_set_budget(mhd_server* srv, size_t hbm_budget_bytes);
/* Server clock now (same clock as the result times). */
double mhd_server_clock(mhd_server* srv);
/* Scheduler statistics: iterations (batched steps), peak bytes admitted, peak active requests. */
int mhd_server_stats(mhd_server* srv, int64_t* iterations, int64_t* peak_bytes, int* peak_active);

/* FP64 diagnostics of caller-owned device arrays without any device allocation.  (The paper has
   no counterpart: this is a service of the library.)  It is for callers that cannot allocate
   device memory at the point of the call: code running while a stream is captured into a CUDA
   graph in global capture mode (cudaMalloc/cudaFree are illegal there), serving processes whose
   HBM budget is fully committed to resident state, and monitors inside another application's
   time loop that must not touch its allocator.
   Inputs: rho, mx, my, mz, E (cells) and bx, by, bz (b_d at face i_d - 1/2) as device float64
   arrays of nx*ny*nz elements, C order; bc_x/y/z 0 periodic or 1 outflow (for the upper faces of
   the divergence).  Output: out, a device pointer to 9 doubles, filled with sum rho, sum m_x,
   sum m_y, sum m_z, sum rho E, sum b_x, sum b_y, sum b_z and max |sum_d (b_d(i_d+1/2) -
   b_d(i_d-1/2))|: the same values, with the same reduction order, as mhd_diagnostics.
   The work is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream) and the call
   returns without waiting.  The block partials live in one fixed device array of
   MHD_NOALLOC_MAX_CELLS / 256 * 9 doubles (1.125 MiB) that every GPU which loads the library holds
   until the process exits; nx*ny*nz above MHD_NOALLOC_MAX_CELLS returns MHD_EINVAL.  The first
   call on a device looks up that array's device address (cudaGetSymbolAddress), so make the first
   call on each device before any stream capture.  The address belongs to the device's current
   context: after that context is replaced (cudaDeviceReset, or a context of the caller's own) the
   next call looks it up again, so that call too belongs before any capture.  Every call shares
   the array: calls that may overlap on the GPU (different streams, or different host threads)
   race and must be serialised by the caller. */
#define MHD_NOALLOC_MAX_CELLS 4194304LL
int mhd_diagnostics_noalloc(const double* rho, const double* mx, const double* my,
                            const double* mz, const double* E, const double* bx, const double* by,
                            const double* bz, int nx, int ny, int nz, int bc_x, int bc_y,
                            int bc_z, double* out, void* stream);

/* Index checks (the paper has no counterpart: a debugging aid in place of a memory checker).  A
   library built with -DMHD_CHECK (libmhd_check.so) tests every computed cell and lattice index of
   its kernels against its array; a bad one is replaced by an in-bounds index and recorded here:
   bit 0 a cell index, bit 1 a face or lattice index.  Synchronises the device; clear = 1 resets
   the flags after reading them.  MHD_EINVAL from the plain library, which has no checks. */
int mhd_check_flags(int clear, unsigned* flags);

/* Measured FMA peak of the current GPU in TFLOP/s (an FMA counted as two flops): a grid of eight
   blocks of 256 threads per SM, each thread running eight independent chains of `iters` dependent
   FMAs in FP64 (fp64 = 1) or FP32 (fp64 = 0), the best of three launches timed with CUDA events
   after one warm-up.  The roofline denominator of the kernels bound by an arithmetic pipe (the
   paper has no counterpart: this is measurement support).  Synchronises the device; allocates and
   frees one small output array.  MHD_EINVAL for fp64 not in {0, 1}, iters < 1 or a null tflops. */
int mhd_probe_fma_peak(int fp64, int iters, double* tflops);

/* Bytes of device memory one sim of this size uses (precision 0 FP64 / 1 FP32, chem 0/1). */
size_t mhd_bytes_needed(int nx, int ny, int nz, int precision, int chem);

#ifdef __cplusplus
}
#endif
#endif /* MHD_H */
