/*
 * elpath.h -- C ABI of the B300 (sm_103a) one-way coupled Eulerian-Lagrangian
 * particle library.
 *
 * The method is that of "A coupled Eulerian-Lagrangian approach for fluid
 * and particle dynamics" (arxiv 2607.17836):
 *   - a Fourier pseudospectral vorticity-streamfunction solver on the periodic
 *     square [0, 2 pi)^2 advanced by second-order Adams-Bashforth
 *     (Sec. 3.1, Eqs. 1, 4-10);
 *   - passive tracers dx/dt = u(x, t) (Sec. 2.2, Eq. 2) and Stokes-drag
 *     inertial particles dx/dt = v, dv/dt = (u(x, t) - v) / St (Sec. 2.3,
 *     Eq. 3), both advanced by classical RK4 (Eqs. 12, 14);
 *   - the fluid velocity at a particle from bilinear, Catmull-Rom or cubic
 *     B-spline interpolation in space (Sec. 3.4, Eqs. 15-22) and linear
 *     interpolation in time between two fluid levels (Eqs. 23-24);
 *   - one coupled step = Algorithm 1: fluid n -> n+1, then every particle
 *     by one RK4 step between levels n and n+1.
 *
 * Conventions (for every call):
 *   - grid nodes x_i = i * 2 pi / n, arrays row-major [j][i] (y slow, x fast);
 *   - host arrays are owned by the caller and copied in/out during the call;
 *   - the device workspace is owned by the caller, must stay allocated until
 *     el_destroy_flow returns, and must be at least el_workspace_bytes(desc)
 *     bytes, 256-byte aligned; the library places every device array of the
 *     flow inside it (cuFFT's plan-internal tables excepted);
 *   - work is issued on the caller's CUDA stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream); el_step_coupled returns without
 *     waiting, every call that returns host data synchronises that stream;
 *   - every call returns an el_status; a failed call leaves the flow as it
 *     was, except EL_ECUDA / EL_ECUFFT, after which the flow should be
 *     destroyed.  el_last_error gives a one-line reason.  No call exits,
 *     throws across the ABI or traps on the device.
 */
#ifndef ELPATH_H
#define ELPATH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct el_flow el_flow;

typedef enum {
    EL_OK = 0,
    EL_EINVAL = 1,      /* bad argument (NULL, size, range, capacity)          */
    EL_ENOMEM = 2,      /* workspace smaller than el_workspace_bytes(desc)      */
    EL_ECUDA = 3,       /* a CUDA runtime call failed                          */
    EL_ECUFFT = 4,      /* a cuFFT call failed                                 */
    EL_ESTATE = 5,      /* call not valid in the flow's current state          */
    EL_ENONFINITE = 6,  /* a NaN/Inf appeared in the fields or particle state  */
    EL_ETIMEOUT = 7     /* a bounded device-side wait ran out                  */
} el_status;

typedef enum {
    EL_BILINEAR = 0,     /* Eq. 16, 2 x 2 nodes                                 */
    EL_CATMULL_ROM = 1,  /* Eqs. 18-19, 4 x 4 nodes i-1..i+2, periodic wrap     */
    EL_BSPLINE = 2,      /* Eqs. 21-22, 4 x 4 nodes, periodic wrap              */
    EL_ANALYTIC = 3      /* kinematic flows only (el_create_kinematic): the
                            prescribed velocity evaluated at the particle at
                            the exact stage time, no grid (Sec. 5.2, approach
                            (i)); tracers only                               */
} el_interp;

#define EL_MAX_SPECIES 8

typedef struct {
    int32_t n;                  /* grid points per side: power of two, 16..4096          */
    int32_t interp;             /* el_interp                                             */
    double nu;                  /* kinematic viscosity (1/Re of Eq. 1), >= 0             */
    double dt;                  /* common fluid and particle step (Sec. 3.1), > 0        */
    int32_t ab2_mode;           /* 0: viscous integrating factor (default);
                                   1: Eq. 10 as printed, viscous term inside R           */
    int32_t bspline_prefilter;  /* EL_BSPLINE only.  1: stencil weights act on
                                   interpolating spline coefficients (default);
                                   0: on raw samples, as Eq. 21 reads (approximating)    */
    int32_t max_species;        /* 0..EL_MAX_SPECIES                                     */
    int32_t sort_every;         /* re-bin particles by cell every k steps; 0 = never     */
    int64_t max_particles;      /* capacity summed over all species                      */
    int32_t tracer_velocity;    /* tracers (St = 0) take the fluid velocity from
                                   0: the interpolated velocity field (default);
                                   1: the interpolated streamfunction at (x +- dx, y)
                                      and (x, y +- dy) and centred differences
                                      (Sec. 3.2, Eq. 11), the paper's production path */
} el_flow_desc;

/* Bytes of device workspace a flow with this description needs (0 if the
 * description is invalid).  Cheap; usable for HBM admission control. */
size_t el_workspace_bytes(const el_flow_desc* desc);

/* Create a flow from the initial vorticity omega0 (host, n*n doubles, [j][i]).
 * The field is projected (mean removed, 2/3 rule of Sec. 3.1 applied), its
 * velocity reconstructed (Eqs. 5-6) and its nonlinear term evaluated, so that
 * the first el_step_coupled can run.  cuFFT plans are made here, once
 * (Sec. 3.1).  On success *out owns the flow; on failure *out is NULL. */
el_status el_create_flow(const el_flow_desc* desc, const double* omega0, void* dev_workspace,
                         size_t workspace_bytes, void* cuda_stream, el_flow** out);

/* The time-periodic kinematic flow of Sec. 5.2 (oscillating Taylor-Green
 * eddies), prescribed instead of solved:
 *   psi = (alpha / k) sin(k [x - eps sin(omega t)]) sin(k [y - eps sin(omega t + phi)]),
 *   u = d psi / dy = alpha sin(k [...x]) cos(k [...y]),
 *   v = -d psi / dx = -alpha cos(k [...x]) sin(k [...y]),
 * on the [0, 2 pi)^2 domain (the paper's L maps to 2 pi: lengths scale by
 * 2 pi / L, speeds too).  k must be a positive integer (periodicity) below
 * n / 3. */
typedef struct {
    double alpha;   /* peak speed                                   */
    double k;       /* wavenumber (integer >= 1)                    */
    double eps;     /* oscillation amplitude (length)               */
    double omega;   /* oscillation frequency                        */
    double phi;     /* phase between the x and y oscillations       */
} el_kinematic;

/* A flow whose levels are the kinematic field above at t = step * dt
 * (level pairs, streamfunction pairs and spline coefficients as for a solved
 * flow: every interpolant and both tracer paths apply unchanged), plus
 * interp = EL_ANALYTIC.  Everything else is as el_create_flow (workspace =
 * el_workspace_bytes(desc)); el_get_stats reports the field's exact E, Z, P;
 * el_get_field evaluates it on the grid.  Such a flow cannot join a batch,
 * and its steps run as direct launches (no captured graph).  EL_EINVAL for a
 * bad k, or EL_ANALYTIC with tracer_velocity = 1. */
el_status el_create_kinematic(const el_flow_desc* desc, const el_kinematic* kin,
                              void* dev_workspace, size_t workspace_bytes, void* cuda_stream,
                              el_flow** out);

/* Place np particles in species slot `species` (0..max_species-1).
 * st = 0: passive tracers (Eq. 2); st > 0: inertial particles (Eq. 3).
 * xy: host, 2*np doubles (x0, y0, x1, y1, ...), finite and at most 1e9 in
 * magnitude: positions are unwrapped and mapped periodically for field
 * evaluation (Sec. 3.2).  A non-finite or larger position, or a non-finite
 * velocity, gives EL_EINVAL naming its first index, with the slot unchanged
 * (the values are checked on the device, on the staged copy).
 * vxy: host, 2*np doubles of initial particle velocity, or NULL for zero slip
 * (velocity = interpolated fluid velocity at the position, current level).
 * Re-placing a slot replaces its particles; the positions passed become the
 * reference x(0) of the mean-square displacement.  Synchronises the stream. */
el_status el_set_particles(el_flow* flow, int32_t species, int64_t np, double st,
                           const double* xy, const double* vxy);

/* Advance nsteps coupled steps (Algorithm 1), asynchronously on the stream. */
el_status el_step_coupled(el_flow* flow, int32_t nsteps);

typedef struct {
    double t;                         /* simulated time                                 */
    int64_t step;                     /* steps taken                                    */
    double energy;                    /* E = 1/2 <u^2 + v^2>                            */
    double enstrophy;                 /* Z = 1/2 <omega^2>                              */
    double palinstrophy;              /* P = 1/2 <|grad omega|^2>                       */
    double msd[EL_MAX_SPECIES][2];    /* <(x - x0)^2>, <(y - y0)^2>, unwrapped          */
    double cluster[EL_MAX_SPECIES];   /* Var(n)/mean(n) - 1 on a 64 x 64 box grid       */
    int64_t np[EL_MAX_SPECIES];       /* particles per species (0 = empty slot)         */
    int32_t finite;                   /* 1 if every reduced quantity is finite          */
    /* Transport statistics of Sec. 5.5 / Sec. 6 per species and axis:          */
    double msd_sem[EL_MAX_SPECIES][2];     /* standard error of msd: sqrt(s^2 / np),    */
                                           /* s^2 the sample variance of (x - x0)^2     */
    double diffusivity[EL_MAX_SPECIES][2]; /* D = msd / (2 t) (0 at t = 0)              */
} el_stats;

/* Diagnostics of the current state, reduced in FP64 in a fixed order (the
 * same inputs give the same bits).  Synchronises the stream.  Returns
 * EL_ENONFINITE (with *out filled) if a NaN/Inf was found.  In a library
 * built with EL_CHECK_BOUNDS=1 (a debug build) it returns EL_ESTATE if any
 * particle step met a particle whose split state broke its invariants
 * (cell index >= n or offset outside [0, 1)); el_last_error says which. */
el_status el_get_stats(el_flow* flow, el_stats* out);

/* Particles of one species in their original order: unwrapped positions
 * (2*np doubles) and velocities (2*np doubles; the fluid-following
 * velocity is not stored for tracers, so vxy is zero-filled for st = 0).
 * Either pointer may be NULL.  Synchronises the stream. */
el_status el_get_particles(el_flow* flow, int32_t species, double* xy, double* vxy);

/* One field of the current level into host memory (n*n doubles):
 * 0 = vorticity, 1 = u, 2 = v, 3/4 = the u/v node values the particle
 * stencil weights (the spline coefficients when prefiltering, else u/v).
 * Synchronises the stream. */
el_status el_get_field(el_flow* flow, int32_t which, double* host_nn);

/* Fluid velocity at np arbitrary points by the flow's interpolant, blended
 * linearly in time between the previous (theta = 0) and the current level
 * (theta = 1): exactly the gather the particle step uses.  d_xy and d_uv are
 * DEVICE arrays of 2*np doubles.  Asynchronous on the stream. */
el_status el_sample_velocity(el_flow* flow, int64_t np, const double* d_xy, double theta,
                             double* d_uv);

/* Run ONE coupled step exactly as el_step_coupled does (re-binning first
 * if it is due), but by direct launches with CUDA events on the flow's
 * stream around each stage, then synchronise and report the stage times in
 * milliseconds: stage_ms[0] = fluid step (Sec. 3.1), stage_ms[1] = RK4 step
 * of every species (one launch), stage_ms[2] = re-binning (0 if not due).
 * nstage must be >= 3. */
el_status el_profile_step(el_flow* flow, double* stage_ms, int32_t nstage);

/* Launch-shape and re-binning settings of a flow.  None of them changes any
 * result: every particle's arithmetic is independent of the order particles
 * are stored in and of the block shape. */
typedef struct {
    int32_t rk4_threads;  /* threads per block of the particle step: multiple of 32, 64..512 */
    int32_t sort_every;   /* re-bin every k steps (0 = never)                                  */
    int32_t sort_shift;   /* re-binning key = tile of 2^shift x 2^shift cells (0..4)           */
    int32_t gather;       /* cubic schemes' stencil gather: EL_GATHER_* (bilinear ignores it)  */
    double ms_per_step;   /* filled by the autotuners: measured time per step of the choice   */
} el_tuning;

/* Stencil gather of the cubic schemes (Eqs. 18-22), same results either way:
 * EL_GATHER_REGISTERS: each thread keeps its particle's 16 level-pair nodes in
 * registers; EL_GATHER_SHARED: the 32 particles of a warp share one patch of
 * nodes in shared memory (pays when many particles share a cell);
 * EL_GATHER_AUTO (the default): the shared patch when some species holds at
 * least 2 particles per cell on average, else registers. */
enum { EL_GATHER_AUTO = 0, EL_GATHER_REGISTERS = 1, EL_GATHER_SHARED = 2 };

el_status el_get_tuning(const el_flow* flow, el_tuning* out);
el_status el_set_tuning(el_flow* flow, const el_tuning* tuning);

/* Autotuner.  Picks the particle step's block size (fastest of {128, 256,
 * 512} over trial_steps steps, each right after a re-binning, for each
 * stencil gather with the cubic schemes), the
 * re-binning tile (fastest of 1, 2, 4 cells per side, counting its cost)
 * and the cadence from a measured model: the step time grows about linearly
 * as particles drift out of cell order, t(k) = t0 + a k, so with re-binning
 * cost c every S steps the mean is t0 + a S / 2 + c / S, least at
 * S = sqrt(2 c / a) (t0, t(W) and c are timed; 0 = never when a is nil).
 * The trial steps advance the simulation like any others; no result depends
 * on the settings.  Synchronises the stream. */
el_status el_autotune(el_flow* flow, int32_t trial_steps, el_tuning* best);

/* Number of kernel launches of the library (not cuFFT) issued so far by
 * this flow; lets a caller count the launches inside a timed region. */
int64_t el_kernel_launches(const el_flow* flow);

/* 1 if the flow's fluid step (Secs. 3.1, Eqs. 4-10) runs the library's fused
 * transforms (256^2 and 512^2 with 4 or 6 inverse-transform planes, 1024^2,
 * 2048^2 with 4 or 6), 0 if it runs cuFFT's, or for a NULL flow.  A fused
 * flow takes no FFT-pool slot in a batch (see el_batch_add_fft_pool). */
int32_t el_flow_fused(const el_flow* flow);

/* ---- Batched engine --------------------------------------------------------
 * Many independent flows (any grid sizes, species mixes, schemes and step
 * counts) advanced together: one coupled step of the batch is one captured
 * graph with one kernel per stage over all members (the fused fluid kernels
 * once per grid size and plane count, the particle kernel once per scheme and
 * stencil gather) and the other members' transforms on concurrent branches.  A member's arithmetic is the
 * same as when it is stepped alone.  While in a batch a flow uses the batch's
 * stream, el_step_coupled on it returns EL_ESTATE, and the other calls on it
 * (particles, statistics, fields) work as usual.  Members join and leave at
 * any step (continuous batching); each keeps its own step count. */
typedef struct el_batch el_batch;

/* Device workspace bytes of a batch of up to max_members flows (its tables). */
size_t el_batch_workspace_bytes(int32_t max_members);
el_status el_batch_create(int32_t max_members, void* dev_workspace, size_t workspace_bytes,
                          void* cuda_stream, el_batch** out);
/* Add a flow (same device; synchronises the flow's stream first). */
el_status el_batch_add(el_batch* batch, el_flow* flow);
/* Remove a member (synchronises the batch stream; the flow gets its own stream back). */
el_status el_batch_remove(el_batch* batch, el_flow* flow);
/* Advance every member by nsteps coupled steps, asynchronously on the batch stream. */
el_status el_batch_step(el_batch* batch, int32_t nsteps);
/* el_autotune over the whole batch (one setting for every member). */
el_status el_batch_autotune(el_batch* batch, int32_t trial_steps, el_tuning* best);
int32_t el_batch_size(const el_batch* batch);
int64_t el_batch_kernel_launches(const el_batch* batch);
const char* el_batch_last_error(const el_batch* batch);
/* Remove every member and free the batch's host state (and its pools' plans). */
el_status el_batch_destroy(el_batch* batch);

/* FFT pools (optional).  The transforms of Eqs. 4-8 for members of one class
 * -- the grid n and the inverse-transform plane count that `desc` implies
 * (4, +2 with the B-spline prefilter, +1 with tracer_velocity = 1) -- can run
 * as one batched cuFFT call per transform over a pool of `slots` members,
 * instead of one call per member (cuFFT's time per plane falls steeply with
 * the batch count).  A pool is device memory the caller provides and keeps
 * until el_batch_destroy, at least el_batch_fft_pool_bytes(desc, slots)
 * bytes, 256-byte aligned (0: invalid desc or slots outside [1, 4096]).
 * A flow added with el_batch_add after the pool takes a free slot of a pool
 * of its class if there is one, the lowest free one (else it transforms
 * alone, as before); it keeps the slot until it leaves.  Flows whose fluid
 * step is fused (el_flow_fused) take no slot: the batch runs their transforms
 * as one launch of each fused kernel for all members of their grid.  The batched calls
 * cover slots 0 .. the highest occupied one.  The results equal the per-member path's up
 * to the rounding of cuFFT's batched kernels.  EL_ENOMEM when `bytes` is too
 * small; EL_ECUFFT when the plans cannot be made. */
size_t el_batch_fft_pool_bytes(const el_flow_desc* desc, int32_t slots);
el_status el_batch_add_fft_pool(el_batch* batch, const el_flow_desc* desc, int32_t slots,
                                void* dev_workspace, size_t bytes);

/* Mean-square displacement and clustering index of np particles, computed
 * without allocating any memory.  The paper has no counterpart: this is a
 * library service for callers that cannot allocate device memory at the
 * moment they need these statistics -- a loop that must not stall (cudaMalloc
 * and cudaFree can synchronise the whole device) or an application whose
 * device memory is all reserved up front by another allocator.
 * d_xy, d_xy0: DEVICE arrays of 2*np doubles, unwrapped positions now and at
 * the reference time (as el_get_particles returns them), each 16-byte
 * aligned (read as (x, y) pairs).  d_out3: DEVICE array of 3 doubles, 8-byte
 * aligned, receiving <(x-x0)^2>, <(y-y0)^2> and the clustering
 * index (Var(n)/mean(n) - 1 on a 64 x 64 box grid of the wrapped positions),
 * reduced in FP64 in the same fixed order as el_get_stats.
 * np must be <= EL_NOALLOC_MAX_PARTICLES and the pointers aligned, else
 * EL_EINVAL (np = 0 gives 0, 0, 0).  Work is queued on
 * cuda_stream and the call returns without waiting.  Scratch: one fixed
 * device array of about 4 MiB inside the library, present on every GPU that
 * loads it until the process exits, shared by all calls: calls whose work
 * overlaps on the GPU race.  Every call looks up the array's device address
 * in the current device's context (nothing is kept across calls, so a call
 * after a cudaDeviceReset finds the reloaded array); the call may be captured
 * into a CUDA graph after a first plain call on that device (which loads the
 * library's module).
 * Errors: el_last_error(NULL). */
#define EL_NOALLOC_MAX_PARTICLES 262144
el_status el_dispersion_noalloc(const double* d_xy, const double* d_xy0, int64_t np,
                                double* d_out3, void* cuda_stream);

/* Checkpoint and resume.  The coupled step (Algorithm 1) depends on a flow
 * only through omega-hat, the AB2 history and N-hat of the current level
 * (Sec. 3.1, Eqs. 9-10), the level pair holding the current velocity field
 * (Sec. 3.2; with tracer_velocity = 1 also the streamfunction pair) and each
 * particle's state and reference position; the state image is exactly that
 * plus the step count, in host byte order, ending in a 64-bit FNV-1a
 * checksum.  Loading an image into a flow created with the same n, interp,
 * nu, dt, ab2_mode, bspline_prefilter and tracer_velocity and stepping on
 * reproduces the uninterrupted run bit for bit.
 *
 * el_save_state: host_buf = NULL stores the image size in *bytes and returns
 * EL_OK.  Otherwise *bytes is the buffer's size; a buffer that is too small
 * gives EL_EINVAL with the needed size in *bytes; on success *bytes is the
 * image size.  Synchronises the stream.
 * el_load_state: replaces the flow's state by the image (bytes = its exact
 * size).  EL_EINVAL, with the flow unchanged, for an image that is not one,
 * is truncated or altered (checksum), was saved by a flow of another
 * descriptor, or has more particles than the flow can hold; EL_ESTATE for a
 * member of a batch.  The tuning settings stay the flow's own.  Synchronises
 * the stream. */
el_status el_save_state(el_flow* flow, void* host_buf, size_t* bytes);
el_status el_load_state(el_flow* flow, const void* host_buf, size_t bytes);

/* Destroy the flow (plans, graphs, host state).  The workspace is the
 * caller's to free afterwards. */
el_status el_destroy_flow(el_flow* flow);

/* One-line reason for the last failure of a call on this flow (or, when
 * flow is NULL, of the last el_create_flow or el_dispersion_noalloc on this
 * thread).  Never NULL. */
const char* el_last_error(const el_flow* flow);

#ifdef __cplusplus
}
#endif

#endif /* ELPATH_H */
