/*
 * aniso.h -- C ABI of libaniso.so, a GB300 (sm_103a) implementation of the
 * directionally split semi-implicit step for anisotropic diffusion of
 * Sharma & Hammett, "A Fast Semi-implicit Method for Anisotropic Diffusion"
 * (arXiv:1008.0861), Section 2.
 *
 * The equation (Section 2, Eqs. aniso_cond and heat_flux):
 *     dT/dt = -div q,   q = -chi_par b (b . grad T)  [+ chi_perp grad T part]
 * on a uniform 2-D Cartesian grid of nx * ny cells (x fastest in memory:
 * T[j*nx + i] is cell (i, j)).  One step is the composition of Eq. op_2step:
 *     T^{n+1} = (1 + dt D_yy)^-1 (1 - dt D_yx) (1 + dt D_xx)^-1 (1 - dt D_xy) T^n,
 * i.e. an x-update (Eq. xup) and then a y-update (Eq. yup).  Each update is
 * implicit in the face-normal flux (one tridiagonal system per grid line,
 * cyclic when the boundary is periodic) and explicit in the transverse flux,
 * whose face differences are limited with van Leer's limiter
 * (Eq. vanLeer, L(a,b,c,d) = L(L(a,b), L(c,d))).  The face value of b is the
 * plain average of the two adjacent cell centres (Section 2).
 *
 * Conventions shared by every call:
 *  - All status codes are `int` (ANISO_OK = 0).  No call aborts, traps or
 *    prints; the message of the last failure on the calling host thread is
 *    returned by aniso_last_error().
 *  - Pointers named "device" must point to device memory of the current
 *    CUDA device; "host" pointers to ordinary host memory.  The caller owns
 *    every buffer it passes; the library owns the buffers inside a handle.
 *  - Element type of T, bx, by follows the handle's precision:
 *    ANISO_PREC_FP64 -> double, ANISO_PREC_FP32 -> float.
 *  - Work is enqueued asynchronously on the handle's stream (the legacy
 *    default stream unless ANISO_OPT_STREAM sets another); only calls that
 *    return host values (aniso_total, aniso_sync, aniso_get_state with a
 *    host copy) synchronise it.
 *  - Units: dx, dy are cell sizes; chi_par, chi_perp diffusivities; dt the
 *    timestep.  Coefficients used per update: lamx = chi_par dt / dx^2,
 *    lamy = chi_par dt / dy^2, mu = chi_par dt / (dx dy).
 */
#ifndef ANISO_H
#define ANISO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aniso_ctx *aniso_t;         /* one grid (opaque, library-owned) */
typedef struct aniso_batch *aniso_batch_t; /* a set of grids stepped together */

/* Status codes. */
enum {
    ANISO_OK = 0,
    ANISO_ERR_ARG = 1,         /* invalid argument (size, spacing, null pointer, range) */
    ANISO_ERR_STATE = 2,       /* call out of order, e.g. aniso_step before aniso_set_field */
    ANISO_ERR_CUDA = 3,        /* a CUDA runtime call failed; message has the CUDA error */
    ANISO_ERR_NONFINITE = 4,   /* a step produced a NaN or infinite temperature */
    ANISO_ERR_TIMEOUT = 5,     /* a kernel's bounded wait for its staged input expired */
    ANISO_ERR_OOM = 6,         /* device allocation failed */
    ANISO_ERR_UNSUPPORTED = 7  /* valid request outside what this build handles */
};

/* Boundary conditions (both directions). */
enum {
    ANISO_BC_ZEROFLUX = 0, /* reflective (Section 3.1): no flux through boundary faces */
    ANISO_BC_PERIODIC = 1, /* wrap-around; line systems become cyclic */
    ANISO_BC_DIRICHLET = 2 /* fixed values on the domain edge (the convergence test of Section
                              3.2): the outer ring of cells holds boundary nodes whose values
                              never change; single handles only (not batches, not with the
                              compensated state) */
};

/* Option keys for aniso_set_option and their values. */
enum {
    ANISO_OPT_PRECISION = 0,  /* ANISO_PREC_FP64 (default) or ANISO_PREC_FP32 */
    ANISO_OPT_FIELD_FP16 = 1, /* 1: store face coefficients as FP16 (FP32 precision only) */
    ANISO_OPT_KAHAN = 2,      /* 1: compensated FP32 state, T + lo (FP32 precision only) */
    ANISO_OPT_LIMITER = 3,    /* ANISO_LIM_* */
    ANISO_OPT_ORDER = 4,      /* ANISO_ORDER_* */
    ANISO_OPT_STREAM = 5,     /* cudaStream_t cast to integer; 0 = legacy default stream */
    ANISO_OPT_GRAPH = 6,      /* 1 (default): replay aniso_step loops from a captured CUDA graph */
    ANISO_OPT_PROFILE = 7,    /* 1: time every sweep launch with CUDA events (aniso_kernel_times);
                                 k > 1: batched calls time the sweeps of every k-th step of a
                                 call (steps 0, k, 2k, ...), so that fewer event nodes sit in
                                 the graph; single-handle calls time every sweep */
    ANISO_OPT_FAST_PATH = 8,  /* kernels of the x-then-y order with a transposed intermediate:
                                 3 (default): warp-autonomous line kernel (coalesced flux phase,
                                 per-lane segment elimination, shuffle-only line solve);
                                 1: block-synchronous vectorised line kernel;
                                 0: general kernels only; 2 is not a valid value */
    ANISO_OPT_SEGMENT = 9,    /* cells per thread segment of the vectorised kernels, in 16-byte
                                 chunks (0 = default 4; larger: fewer threads per line and so a
                                 shallower PCR) */
    ANISO_OPT_BLOCK_WARPS = 10, /* warps per block of the warp-autonomous kernel (0 = default 4;
                                   1, 2, 4 or 8): lines per block = warps x lines per warp */
    ANISO_OPT_SCHEME = 11,     /* ANISO_SCHEME_2STEP (default), _4STEP or _EXPLICIT; the other
                                  schemes run on single handles (aniso_step, not batches) with
                                  the plain state; ANISO_ERR_UNSUPPORTED with the compensated one */
    ANISO_OPT_DIAGNOSTICS = 12, /* 1: batched calls record, after every step of every grid on the
                                  fast path, the FP64 sum of T, its minimum and its maximum (read
                                  with aniso_batch_diagnostics); taken from the batch's first handle */
    ANISO_OPT_TMA_LINES = 13,  /* batched calls, FP32 with FP32 coefficients: 1 solves the lines of
                                  768 to 1024 cells (multiples of 32) with the kernel that stages
                                  each block's rows by tensor-map (TMA) tile loads and keeps the
                                  line state in registers; 0 (default: faster on the uneven batch,
                                  where that kernel shares the GPU with the other line classes)
                                  uses the warp-per-line kernel for all lines; 2 is for testing
                                  the failure path only: that kernel
                                  issues no loads, its bounded wait gives up and the call reports
                                  ANISO_ERR_TIMEOUT at the next aniso_sync / aniso_total of the
                                  first handle.  Taken from the batch's first handle.  Y-updates
                                  recorded by ANISO_OPT_DIAGNOSTICS use the warp-per-line kernel. */
    ANISO_OPT_TMEM = 14,       /* FP32: 1 (default) keeps part of the line state in the SM's tensor
                                  memory (TMEM) instead of shared memory, so more blocks fit an SM:
                                  in batched calls the warp-per-line kernel's (four-warp blocks,
                                  lines of at most 8 chunks of 4 cells a lane; chosen grid by grid
                                  where it keeps more blocks resident; taken from the batch's first
                                  handle), and the cluster kernel's for the plain state.  0 keeps
                                  it all in shared memory.  Results are the same bit for bit. */
    ANISO_OPT_CLUSTER_LINES = 15 /* FP32 fast path, lines cut across the blocks of one thread-block
                                  cluster (pieces of 2048 or 1024 cells), so that lines too long for
                                  one block need no transpose pass.  2 (default): lines of 4096,
                                  8192 and 16384 cells, and both directions of a compensated-state grid
                                  (ANISO_OPT_KAHAN) whose sides are 1024, 2048, 4096, 8192 or 16384
                                  cells; 1: as 2, but lines of 2049-4096 cells stay on the
                                  long-line kernel; 0: none (the general kernels).  With
                                  ANISO_OPT_TMEM the plain state keeps part of its line state in
                                  tensor memory. */
};
enum { ANISO_PREC_FP64 = 0, ANISO_PREC_FP32 = 1 };
enum {
    ANISO_SCHEME_2STEP = 0, /* Eq. op_2step: one semi-implicit update per direction */
    ANISO_SCHEME_4STEP = 1, /* Eq. 4step: per direction, the semi-implicit update with its implicit
                               part over dt/2, then a fully implicit dt/2 update (Section 2.1) */
    ANISO_SCHEME_EXPLICIT = 2 /* the explicit limited scheme the paper compares against: the face
                                 fluxes of Eqs. xup and yup all from T^n, applied explicitly;
                                 stable only up to about the explicit limit (kernel timings are
                                 reported under ANISO_KERNEL_XSWEEP) */
};
enum {
    ANISO_LIM_VANLEER = 0, /* Eq. vanLeer (default) */
    ANISO_LIM_ARITH = 1,   /* arithmetic mean of the four differences: the linear
                              reading used for Eqs. amp1/amp2 (testing only) */
    ANISO_LIM_MINMOD = 2,  /* minmod, named in Section 2 */
    ANISO_LIM_MC = 3       /* monotonized central, named in Section 2 */
};
enum {
    ANISO_ORDER_XY = 0,       /* Eq. op_2step: x-update then y-update every step (default) */
    ANISO_ORDER_YX = 1,       /* the reversed order the paper mentions after Eq. op_2step */
    ANISO_ORDER_ALTERNATE = 2 /* x,y on even step counters, y,x on odd ones */
};
/* Directions for aniso_sweep. */
enum { ANISO_DIR_X = 0, ANISO_DIR_Y = 1 };
/* Kernel kinds for aniso_kernel_times. */
enum { ANISO_KERNEL_XSWEEP = 0, ANISO_KERNEL_YSWEEP = 1, ANISO_KERNEL_TRANSPOSE = 2 };

/* Create a handle for one nx * ny grid.
 *   nx, ny   : cells per direction, each >= 3.
 *   dx, dy   : cell sizes, > 0.
 *   chi_par  : parallel diffusivity, > 0 (Eq. heat_flux).
 *   chi_perp : perpendicular diffusivity, 0 <= chi_perp <= chi_par.  It adds
 *              chi_perp * I to the diffusion tensor (Section 2.1's general
 *              symmetric tensor); the paper's tests use 0.
 *   bc       : ANISO_BC_*.
 *   out      : receives the handle.
 * Allocates nothing on the device yet (buffers are sized on
 * aniso_set_field).  Errors: ANISO_ERR_ARG. */
int aniso_create(int nx, int ny, double dx, double dy, double chi_par, double chi_perp, int bc,
                 aniso_t *out);

/* Set an option (ANISO_OPT_*).  PRECISION, FIELD_FP16 and KAHAN must be set
 * before aniso_set_field; the others any time.  Errors: ANISO_ERR_ARG (key
 * or value), ANISO_ERR_STATE (precision change after the field is set). */
int aniso_set_option(aniso_t h, int key, long long value);

/* Set the unit field b (Section 2): bx, by are device arrays of nx*ny cell-
 * centred components in the handle's precision.  The library averages b to
 * faces (Section 2: the plain mean of the two cells) in FP64 and stores the face
 * coefficients it needs, in units of chi_par (kappa = chi_perp/chi_par):
 *     x faces: kappa + (1-kappa) bx^2,  (1-kappa) bx by
 *     y faces: kappa + (1-kappa) by^2,  (1-kappa) by bx
 * rounded once to the storage type (FP64, FP32 or FP16).  Under zero-flux
 * boundaries the boundary-face coefficients are zero.  b is not required to
 * be unit length; the paper's b is.  The caller may free bx, by after the
 * call returns and the stream has passed it.  Errors: ANISO_ERR_ARG (null),
 * ANISO_ERR_OOM, ANISO_ERR_CUDA. */
int aniso_set_field(aniso_t h, const void *bx, const void *by);

/* Source term Q (device pointer, nx*ny, handle precision, row-major; the
 * convergence test of Section 3.2 adds Q to Eq. 1): copied into the handle and
 * applied in every later step as an explicit stage T += dt Q before the
 * directional updates.  NULL removes it.  ANISO_ERR_STATE before
 * aniso_set_field; ANISO_ERR_UNSUPPORTED with the compensated state.  A
 * handle with a source cannot join a batch. */
int aniso_set_source(aniso_t h, const void *Q);

/* Advance T by nsteps steps of size dt (Eq. op_2step), in place.
 *   T      : device array nx*ny in the handle's precision.
 *   dt     : > 0.  nsteps >= 0.
 * The update order of each step follows ANISO_OPT_ORDER; the handle's step
 * counter (used by ANISO_ORDER_ALTERNATE) advances by nsteps.  With
 * ANISO_OPT_KAHAN the handle keeps the low parts of T between calls.
 * Asynchronous.  Errors: ANISO_ERR_ARG, ANISO_ERR_STATE (no field),
 * ANISO_ERR_CUDA, ANISO_ERR_UNSUPPORTED (a line longer than the on-chip
 * limit: 16384 cells in FP32, 8192 in FP64). */
int aniso_step(aniso_t h, void *T, double dt, int nsteps);

/* One directional update: Eq. xup (dir = ANISO_DIR_X) or Eq. yup
 * (ANISO_DIR_Y) from Tin to Tout (device arrays, nx*ny, distinct).  Exposes
 * a single half of the split for line-by-line checks.  Does not touch the
 * step counter or the Kahan state.  Asynchronous.  Errors as aniso_step. */
int aniso_sweep(aniso_t h, int dir, const void *Tin, void *Tout, double dt);

/* Conservation and bounds diagnostics of T (device array, handle precision):
 * sum in FP64 (deterministic order; with Kahan state the sum of T + lo),
 * minimum, maximum and the count of non-finite values.  Any output pointer
 * may be NULL.  Synchronises the handle's stream.  Returns
 * ANISO_ERR_NONFINITE when a step since the last check produced a
 * non-finite value (the flag is then cleared). */
int aniso_total(aniso_t h, const void *T, double *sum, double *tmin, double *tmax,
                long long *nonfinite);

/* Step counter and compensated low part (checkpoint / resume).
 * get: *step_counter receives the counter; if lo_out (device, nx*ny float)
 *      is non-NULL and Kahan is on, the low parts are copied there.
 * set: sets the counter; lo_in (device) may be NULL to clear the low parts.
 * Asynchronous copies on the handle's stream. */
int aniso_get_state(aniso_t h, long long *step_counter, void *lo_out);
int aniso_set_state(aniso_t h, long long step_counter, const void *lo_in);

/* Wait for the handle's stream; returns ANISO_ERR_NONFINITE if a step since
 * the last check produced a non-finite value. */
int aniso_sync(aniso_t h);

/* Sum of CUDA-event durations (milliseconds) and number of launches of one
 * kernel kind (ANISO_KERNEL_*) recorded while ANISO_OPT_PROFILE was on, for
 * a handle (h) or a batch (b; pass h = NULL).  Synchronises.  reset = 1
 * clears the counters after reading. */
int aniso_kernel_times(aniso_t h, aniso_batch_t b, int kind, double *ms, long long *launches,
                       int reset);

/* Free a handle and its device buffers (after synchronising its stream). */
void aniso_destroy(aniso_t h);

/* Message of the last failed call on this host thread ("" if none). */
const char *aniso_last_error(void);

/* Group n handles (same precision, limiter and field storage; each with its
 * field set) so that each sweep advances all of them together: one launch per
 * class of line lengths with the same occupancy (at most five, run
 * concurrently), the paper's update applied to independent grids of uneven
 * sizes, fields and timesteps.  The batch uses the first handle's stream and options
 * GRAPH/PROFILE.  The handles must outlive the batch.  Grids with more than
 * 1024 rows take their y-updates through the transpose path, captured into the
 * same graph.  Errors: ANISO_ERR_ARG, ANISO_ERR_STATE. */
int aniso_batch_create(int n, const aniso_t *hs, aniso_batch_t *out);

/* Advance grid k of the batch by nsteps[k] steps of size dt[k] in place on
 * T[k] (host arrays of n entries; T[k] a device pointer).  Grids with fewer
 * steps drop out as they finish.  The whole call is captured once into a
 * CUDA graph and replayed while T, dt and nsteps stay the same.
 * Asynchronous. */
int aniso_step_batched(aniso_batch_t b, void *const *T, const double *dt, const int *nsteps);

/* aniso_step_batched on host arrays: T_host[k] is a host array of grid k's
 * nx*ny values (handle precision; page-locked memory makes the copies
 * asynchronous DMA, pageable memory works too).  Each grid is copied into a
 * device buffer the batch owns (allocated on the first call, freed by
 * aniso_batch_destroy), the batched call runs as above, and the results are
 * copied back.  Returns when T_host holds the result (synchronises the
 * batch's stream).  Errors: as aniso_step_batched, ANISO_ERR_OOM. */
int aniso_step_batched_host(aniso_batch_t b, void *const *T_host, const double *dt, const int *nsteps);

/* Per-step diagnostics of the last aniso_step_batched(_host) call that ran
 * with ANISO_OPT_DIAGNOSTICS on the batch's first handle: for grid k and
 * step s (0-based within the call), out[(k * steps + s) * 3 + {0, 1, 2}] =
 * FP64 sum of T after that step, minimum, maximum.  The abstract calls the
 * scheme conservative; the sum follows conservation step by step, and min T
 * the monotonicity Section 3.1 measures (its relative non-monotonicity is
 * (min T0 - min T) / min T0).  The values are formed inside the y-update
 * kernel (each block's values in a fixed order, FP64 across blocks) and
 * finished by one small kernel per launch, so the call stays one graph.
 * Slots of steps a grid does not take, and of grids whose y-update does not
 * run on the warp-per-line kernel (off the fast path, columns above 2048
 * cells, or on the cluster kernel of ANISO_OPT_CLUSTER_LINES), are NaN.
 * *steps (may be NULL) receives the steps per grid (the call's largest
 * nsteps); out may be NULL to query it.  capacity: doubles available at out.
 * Synchronises the batch's stream.  Errors: ANISO_ERR_ARG (capacity),
 * ANISO_ERR_STATE (no such call yet). */
int aniso_batch_diagnostics(aniso_batch_t b, double *out, long long capacity, int *steps);

void aniso_batch_destroy(aniso_batch_t b);

/* Block-shape autotuner for aniso_step_batched (the batched configuration
 * asks for rows per block and PCR depth chosen by measurement; the paper has
 * no counterpart).  For each candidate of a fixed table (fast-path kernel,
 * warps per block of the warp-autonomous kernel, 16-byte chunks per lane,
 * which sets the team size and so the PCR depth), the batch's steps run on
 * device copies of T[k] (`nsteps` steps per call, one untimed call, then
 * `reps` calls timed with CUDA events on the batch's stream); the fastest
 * candidate's options are set in every handle of the batch.
 * T[k]: device pointers as for aniso_step_batched, read only; dt[k] > 0.
 * nsteps >= 1, reps >= 1.  Outputs (may be NULL): *choice = the candidate's
 * index (-1 when no grid of the batch takes the fast path: nothing is
 * changed), *best_ms = its time per call.  The handles' step counters are
 * restored.  Allocates (and frees) one scratch buffer the size of all grids.
 * Synchronises the batch's stream.  ANISO_ERR_OOM when the scratch buffer
 * cannot be allocated; the handles keep their options on any error. */
int aniso_batch_autotune(aniso_batch_t b, void *const *T, const double *dt, int nsteps, int reps,
                         int *choice, double *best_ms);
/* The autotuner's candidate `index`: fast-path option value, warps per block
 * (0 = default) and chunks per lane.  ANISO_ERR_ARG when out of range. */
int aniso_autotune_candidate(int index, int *fast, int *warps, int *seg);
/* Temperature-dependent diffusivity (Section 3.3 runs the method with chi_par
 * proportional to T^(5/2)): chi_par becomes chi_par * (max(T,0)/t_ref)^alpha,
 * taken at each face as the harmonic mean of the two cells' values, from the
 * input of each directional update (T^n for the x-update, T* for the
 * y-update); chi_perp scales alike.  alpha = 0 (the default) restores the
 * constant diffusivity.  aniso_step then needs the 2-step x-then-y scheme on
 * the line4 fast path (both line lengths multiples of the 16-byte vector and
 * at most 2048), the plain state, an FP32 or FP64 field, and neither fixed
 * boundaries nor a source; otherwise it returns ANISO_ERR_UNSUPPORTED, as do
 * aniso_sweep and aniso_batch_create for such a handle.
 * Errors: ANISO_ERR_ARG (alpha < 0, t_ref <= 0, not finite). */
int aniso_set_nonlinear(aniso_t h, double alpha, double t_ref);

/* Kernel launches in one aniso_step_batched call of the batch's current plan
 * (the kernel nodes of its captured graph; 0 before the first call).  The
 * plan splits each sweep's lines by the occupancy their shared memory allows
 * and runs those launches concurrently, so a sweep can be several kernels.
 * Errors: ANISO_ERR_ARG (null). */
int aniso_batch_kernel_count(aniso_batch_t b, long long *kernels);

/* aniso_step without any device allocation.  (No counterpart in the paper: it
 * exists for callers that are not allowed to allocate GPU memory, such as code
 * running inside another framework's memory pool or under a fixed device
 * memory budget; aniso_create/aniso_set_field allocate, this call does not.)
 * It runs nsteps x-then-y steps (Eq. op_2step, van Leer limiter) of one grid
 * in place on T, with the grid described by the same arguments as
 * aniso_create and the field by device arrays bx, by (cell-centred, nx*ny,
 * element type given by `precision`, ANISO_PREC_FP64 or ANISO_PREC_FP32).
 * `stream` is a cudaStream_t (NULL: the legacy default stream); the call is
 * asynchronous on it.
 * Working memory (the face coefficients and T*) lives in one fixed device
 * array of 20 MiB compiled into the library, allocated on first use per
 * device and then held by that GPU until the process exits: at most
 * 1,048,576 cells in FP32 and 524,288 in FP64 (larger grids fail with
 * ANISO_ERR_ARG and a message), and ny <= 1024.  Each call made outside a
 * stream capture looks up that array's device address (with the device
 * current); a call inside a capture reuses the address of the last such call
 * on the device, so make a first call before any stream capture
 * (ANISO_ERR_STATE otherwise).  Every call reuses the same array, so calls whose
 * GPU work overlaps (other streams or host threads) race and corrupt each
 * other: serialise them.  Non-finite results are not reported by this call. */
int aniso_step_noalloc(int nx, int ny, double dx, double dy, double chi_par, double chi_perp, int bc,
                       int precision, const void *bx, const void *by, void *T, double dt, int nsteps,
                       void *stream);

/* ------------------------------------------------------ three dimensions
 *
 * The split step on an nx * ny * nz grid (Section 2.1: three updates per
 * step, each implicit in its face-normal flux and explicit in the two limited
 * transverse fluxes, whose 2-step form is stable for chi dt / dx^2 up to
 * about 8.25 with equal spacings; the 4-step form of Eq. 4step, with six
 * half-coefficient line solves per step, at any timestep).
 * Arrays are [nz][ny][nx], x fastest, device memory, element type of the
 * handle's precision.  Every line length must be a multiple of the 16-byte
 * vector (4 cells in FP32, 2 in FP64), at least two vectors, and at most
 * 2048 cells in FP32 or 1024 in FP64 (with the default segment option);
 * other shapes give ANISO_ERR_UNSUPPORTED at aniso3_set_field.
 * Boundaries: ANISO_BC_ZEROFLUX or ANISO_BC_PERIODIC on all six faces.
 * Status codes and aniso_last_error() as for the 2-D calls. */
typedef struct aniso3_ctx *aniso3_t;

/* Create a handle; arguments as aniso_create plus nz and dz.  Allocates
 * nothing on the device.  Errors: ANISO_ERR_ARG. */
int aniso3_create(int nx, int ny, int nz, double dx, double dy, double dz, double chi_par, double chi_perp,
                  int bc, aniso3_t *out);
/* Options: ANISO_OPT_PRECISION and FIELD_FP16 (FP16 face coefficients, FP32
 * precision only; both before aniso3_set_field), LIMITER, SCHEME
 * (ANISO_SCHEME_2STEP or _4STEP), STREAM, BLOCK_WARPS, SEGMENT.  The other
 * keys accept only their default 0 (ANISO_ERR_UNSUPPORTED otherwise). */
int aniso3_set_option(aniso3_t h, int key, long long value);
/* Cell-centred unit field (device arrays, [nz][ny][nx]); the library averages
 * it to the faces and keeps nine coefficient arrays plus two intermediates
 * (11 arrays of the grid's size).  Errors: ANISO_ERR_ARG, _UNSUPPORTED
 * (shape), _OOM, _CUDA. */
int aniso3_set_field(aniso3_t h, const void *bx, const void *by, const void *bz);
/* nsteps steps in place on T (device, [nz][ny][nx], 16-byte aligned), the
 * updates in the order x, y, z.  Asynchronous on the handle's stream.
 * Errors: ANISO_ERR_ARG, ANISO_ERR_STATE (no field), ANISO_ERR_CUDA. */
int aniso3_step(aniso3_t h, void *T, double dt, int nsteps);
/* FP64 sum, min, max and non-finite count of T; synchronises.  Also returns
 * ANISO_ERR_NONFINITE if a step since the last check produced a NaN or
 * infinity. */
int aniso3_total(aniso3_t h, const void *T, double *sum, double *tmin, double *tmax, long long *nonfinite);
/* Wait for the handle's stream; ANISO_ERR_NONFINITE as aniso3_total. */
int aniso3_sync(aniso3_t h);
void aniso3_destroy(aniso3_t h);

#ifdef __cplusplus
}
#endif
#endif /* ANISO_H */
