/*
 * prc_lbm.h -- C ABI of the GB300 PRC-LBM library (libprc_lbm.so).
 *
 * The library advances the preconditioned rectangular central-moment lattice
 * Boltzmann method (PRC-LBM) of E. Yahia & K. N. Premnath, arXiv:2208.03562,
 * on the D2Q9 lattice with grid aspect ratio r = dy/dx and preconditioning
 * parameter gamma.  One time step is the fused per-node update
 *     pull-stream (App. A, streaming) with half-way bounce-back walls and a
 *     moving lid  ->  raw moments (Eq. 62), scaling S, central moments F
 *     (Sec. 4.2)  ->  preconditioned equilibria with the grid-anisotropy and
 *     cubic-velocity corrections (Eqs. 14, 30-40; App. A), local strain rates
 *     (Eqs. 43-48)  ->  relaxation (App. A)  ->  F^-1, S^-1, P^-1 (Eq. 72),
 * executed by hand-written sm_103a CUDA kernels.  No call falls back to the
 * CPU.
 *
 * Units: lattice units dx = dt = 1, dy = r.  Node (i, j), i in [0, nx) along
 * x, j in [0, ny) along y, sits at x = i + 1/2, y = (j + 1/2) r.
 * Directions 0..8: rest, E, N, W, S, NE, NW, SW, SE (Eq. 3).
 *
 * Conventions for every entry point:
 *  - every call returns an lbm_status and never aborts, traps or exits;
 *  - asynchronous failures (divergence, a bounded wait that ran out) are
 *    reported by the next call that synchronises (lbm_run, lbm_residual,
 *    lbm_info, lbm_fields, lbm_sync ...);
 *  - a handle is not thread-safe; distinct handles are independent;
 *  - "device" pointers are CUDA device addresses on the handle's device,
 *    "host" pointers are ordinary (pageable or pinned) host memory;
 *  - population arrays are [9][ny][nx] (x fastest) of FP64 *full*
 *    populations f_i (not the internal shifted storage);
 *  - field arrays are [ny][nx] FP64.
 */
#ifndef PRC_LBM_H
#define PRC_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_s *lbm_t;

typedef enum {
    LBM_F64 = 0, /* FP64 storage, FP64 collision                          */
    LBM_F32 = 1, /* FP32 storage of f_i - w_i rho0, FP32 collision        */
    LBM_F16 = 2  /* FP16 storage of f_i - w_i rho0, FP32 collision        */
} lbm_dtype;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,        /* bad argument or parameter                       */
    LBM_ENOMEM = 2,        /* device allocation failed / workspace too small  */
    LBM_ECUDA = 3,         /* a CUDA runtime call failed (see lbm_last_error) */
    LBM_EDIVERGED = 4,     /* non-finite residual or mass                     */
    LBM_ETIMEOUT = 5,      /* a bounded device wait ran out                   */
    LBM_ENOTCONVERGED = 6  /* lbm_run hit max_steps above tol                 */
} lbm_status;

typedef enum {
    LBM_BC_CAVITY = 0,   /* walls at x = 0, x = nx, y = 0; lid (u_lid, 0) at y = ny r */
    LBM_BC_CHANNEL = 1,  /* periodic in x; wall at y = 0; wall moving (u_lid, 0) on top */
    LBM_BC_PERIODIC = 2  /* periodic in x and y                                       */
} lbm_bc;

typedef enum {
    LBM_DRHO_CURRENT = 0, /* d rho from the density of the same step (default) */
    LBM_DRHO_OFF = 1      /* density-gradient terms dropped                     */
} lbm_drho;

typedef enum {
    LBM_MODEL_PRC = 0,  /* central moments: PRC-LBM (Sec. 4.2, App. A), default    */
    LBM_MODEL_PRNR = 1  /* raw moments: PRNR-LBM (Sec. 4.1, Eq.
                           LBErawmomentrectangularlattice; compared in Sec. 5.3);
                           same corrections, higher-order rates 1; runs on the
                           general kernel and the cluster engine               */
} lbm_model;

/*
 * Run parameters.  nu is the kinematic shear viscosity; the shear relaxation
 * rate follows Eq. transport-coefficients, nu = gamma q^2 c_s*^2
 * (1/omega_nu - 1/2), with q = min(1, r) and c_s*^2 = 1/3 (Eqs. 1-2).
 * omega_xi is the bulk-viscosity rate (the paper uses 1; App. A).  (fx, fy)
 * is a uniform body force entering through the gamma-scaled sources of
 * Eq. 13-central.  The density at the walls is rho0 = 1.
 */
typedef struct {
    int32_t nx, ny;
    double r, gamma, nu, u_lid;
    double omega_xi;
    double fx, fy;
    int32_t dtype; /* lbm_dtype */
    int32_t bc;    /* lbm_bc    */
    int32_t drho;  /* lbm_drho  */
    int32_t model; /* lbm_model */
} lbm_params;

/* Progress record filled by lbm_info. */
typedef struct {
    int64_t step;          /* completed time steps                              */
    int64_t residual_step; /* step at which `residual` was evaluated (0: none)  */
    double residual;       /* ||u_x(t) - u_x(t-20)||_2, FP64 (Sec. 5.2)         */
    double mass;           /* sum over nodes of rho at residual_step, FP64       */
    int32_t converged;     /* residual < tol of the last lbm_run                 */
    int32_t diverged;      /* residual or mass non-finite                        */
} lbm_info_t;

/* Fill p with the defaults: cavity walls, omega_xi = 1, no force,
 * LBM_DRHO_CURRENT, LBM_MODEL_PRC, and the given values. EINVAL if p is NULL. */
lbm_status lbm_params_init(lbm_params *p, int nx, int ny, double r, double gamma,
                           double nu, double u_lid, int dtype);

/* Check p without allocating: nx, ny >= 3; r > 0; 0 < gamma <= 1; nu > 0 with
 * 0 < omega_nu < 2; 0 < omega_xi < 2; |u_lid| < q c_s*; dtype, bc, drho in
 * range; model in range; nx * ny * 9 populations addressable. */
lbm_status lbm_params_check(const lbm_params *p);

/* Device bytes a handle needs for p (two population sets, u_x snapshot,
 * reduction scratch, status words), for lbm_create_ex. */
lbm_status lbm_workspace_bytes(const lbm_params *p, size_t *bytes);

/*
 * Create a handle with library-owned device memory (cudaMalloc on the
 * current device) and a library-owned non-blocking stream.  The state starts
 * at rest: every post-collision population equals w_i(r) rho0 (the rest
 * equilibrium of Eq. 12 at u = 0).  *out is NULL on failure.
 */
lbm_status lbm_create(int nx, int ny, double r, double gamma, double nu, double u_lid,
                      int dtype, lbm_t *out);
lbm_status lbm_create_p(const lbm_params *p, lbm_t *out);

/*
 * Create a handle on caller-owned memory: `workspace` is a device buffer of
 * at least lbm_workspace_bytes(p) bytes, 256-byte aligned, that the caller
 * keeps alive until lbm_destroy and never frees through the library;
 * `stream` is a cudaStream_t (NULL = legacy default stream) on which every
 * kernel of the handle is enqueued.  ENOMEM if workspace_bytes is too small.
 */
lbm_status lbm_create_ex(const lbm_params *p, void *workspace, size_t workspace_bytes,
                         void *stream, lbm_t *out);

/* Switch the stream later calls enqueue on (cudaStream_t). */
lbm_status lbm_set_stream(lbm_t h, void *stream);

/* Release the handle (and its memory if library-owned). NULL is ignored. */
void lbm_destroy(lbm_t h);

/* Message of the last failing call on h (or of the last failing create when
 * h is NULL); valid until the next call on h. */
const char *lbm_last_error(lbm_t h);

/*
 * Enqueue n time steps (App. A, one fused kernel per step) on h's stream;
 * asynchronous.  Every 20th step (t = 20, 40, ...) also evaluates the
 * residual ||u_x(t) - u_x(t-20)||_2 and the total mass in FP64 (Sec. 5.2).
 * Aligned blocks of 20 steps replay a captured CUDA graph.
 */
lbm_status lbm_step(lbm_t h, long n);

/*
 * Advance until the residual (evaluated every 20 steps) drops below tol, or
 * max_steps is reached; synchronises.  *steps_done (may be NULL) receives the
 * number of steps this call performed.  Returns OK when converged,
 * ENOTCONVERGED when max_steps was reached first, EDIVERGED on a non-finite
 * residual.  The device stops stepping at the step it converges (later
 * launches of the same graph batch exit at entry).
 */
lbm_status lbm_run(lbm_t h, double tol, long max_steps, long *steps_done);

/* Synchronise and return the last residual (FP64; +inf before step 20). */
lbm_status lbm_residual(lbm_t h, double *res);

/* Synchronise and return the total mass sum rho of the current state, FP64. */
lbm_status lbm_mass(lbm_t h, double *mass);

/*
 * Set the total mass sum rho to `mass` by a uniform density shift
 * f~_i += w_i(r) delta at every node (w_i(r): the rest populations, which
 * carry density and no momentum).  The method conserves mass exactly in a
 * closed domain (App. A: k~00 = k00, and bounce-back returns every
 * population); reduced-precision storage does not, because every stored
 * population is rounded.  A caller that moves a state from FP16 to wider
 * storage uses this to restore the invariant.  Synchronises.  EINVAL for a
 * mass that is not finite and positive.
 */
lbm_status lbm_set_mass(lbm_t h, double mass);

/* Synchronise and fill the progress record. */
lbm_status lbm_info(lbm_t h, lbm_info_t *info);

/* Wait for h's stream; reports asynchronous errors. */
lbm_status lbm_sync(lbm_t h);

/*
 * Macroscopic fields of the current state (App. A, hydrodynamic fields):
 * rho = sum f_i and rho u = sum f_i e_i + F / (2 gamma) of the streamed
 * populations of the last step (computed from the stored post-collision
 * populations as sum f~_i e_i - F / (2 gamma)).  rho, ux, uy are [ny][nx]
 * FP64 arrays, device pointers if on_device else host; any may be NULL.
 * Host arrays in page-locked memory that the device can address
 * (cudaHostAlloc, cudaHostRegister) are written by the kernel directly over
 * the host link; other host arrays go through a device staging buffer.
 * Synchronises.
 */
lbm_status lbm_fields(lbm_t h, double *rho, double *ux, double *uy, int on_device);

/*
 * Set the state to the equilibrium of Eq. 12 (no corrections) of the given
 * fields: f~_i = f^eq_i(rho, u) at every node.  Arrays [ny][nx] FP64, device
 * pointers if on_device else host (page-locked host arrays are read by the
 * kernel directly, as in lbm_fields).  Resets the step counter to 0 and the
 * residual snapshot to this u_x.
 */
lbm_status lbm_init_fields(lbm_t h, const double *rho, const double *ux, const double *uy,
                           int on_device);

/*
 * Set / get the post-collision populations f~_i, [9][ny][nx] FP64 (device
 * pointer if on_device else host).  Set rounds to the storage precision
 * (round-to-nearest-even) and resets the step counter and the snapshot.
 */
lbm_status lbm_set_populations(lbm_t h, const double *f, int on_device);
lbm_status lbm_get_populations(lbm_t h, double *f, int on_device);

/*
 * Checkpoint: copy the raw storage (populations, snapshot, step counter,
 * last residual) to a host buffer of lbm_save_bytes(h) bytes; lbm_load
 * restores it bitwise, so a resumed run equals an uninterrupted one.
 */
lbm_status lbm_save_bytes(lbm_t h, size_t *bytes);
lbm_status lbm_save(lbm_t h, void *host_buf, size_t n);
lbm_status lbm_load(lbm_t h, const void *host_buf, size_t n);

/*
 * Kernel variants.  Nodes at least two lattice spacings from every wall are
 * updated by a TMA-staged persistent kernel compiled in a few tile shapes
 * (variants 0 .. n-1); the edge strips ride in the same launch.  Variant -1
 * is the general wall-aware kernel everywhere.  Variant LBM_VARIANT_CLUSTER
 * (-2) is the cluster-resident engine for small grids: one thread-block
 * cluster of up to 16 CTAs keeps the whole state in distributed shared
 * memory and advances it many steps per launch (a slab of rows per CTA,
 * cluster barriers between steps); it needs every slab of >= 2 rows to fit
 * the shared memory of a CTA (e.g. up to about 50 000 nodes in FP32), and is
 * the default of lbm_create when it fits.  All variants give the same
 * populations up to round-off; the cluster engine and the general kernel
 * give bitwise the same populations.
 * lbm_variant_count / _info list the interior variants of a storage type;
 * lbm_set_variant selects one for a handle (EINVAL when the cluster engine
 * does not fit the grid).  lbm_autotune times every candidate on the
 * handle's own grid: `steps` plain steps each (rounded up to even), then
 * restores the populations, the residual snapshot, the status and the step
 * counter exactly, selects the fastest and returns it in *best;
 * ms_per_step[0..n) receives the milliseconds per step of the interior
 * variants, ms_per_step[n] that of the cluster engine (-1 when it does not
 * fit) and ms_per_step[n + 1] that of the general kernel, so the array holds
 * n + 2 values.  Either pointer may be NULL.
 * No counterpart in the paper: these choose how the same update is executed.
 */
#define LBM_VARIANT_CLUSTER (-2)
lbm_status lbm_variant_count(int dtype, int *n);
lbm_status lbm_variant_info(int dtype, int variant, int *tile_w, int *tile_h, int *threads, int *ctas_per_sm);
lbm_status lbm_get_variant(lbm_t h, int *variant);
lbm_status lbm_set_variant(lbm_t h, int variant);
lbm_status lbm_autotune(lbm_t h, int steps, int *best, double *ms_per_step);

/*
 * One time step that allocates nothing.  The paper has no counterpart: this
 * serves callers that cannot allocate device memory -- code whose device
 * memory is wholly owned by another allocator (a framework's caching
 * allocator that has reserved the GPU, so cudaMalloc fails or fragments it),
 * programs that fix their memory budget at start-up and must not allocate
 * afterwards, and tight loops that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree.
 *
 * The caller owns every buffer (device pointers on the current device):
 *   src, dst  the post-collision populations before / after the step, in the
 *             library's storage: 9 planes of ny rows of `pitch` elements,
 *             pitch = nx rounded up to a multiple of 32, each element the
 *             shifted population f_i - w_i(r) rho0 (rho0 = 1) in the storage
 *             type of p->dtype (double, float or IEEE half); src != dst;
 *   snap      ny x pitch values of u_x from the previous residual evaluation
 *             (double for LBM_F64, float otherwise); read and overwritten
 *             with the new u_x when with_residual != 0, untouched otherwise;
 *   out       when with_residual != 0: out[0] = the L2 norm of u_x minus
 *             snap over the grid and out[1] = sum of rho over the grid, both
 *             FP64.
 * The step is enqueued on `stream` (cudaStream_t, NULL = legacy default) and
 * runs the general wall-aware kernel on every node.
 *
 * Scratch: a file-scope device array of 16384 FP64 pairs (256 KiB) plus one
 * status word, held by every GPU that loads the library until the process
 * exits.  Grids with ceil(nx/32) * ceil(ny/8) > 16384 are rejected with
 * LBM_EINVAL (e.g. 2048 x 2048 is the largest square grid).  Every call
 * shares that scratch and leaves its contents behind; the call clears the
 * status word itself.  Calls whose kernels overlap on the GPU (different
 * streams, or different host threads) race on the scratch: serialise them.
 * The first call on each device looks up the scratch's device address
 * (cudaGetSymbolAddress with that device current) and keeps it for the rest
 * of the process; make that first call before any stream capture.  A device
 * reset (cudaDeviceReset) ends the context that address belongs to: after
 * one, do not call this entry point again in the same process.  The call
 * itself performs no cudaMalloc, cudaFree or allocating library call.
 * Arguments are checked before anything is enqueued: a null src, dst or
 * snap, src == dst, or with_residual without out return LBM_EINVAL.
 */
lbm_status lbm_step_noalloc(const lbm_params *p, const void *src, void *dst, void *snap, int with_residual,
                            double *out, void *stream);

/*
 * Batched engine.  A batch holds up to `capacity` independent instances
 * (slots) of one storage type, each with its own grid, parameters, residual
 * tolerance and step limit (for example the uneven cavities of a parameter
 * sweep, or the requests of a solve server).  lbm_batch_launch advances every
 * active slot with ONE persistent cooperative kernel launch (through a
 * captured CUDA graph when use_graph != 0): each step sweeps the tiles of
 * all active slots (64 x 8 nodes in pairs for FP32 / FP16 storage, 32 x 8 for
 * FP64) with the wall-aware fused update (the tile body is chosen as
 * lbm_batch_set_body describes), a bounded grid barrier separates the steps,
 * and every slot evaluates its FP64 residual on
 * its own step counter (every 20 steps, Sec. 5.2).  A slot retires on the
 * device as soon as its residual is below its tolerance (CONVERGED), is not
 * finite (DIVERGED) or it reached its step limit (MAXSTEPS); the others
 * continue.  An instance's results do not depend on the other slots: its
 * sums are reduced in a fixed order over its own tiles.  Slots may be added
 * and removed between launches (continuous batching); adding allocates the
 * slot's memory stream-ordered (lbm_batch_instance_bytes tells how much) and
 * returns ENOMEM when the device is full.  A launch is asynchronous; call
 * lbm_batch_wait before touching slots again.  A barrier that runs out
 * (about two seconds) ends the launch with LBM_ETIMEOUT.
 */
typedef struct lbm_batch_s *lbm_batch_t;

typedef enum {
    LBM_SLOT_ACTIVE = 0,
    LBM_SLOT_CONVERGED = 1,
    LBM_SLOT_DIVERGED = 2,
    LBM_SLOT_MAXSTEPS = 3,
    LBM_SLOT_EMPTY = 4,
    LBM_SLOT_STALLED = 5
} lbm_slot_state;

lbm_status lbm_batch_create(int capacity, int dtype, void *stream, lbm_batch_t *out);
void lbm_batch_destroy(lbm_batch_t b);
const char *lbm_batch_last_error(lbm_batch_t b);
lbm_status lbm_batch_instance_bytes(const lbm_params *p, size_t *bytes);
/* Fill a free slot with an instance at rest; *slot receives its index. */
lbm_status lbm_batch_add(lbm_batch_t b, const lbm_params *p, double tol, long max_steps, int *slot);
lbm_status lbm_batch_remove(lbm_batch_t b, int slot);
/*
 * Optional stall retirement of a slot (off by default; window = 0 turns it
 * off).  Every `window` steps of the slot's own counter the residual is
 * compared with the one recorded `window` steps earlier; if it is above
 * ratio times that value the slot retires as LBM_SLOT_STALLED.  This detects
 * the noise floor of a storage format (FP16 keeps 11 significant bits, and
 * its rounding noise stops the residual of Sec. 5.2 from falling further), so
 * that a caller can continue the instance in a wider format.  No counterpart
 * in the paper.  EINVAL for window < 0 or window > 0 with ratio <= 0.
 */
lbm_status lbm_batch_set_stall(lbm_batch_t b, int slot, long window, double ratio);
/*
 * Check of the failure detection; no counterpart in the paper.  For the next
 * lbm_batch_launch only:
 *   cycles  the grid barrier between steps waits at most this many SM clock
 *           cycles (0 keeps the default, about two seconds);
 *   hold    != 0: the first CTA withholds its arrival at the first barrier,
 *           so that every other CTA's wait runs out.
 * A launch whose barrier wait runs out ends early: lbm_batch_wait (and
 * lbm_batch_run) return LBM_ETIMEOUT, and the device stays usable.  With
 * hold the launch stops at its first barrier, before any slot's step counter
 * moves, so every slot keeps its state.  EINVAL for cycles < 0.
 */
lbm_status lbm_batch_set_wait_limit(lbm_batch_t b, long long cycles, int hold);
/*
 * Tile body of the batch engine (no counterpart in the paper: it chooses how
 * the same update is executed).  With LBM_BATCH_BODY_AUTO (the default), a
 * launch of at most 512 active slots, every one a cavity (LBM_BC_CAVITY) with
 * the density-gradient terms, no body force and the central-moment scheme,
 * in FP32 or FP16 storage, stages every 64 x 8 tile of each slot through TMA
 * copies into shared memory: tiles clear of the walls with the arithmetic of
 * the single-instance interior kernel, tiles at a wall with wall-aware
 * streaming from the staged windows.  Every node computes what a single
 * handle on the 64 x 8, 256-thread interior-kernel variant
 * (lbm_variant_info) computes for it, so a slot's populations are bitwise
 * that handle's.  Otherwise, or with
 * LBM_BATCH_BODY_GENERAL, every tile takes the general wall-aware body with
 * L2-served pulls, bitwise that of a single handle on variant -1.
 * lbm_batch_get_body: *tma = 1 when the next launch takes the TMA-staged body.
 * EINVAL for any other body value.
 */
#define LBM_BATCH_BODY_AUTO 0
#define LBM_BATCH_BODY_GENERAL 1
lbm_status lbm_batch_set_body(lbm_batch_t b, int body);
lbm_status lbm_batch_get_body(lbm_batch_t b, int *tma);
/*
 * Launch shape of the batch engine (no counterpart in the paper: it chooses
 * how the same update is executed; a slot's results do not depend on it).
 * The persistent grid of lbm_batch_launch is ctas_per_sm x (SM count) CTAs of
 * the tile body the launch takes, capped at the number of tiles.
 * lbm_batch_set_ctas_per_sm: 0 <= ctas_per_sm <= the largest resident count
 * of either body, else EINVAL; 0 selects the maximum of the body a launch
 * takes, and a larger value than that maximum is taken as the maximum.
 * lbm_batch_get_ctas_per_sm reports the effective value and the maximum
 * (*max_ctas_per_sm) for the body of the next launch.
 * lbm_batch_autotune times `steps` steps (1 <= steps <= 100000) of the
 * active slots at every ctas_per_sm from 1 to the maximum, each after one
 * untimed launch of the same length, then restores every slot's populations,
 * residual snapshot, step counter and state exactly and keeps the fastest
 * choice.  *best receives it; ms_per_step[c - 1] receives the milliseconds per
 * step at ctas_per_sm = c (room for *max_ctas_per_sm values).  Either pointer
 * may be NULL.  Synchronous; it allocates a device copy of the slots' state
 * for the restore (LBM_ENOMEM when that fails, with nothing changed).  With no
 * active slot it times nothing and returns LBM_OK with *best = the current
 * choice.  A timeout of the grid barrier during the timing returns
 * LBM_ETIMEOUT after the restore.
 */
lbm_status lbm_batch_set_ctas_per_sm(lbm_batch_t b, int ctas_per_sm);
lbm_status lbm_batch_get_ctas_per_sm(lbm_batch_t b, int *ctas_per_sm, int *max_ctas_per_sm);
lbm_status lbm_batch_autotune(lbm_batch_t b, int steps, int *best, double *ms_per_step);
/* Advance every active slot by up to `steps` steps (one persistent launch). */
lbm_status lbm_batch_launch(lbm_batch_t b, long steps, int use_graph);
/* Wait for the launch; *n_active receives the slots still active. */
lbm_status lbm_batch_wait(lbm_batch_t b, int *n_active);
/* lbm_batch_launch(use_graph = 1) + lbm_batch_wait. */
lbm_status lbm_batch_run(lbm_batch_t b, long steps, int *n_active);
/* Progress of a slot (as of the last wait) and its lbm_slot_state. */
lbm_status lbm_batch_query(lbm_batch_t b, int slot, lbm_info_t *info, int *state);
/* Fields / populations of a slot, conventions as lbm_fields and
 * lbm_set_populations (setting resets the slot's step counter and makes it
 * active). */
lbm_status lbm_batch_fields(lbm_batch_t b, int slot, double *rho, double *ux, double *uy, int on_device);
lbm_status lbm_batch_set_populations(lbm_batch_t b, int slot, const double *f, int on_device);
lbm_status lbm_batch_get_populations(lbm_batch_t b, int slot, double *f, int on_device);
/* Total mass of a slot's current state (FP64), and the density shift of
 * lbm_set_mass applied to a slot. */
lbm_status lbm_batch_mass(lbm_batch_t b, int slot, double *mass);
lbm_status lbm_batch_set_mass(lbm_batch_t b, int slot, double mass);

/* Derived constants: shear relaxation rate omega_nu and q = min(1, r). */
lbm_status lbm_omega_nu(const lbm_params *p, double *omega_nu);

#ifdef __cplusplus
}
#endif

#endif /* PRC_LBM_H */
