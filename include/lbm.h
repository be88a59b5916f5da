/*
 * lbm.h -- C ABI of the GB300 (sm_103a) solver for the coupled Cahn-Hilliard--Navier-Stokes
 * equations by the hybrid central-moment / BGK lattice Boltzmann scheme of
 * De Rosis, Saito, Kaneko & Abe, "Central-moments-based lattice Boltzmann scheme for coupled
 * Cahn-Hilliard--Navier-Stokes equations" (arXiv:1803.11345).
 *
 * One lattice of nx * ny D2Q9 nodes lives on one GPU.  Each node carries two population sets:
 * f (velocity; relaxed in the paper's non-orthogonal central-moment space, Eqs. 15-17, with
 * the surface-tension pressure tensor in its equilibrium, Eqs. 8, 11, 14) and g (order
 * parameter phi; BGK, Eqs. 7 and 9).  One call of lbm_step advances both sets by one time
 * step in a single fused kernel: streaming (Eqs. 4-5), phi = sum g, the isotropic stencils of
 * Eq. 12, mu = a(-phi + phi^3) - gamma Lap(phi), p0 and p~ (Eqs. 13-14), both collisions.
 *
 * Conventions for every entry point
 *   - Host arrays are owned by the caller, row-major with index y * nx + x, FP64 whatever the
 *     storage precision.  Population arrays are 9 planes of nx * ny values, plane i = direction
 *     i in the paper's order c_x = [0,1,0,-1,0,1,-1,-1,1], c_y = [0,0,1,0,-1,1,1,-1,-1].
 *   - The state kept between calls is the post-collision populations f*, g* of the last
 *     completed time step; the macroscopic fields returned are those of that time level
 *     (the collision leaves rho, rho v and phi unchanged).
 *   - Every call returns an lbm_status.  On failure the handle (or, for lbm_init, the calling
 *     thread) keeps a message readable with lbm_last_error.  A handle must not be used from two
 *     host threads at once.
 *   - Kernels run on the CUDA stream given to lbm_init (NULL = legacy default stream).
 *     lbm_step only enqueues work; lbm_fields, lbm_conservation, lbm_get_populations,
 *     lbm_set_populations and lbm_check synchronise that stream.
 */
#ifndef LBM_CH_H
#define LBM_CH_H

#include <stddef.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_ERR_PARAM = -1,     /* invalid argument; nothing was changed                        */
  LBM_ERR_OOM = -2,       /* device allocation failed or the caller's buffer is too small */
  LBM_ERR_CUDA = -3,      /* a CUDA call failed; the message names it                     */
  LBM_ERR_NONFINITE = -4, /* a node produced a non-finite rho or phi (state still readable)*/
  LBM_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up                            */
  LBM_ERR_STATE = -6      /* call not valid for this handle                                */
} lbm_status;

/* Storage precision of the populations.  Every precision computes the collision on deviations
 * d_i = f_i - w_i from the rest state (rho = 1, v = 0), with every moment carried minus its rest
 * value, so that no order-one quantity is added to the small departures that carry the flow.
 * FP64: f_i stored and computed in FP64.  FP32: d_i and g_i stored and computed in FP32.
 * FP16S / BF16S: the moving populations d_i and g_i (i >= 1) stored as 16-bit values; the rest
 * populations d_0 and g_0 stored in FP32 as closures (Eq. 10) of the rounded moving ones, so that
 * storage conserves rho and phi exactly; all arithmetic in FP32.  Whatever the precision, the FP64
 * views of the state (lbm_fields, lbm_get_populations, lbm_set_populations) carry f_i itself. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16S = 2, LBM_BF16S = 3 } lbm_precision;

/* Boundaries.  PERIODIC: both directions.  WALLS_Y: periodic in x, halfway bounce-back walls
 * at y = -1/2 (moving with x-velocity u_bottom) and y = ny - 1/2 (u_top).  For the stencils phi
 * continues into one ghost row beyond each wall: phi(x, -1) = phi(x, 0) + wet_bottom and
 * phi(x, ny) = phi(x, ny - 1) + wet_top, where wet_* is the wall gradient of phi along the
 * outward normal of Eq. 18 (0: mirror, neutral wetting, 90 degrees; > 0: the phase phi = +1
 * wets the wall).  The paper's tests use no-slip and moving walls without stating the discrete
 * form (contact-angle and shear paragraphs). */
typedef enum { LBM_PERIODIC = 0, LBM_WALLS_Y = 1 } lbm_bc;

/* How the f relaxation frequency varies with phi.  OMEGA_LINEAR is the paper's
 * omega_rho = omega_g + (phi+1)/2 (omega_l - omega_g) (paragraph after Eq. 14); TAU_LINEAR
 * interpolates tau = 1/omega the same way. */
typedef enum { LBM_OMEGA_LINEAR = 0, LBM_TAU_LINEAR = 1 } lbm_visc_interp;

/* The gradient term of k8_eq.  PROJECTED (default): -(c_s^2/2) gamma |grad phi|^2, the value of
 * the projection T^T f_eq that defines k_eq.  PRINTED: -(c_s^2/2) gamma Lap(phi) as printed in
 * Eq. 16. */
typedef enum { LBM_K8_PROJECTED = 0, LBM_K8_PRINTED = 1 } lbm_k8_form;

/* Collision of f.  CM: the paper's central-moment collision (Eq. 17; omega_4 = omega_5 =
 * omega_rho, omega_3 free, omega_6..8 = 1).  BGK: the double-BGK baseline of Eq. 6. */
typedef enum { LBM_COLLIDE_CM = 0, LBM_COLLIDE_BGK = 1 } lbm_collision;

/* Body force per unit volume (the contact-angle test applies one; the paper prints no forcing
 * scheme).  UNIFORM: F = (force_x, force_y) everywhere.  PHASE_L: F (1 + phi)/2, acting on the
 * phase phi = +1 only (with matched densities a uniform force would only build a pressure
 * gradient).  The force enters as Guo's source term S_i = w_i [(c_i - u)/c_s^2 +
 * (c_i . u) c_i / c_s^4] . F projected to central moments: k*_j = k_j + omega_j (k_j^eq - k_j)
 * + (1 - omega_j/2) (T^T S)_j, with u = (sum f c + F/2)/rho; the velocity reported by
 * lbm_fields is that u. */
typedef enum { LBM_FORCE_UNIFORM = 0, LBM_FORCE_PHASE_L = 1 } lbm_force_mode;

/* Rounding of the 16-bit stored populations.  NEAREST: round to nearest even (default).
 * STOCHASTIC: round up with probability equal to the fraction of the 16-bit unit that is dropped,
 * so that every stored value is unbiased; rounding errors then average out instead of adding up
 * where neighbouring nodes hold similar values (a slow shear).  The random bits are a counter-based
 * stream of (seed, time step, node), so runs are reproducible.  Needs FP16S or BF16S storage; not
 * available with the staged kernel.  In a batch each member draws the stream a single lattice with
 * its seed draws (the step's key is derived on the device from the batch's step counter). */
typedef enum { LBM_ROUND_NEAREST = 0, LBM_ROUND_STOCHASTIC = 1 } lbm_rounding;

/* The problem statement, in the paper's symbols (paragraph after Eq. 14 and the set-ups of
 * the bubble, contact-angle and shear tests). */
typedef struct lbm_params {
  int nx, ny;             /* lattice size, each >= 3; (pitch * ny) must fit in int32          */
  double tau_l, tau_g;    /* f relaxation times of phase l (phi = +1) and g (phi = -1);       */
                          /* nu = c_s^2 (tau - 1/2), c_s^2 = 1/3; each tau > 1/2              */
  double M, Gamma;        /* mobility and the free parameter Gamma: omega_phi from            */
                          /* M = (1/omega_phi - 1/2) Gamma c_s^2; M > 0, Gamma > 0            */
  double gamma, a;        /* free-energy constants (sigma = sqrt(8 gamma a / 9)); >= 0        */
  double omega3;          /* relaxation frequency of k3 (bulk viscosity), in (0, 2)           */
  int k8_form;            /* lbm_k8_form                                                      */
  int visc;               /* lbm_visc_interp                                                  */
  int bc;                 /* lbm_bc                                                           */
  double u_top, u_bottom; /* wall x-velocities for LBM_WALLS_Y                                */
  int prec;               /* lbm_precision                                                    */
  int collision;          /* lbm_collision                                                    */
  double wet_bottom, wet_top; /* wall gradients of phi (Eq. 18) for LBM_WALLS_Y; 0 = neutral;   */
                          /* must be 0 with LBM_PERIODIC                                       */
  double force_x, force_y;  /* body force per unit volume (0 = none)                           */
  int force_mode;         /* lbm_force_mode                                                   */
  int rounding;           /* lbm_rounding (16-bit storage)                                     */
  unsigned int seed;      /* seed of the stochastic-rounding stream                            */
} lbm_params;

typedef struct lbm_lattice lbm_lattice; /* opaque handle */

/* Fill *p with the paper's defaults: M = 0.1, Gamma = 1, gamma = a = 0.04, tau_l = tau_g = 0.8
 * (nu = 0.1), omega3 = 1, projected k8, omega-linear viscosity, periodic, FP32, CM collision,
 * round to nearest, seed 0.  nx = ny = 0 (the caller must set them). */
LBM_API void lbm_default_params(lbm_params* p);

/* Wall gradient of phi along the outward normal for a contact angle theta (radians) measured in
 * the phase phi = +1, Eq. 18: sign(pi/2 - theta) sqrt((2a/gamma) cos(t/3)(1 - cos(t/3))) with
 * t = acos(sin^2 theta).  Host function; NaN for gamma <= 0 or a < 0. */
LBM_API double lbm_wall_gradient(double theta, double a, double gamma);

/* Device bytes one lattice needs (both population copies plus a small status block) when the
 * caller supplies the memory to lbm_init.  Returns LBM_ERR_PARAM for invalid parameters. */
LBM_API int lbm_state_bytes(const lbm_params* p, size_t* bytes);

/* Create a lattice and set its state from the initial fields, following the paper's start
 * ("fluid initially at rest, density 1", stability paragraph): the populations are the
 * equilibria of Eqs. 8-10 built from phi0 (with the Eq. 12 stencils), ux0, uy0, rho0, after
 * one collision at t = 0.
 *   phi0            host, nx*ny FP64, required, finite.
 *   ux0, uy0, rho0  host, nx*ny FP64 or NULL (NULL means 0, 0 and 1).
 *   device_buffer   NULL: the library allocates (cudaMalloc) and frees in lbm_free.
 *                   Otherwise a device pointer, 256-byte aligned, of buffer_bytes >=
 *                   lbm_state_bytes(); the caller keeps ownership and must keep it alive
 *                   until lbm_free.
 *   stream          cudaStream_t to run on, or NULL.
 *   out             receives the handle; *out is NULL on failure.
 * Errors: LBM_ERR_PARAM (bad parameters or non-finite input), LBM_ERR_OOM, LBM_ERR_CUDA. */
LBM_API int lbm_init(const lbm_params* p, const double* phi0, const double* ux0, const double* uy0,
             const double* rho0, void* device_buffer, size_t buffer_bytes, void* stream,
             lbm_lattice** out);

/* Advance n >= 0 time steps (Eqs. 4-5 streaming, then both collisions), one fused kernel launch
 * per step, asynchronously on the lattice's stream.  Errors: LBM_ERR_PARAM (n < 0),
 * LBM_ERR_CUDA (launch failure). */
LBM_API int lbm_step(lbm_lattice* h, int n);

/* Copy the macroscopic fields rho = sum f, v = sum f c / rho, phi = sum g (paragraph after
 * Eq. 14) of the current time level into host arrays of nx*ny FP64; any pointer may be NULL.
 * Synchronises.  Returns LBM_ERR_NONFINITE if any step since the last check produced a
 * non-finite rho or phi (the fields are still copied). */
LBM_API int lbm_fields(lbm_lattice* h, double* rho, double* ux, double* uy, double* phi);

/* FP64 totals over the lattice, computed on the GPU in a fixed order (deterministic):
 * sum phi, sum rho and the momentum sum rho v (mom[0], mom[1]); any pointer may be NULL.
 * The scheme conserves sum phi and sum rho exactly (Eq. 10 closures, k_0 invariance) and the
 * momentum on a periodic lattice (k_1 = k_2 = 0 invariance, discussion after Eq. 17).
 * Synchronises. */
LBM_API int lbm_conservation(lbm_lattice* h, double* sum_phi, double* sum_rho, double* mom);

/* Raw post-collision populations f*, g* as 9 planes of nx*ny FP64 each (host, caller-owned);
 * either pointer may be NULL.  Synchronises. */
LBM_API int lbm_get_populations(lbm_lattice* h, double* f, double* g);

/* Replace the state with the given post-collision populations (same layout), e.g. to resume a
 * checkpoint.  16-bit storage rounds them.  Synchronises.  LBM_ERR_PARAM on NULL input. */
LBM_API int lbm_set_populations(lbm_lattice* h, const double* f, const double* g);

/* Synchronise and report whether any step since the last check had a bounded device-side wait
 * give up (LBM_ERR_TIMEOUT, reported first), produced a non-finite rho or phi
 * (LBM_ERR_NONFINITE), or a CUDA error occurred (LBM_ERR_CUDA); clears the flags.  After
 * LBM_ERR_TIMEOUT the steps enqueued since the last check may be incomplete: the handle stays
 * usable, but its state is undefined until lbm_set_populations restores one (a checkpoint). */
LBM_API int lbm_check(lbm_lattice* h);

/* Probes a bulk-copy wait of the staged kernels (LBM_KERNEL_STAGED, LBM_KERNEL_PAIR_STAGED) makes
 * before it gives up.
 * probes < 0 restores the default, 2^22 probes, each a short hardware-timed suspend: far beyond
 * any legitimate copy latency and well under a second.  probes = 0 makes every wait of the
 * kernel's main loop give up at once; it exists to exercise the timeout path.  A wait that gives
 * up makes its CTA stop stepping: it sets the lattice's timeout flag, waits (always with the
 * default limit) for the copies it has in flight, and returns, so the GPU stays usable and the
 * next lbm_check reports LBM_ERR_TIMEOUT.  Affects later lbm_step calls only; the other kernels
 * have no such waits.  Errors: LBM_ERR_PARAM (h NULL). */
LBM_API int lbm_set_wait_limit(lbm_lattice* h, int probes);

/* Fused-step kernel choice.  AUTO: the fastest measured on GB300 — PAIR for 16-bit storage on
 * lattices of 4 M nodes or more where it can serve them, else GENERIC, each with its default tile
 * (lbm_autotune times all of them).  GENERIC: populations pulled straight from global memory; plane offsets are formed
 * in 32-bit arithmetic while a population copy is under 4 GiB, in 64-bit beyond.  GENERIC_WIDE:
 * the same kernel with 64-bit offsets for any lattice (what GENERIC runs for copies of 4 GiB or
 * more; selectable so that this path can be checked on small lattices).  PAIR: 16-bit storage
 * only, two neighbouring nodes per thread so that 16-bit populations move as 32-bit words (bx x by
 * threads cover 2 bx columns; with walls a second launch steps the two wall rows); needs even nx and
 * a copy under 4 GiB.  STAGED: whole rows
 * staged in shared memory by bulk copies; needs nx to be a multiple of 16 bytes / stored element
 * size (2 columns FP64, 4 FP32, 8 16-bit).  PAIR_STAGED: the PAIR arithmetic with every row it
 * pulls from staged in shared memory by bulk copies (128 x 1 threads, 256 columns per CTA; depth 1
 * or 2 rows of prefetch); 16-bit storage on periodic lattices with nx a multiple of 8 and a copy
 * under 4 GiB; same results as PAIR. */
typedef enum {
  LBM_KERNEL_AUTO = 0,
  LBM_KERNEL_GENERIC = 1,
  LBM_KERNEL_STAGED = 2,
  LBM_KERNEL_GENERIC_WIDE = 3,
  LBM_KERNEL_PAIR = 4,
  LBM_KERNEL_PAIR_STAGED = 5
} lbm_kernel;

/* Override the kernel and its tile: bx x by threads per CTA (0, 0 = default for the variant),
 * depth = bands of prefetch of the staged kernel (0 = default), rows = lattice rows per CTA
 * (0 = sized so the grid fills the GPU in one wave; for PAIR on a periodic lattice up to 4 waves
 * of at least 32 rows).
 * Affects later lbm_step calls only.  Every variant performs the same operations per node, so
 * results depend on the choice only through rounding: separately compiled kernels may fuse
 * different multiply-adds (1-2 ulp per step in FP64 or FP32; PAIR computes in packed FP32
 * instructions with its own fusions, and a 16-bit rounding can then land differently).
 * LBM_ERR_PARAM for a combination without a compiled kernel or a lattice the variant cannot
 * serve. */
LBM_API int lbm_set_kernel(lbm_lattice* h, int variant, int bx, int by, int depth, int rows);

/* The kernel and tile lbm_step uses now (variant is GENERIC, GENERIC_WIDE, PAIR, STAGED or
 * PAIR_STAGED); NULL
 * pointers skipped. */
LBM_API int lbm_get_kernel(const lbm_lattice* h, int* variant, int* bx, int* by, int* depth, int* rows);

/* Time the compiled kernels and tiles on this lattice (trial_steps launches each, after a warm-up)
 * and keep the fastest for later lbm_step calls; *best_ms (may be NULL) receives its time per
 * step.  Trials relaunch the step from the current state into the spare copy, so the state and
 * lbm_time are unchanged.  Winners are cached per (precision, nx, ny, boundary, SM count) for the
 * process: later lattices of the same shape start with the winner. */
LBM_API int lbm_autotune(lbm_lattice* h, int trial_steps, double* best_ms);

/* ---------------------------------------------------------------------------------------------
 * Batches: many independent lattices (a batched parameter sweep; the paper runs one
 * lattice at a time).  Every member has its own lbm_params (sizes, viscosities, gamma, a, walls...)
 * but all share one precision.  One launch of a persistent kernel per time step advances every
 * member: resident CTAs walk a work list of tiles of roughly equal node count drawn from all
 * members, largest first.  Runs of 16 steps are captured once in a CUDA graph and replayed.
 * Each member computes exactly what a single lattice with the same parameters computes. */
typedef struct lbm_batch lbm_batch;

/* Device bytes of a batch (all members' population copies, tables, flags). */
LBM_API int lbm_batch_state_bytes(const lbm_params* params, int count, size_t* bytes);

/* Create a batch: params[count], phi0[count] (host arrays of nx*ny FP64 each; velocity 0, density 1
 * as in the paper's set-ups), device_buffer/buffer_bytes as in lbm_init (NULL = library allocates),
 * stream (NULL = the batch creates its own non-blocking stream; graphs cannot be captured on the
 * legacy default stream).  Errors as lbm_init; the message names the member. */
LBM_API int lbm_batch_init(const lbm_params* params, int count, const double* const* phi0, void* device_buffer,
                           size_t buffer_bytes, void* stream, lbm_batch** out);

/* Advance every member by n >= 0 steps (asynchronous). */
LBM_API int lbm_batch_step(lbm_batch* b, int n);

/* Fields / populations of one member, as lbm_fields / lbm_get_populations (synchronise). */
LBM_API int lbm_batch_fields(lbm_batch* b, int member, double* rho, double* ux, double* uy, double* phi);
LBM_API int lbm_batch_get_populations(lbm_batch* b, int member, double* f, double* g);

/* A member's macroscopic state as a device array, without a host round trip (to couple the solver
 * with other GPU code, e.g. a learned model that advances the fields between solver windows).
 * state: device pointer (4-byte aligned, caller-owned) to nx*ny nodes of 3 FP32 values each,
 * node (x, y) at 3 * (y * nx + x): phi, v_x, v_y.  lbm_batch_set_state replaces the member's
 * populations by the equilibria of Eqs. 8-10 built from those fields with rho = 1 (the Eq. 12
 * stencils of phi, then one collision: the start lbm_init makes); lbm_batch_get_state writes the
 * member's phi and velocity (as lbm_batch_fields) into state.  Both only enqueue work on the
 * batch's stream (no synchronisation): the caller orders its own streams against it.  Errors:
 * LBM_ERR_PARAM (bad member, NULL or misaligned state), LBM_ERR_CUDA. */
LBM_API int lbm_batch_set_state(lbm_batch* b, int member, const float* state);
LBM_API int lbm_batch_get_state(lbm_batch* b, int member, float* state);

/* Synchronise; nonfinite[count] (may be NULL) receives 1 for members that produced a non-finite
 * rho or phi since the last check (flags are then cleared); returns LBM_ERR_NONFINITE if any did. */
LBM_API int lbm_batch_check(lbm_batch* b, int* nonfinite);

/* Tile of the batch kernel: bx x by threads per CTA and about target_nodes nodes per work item
 * (>= 2048).  Tiles: 32x4, 64x2, 64x4, 128x1, 128x2, 256x1. */
LBM_API int lbm_batch_set_tile(lbm_batch* b, int bx, int by, int target_nodes);
LBM_API int lbm_batch_get_tile(const lbm_batch* b, int* bx, int* by, int* target_nodes, int* items, int* grid);

/* Kernel of the batch: LBM_KERNEL_GENERIC (the one-node tile, 64 x 4 until lbm_batch_set_tile or
 * lbm_batch_autotune picks another) or LBM_KERNEL_PAIR (the paired 16-bit tile of lbm_set_kernel:
 * 128 x 1 threads, 256 columns per work item; every member periodic 16-bit with even nx), with
 * about target_nodes nodes per work item (>= 2048).  A member of a PAIR batch steps exactly as a
 * single lattice with LBM_KERNEL_PAIR (same words, same arithmetic, same stochastic-rounding keys).
 * A new batch starts with PAIR where it can serve it, else with the one-node 64 x 4 tile (or with
 * the autotuner's cached winner for batches of the same member sizes).
 * Errors: LBM_ERR_PARAM (other variants, members the variant cannot serve, target below 2048). */
LBM_API int lbm_batch_set_kernel(lbm_batch* b, int variant, int target_nodes);
LBM_API int lbm_batch_get_kernel(const lbm_batch* b, int* variant);

/* Time every tile x item size (trial_steps launches each, state unchanged as in lbm_autotune; the
 * paired tile too where it can serve the batch), keep the fastest, cache it for batches of the
 * same member sizes; *best_ms = its step time. */
LBM_API int lbm_batch_autotune(lbm_batch* b, int trial_steps, double* best_ms);

/* Completed steps; last error (b = NULL: this thread's last lbm_batch_init failure); release. */
LBM_API long long lbm_batch_time(const lbm_batch* b);
LBM_API const char* lbm_batch_last_error(const lbm_batch* b);
LBM_API void lbm_batch_free(lbm_batch* b);

/* Conservation totals of a population state in device memory, computed without allocating.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a host framework that owns all device memory and hands out a fixed arena, a
 * process held to a device-memory budget, or a state restored into a preallocated slab -- and
 * that hold no lattice handle whose spare population copy lbm_conservation could use as scratch.
 * It runs the same deterministic FP64 reduction as lbm_conservation and gives bit-identical
 * totals for the same state.
 *   state   device pointer (16-byte aligned) to one population copy in the layout lbm_init
 *           builds: pitch = nx rounded up to a multiple of 32, plane = pitch * ny elements;
 *           FP64: 18 planes (f_0..f_8, g_0..g_8); FP32: 18 planes (f_0 - w_0 .. f_8 - w_8,
 *           g_0..g_8); FP16S/BF16S: 16 16-bit planes (f_1 - w_1 .. f_8 - w_8, then g_1..g_8)
 *           followed by two FP32 planes (f_0 - w_0, g_0).  For a lattice created
 *           on a caller-supplied device_buffer, each population copy takes
 *           (lbm_state_bytes(p) - 256) / 2 bytes and the state after t = lbm_time(h) steps is the
 *           copy at device_buffer + (t % 2) * that size.
 *   nx, ny, prec  the lattice the state belongs to.
 *   totals  host array of 4 doubles: sum phi, sum rho, sum rho v_x, sum rho v_y.
 *   stream  cudaStream_t to run on, or NULL; the call synchronises it.
 * Scratch: a library-wide static device array of 1024 * 4 + 4 doubles (32 KiB), which every GPU
 * that loads the library keeps until the process exits.  The kernel launches at most 1024 blocks
 * whatever the lattice size, so every lattice the library accepts fits; lattices beyond the
 * library's limit (pitch * ny >= 2^31) are rejected with LBM_ERR_PARAM.  No call allocates or
 * frees device memory.  All calls share the array and it keeps the last call's contents; every
 * call overwrites what it reads, so nothing needs clearing, but calls that overlap on the GPU
 * (other streams, other host threads) race on it.  The first call on each device looks up the
 * array's device address with that device current and keeps it for the process; make that first
 * call before any stream capture.  A device reset (cudaDeviceReset) after that call is not
 * supported: the kept address would be stale.
 * Errors: LBM_ERR_PARAM (NULL pointers, bad sizes or precision, misaligned state), LBM_ERR_CUDA;
 * the message is readable with lbm_last_error(NULL) on the calling thread. */
LBM_API int lbm_totals_noalloc(const void* state, int nx, int ny, int prec, double* totals, void* stream);

/* Time level reached (number of completed steps since lbm_init). */
LBM_API long long lbm_time(const lbm_lattice* h);

/* Message of the last failure on this handle, or of the calling thread's last lbm_init failure
 * when h is NULL.  Never NULL; the empty string when there was none. */
LBM_API const char* lbm_last_error(const lbm_lattice* h);

/* Release the handle and any memory the library allocated.  NULL-safe. */
LBM_API void lbm_free(lbm_lattice* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_CH_H */
