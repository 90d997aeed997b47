/*
 * cgevap.h -- C ABI of the GB300 (sm_103a) library for the two-component colour-gradient (CG)
 * lattice Boltzmann step with reaction-limited (RL) evaporation of Nath, Aouane and Harting,
 * "Reaction-limited evaporation for the color-gradient lattice Boltzmann model",
 * arXiv:2412.14859.
 *
 * One timestep (cgevap_step) is one fused CUDA kernel performing, in the order of the method
 * summary at the end of the paper's Sec. II.B:
 *   streaming (Eq. Stream, pull form, halfway bounce-back at walls, Sec. III first paragraph),
 *   site selection (|F| > Gamma with |F| of the previous step, Sec. II.B; or a phase-field band),
 *   mass exchange of the rest populations f0^r -= varphi, f0^b += varphi (Eq. exchange) with
 *   varphi = phi / S-bar (Eq. relation), moments, colour gradient (Eq. cg, isotropic stencil),
 *   BGK collision with harmonic tau (Eq. collision, Eq. feq), perturbation (Eq. perturb) and
 *   recoloring (Eq. recolor).  The evaporated mass is summed in FP64 on the device.
 *
 * Conventions for every function:
 *   - return 0 (CGEVAP_OK) on success or a negative CGEVAP_ERR_* code; nothing throws, aborts or
 *     exits across this boundary; cgevap_last_error(sim) gives a message for the last failure
 *     on that handle (cgevap_last_error(NULL) for failures of cgevap_create and of
 *     cgevap_step_static_scratch on the calling thread);
 *   - pointers named dev_* are CUDA device pointers owned by the caller, host_* host pointers;
 *     inputs are copied into library-owned buffers, outputs are written into the caller's buffers;
 *   - work is enqueued on the handle's stream (cgevap_set_stream) and is asynchronous unless the
 *     function says it synchronises;
 *   - field layouts are C order [z][y][x] with x fastest (nz = 1 for D2Q9); population arrays
 *     exchanged with the caller are [k][i][z][y][x], k = 0 red (the evaporating liquid), 1 blue;
 *   - the stored state is the post-recoloring population f_i^{k*} of the last completed step.
 */
#ifndef CGEVAP_H
#define CGEVAP_H

#include <stddef.h>
#include <stdint.h>

#if defined(CGEVAP_BUILD) && defined(__GNUC__)
#define CGEVAP_API __attribute__((visibility("default")))
#else
#define CGEVAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define CGEVAP_OK 0
#define CGEVAP_ERR_ARG -1          /* invalid argument or parameter set                       */
#define CGEVAP_ERR_CUDA -2         /* a CUDA runtime call or kernel launch failed             */
#define CGEVAP_ERR_OOM -3          /* device or host allocation failed                        */
#define CGEVAP_ERR_TIMEOUT -4      /* a bounded device-side wait gave up                      */
#define CGEVAP_ERR_NAN -5          /* the health check found a non-finite or negative density */
#define CGEVAP_ERR_UNSUPPORTED -6  /* valid request the library does not support               */
#define CGEVAP_ERR_IO -7           /* checkpoint file could not be read or written            */

/* ---- evaporation-site rules ---- */
#define CGEVAP_SITES_GRADIENT 0 /* site if |F| of the previous step > threshold (Sec. II.B)     */
#define CGEVAP_SITES_BAND 1     /* site if |rho^N| after streaming < threshold (phase band)     */
#define CGEVAP_SITES_GIVEN 2    /* site where bit0 of the site bytes read by the step is set: a
                                   recorded site set replayed (cgevap_set_mask before each step) */

/* ---- population storage formats (internal layouts; all arithmetic as stated) ---- */
#define CGEVAP_F64 0      /* FP64 storage, FP64 arithmetic                                     */
#define CGEVAP_F32 1      /* FP32 storage, FP32 arithmetic                                     */
#define CGEVAP_F16DEV 2   /* FP32 rest populations + FP16 deviations of the moving ones from
                             the rest state of the cell's own rest population, FP32 arithmetic;
                             each step sums each colour's pulled mass without rounding error
                             and sets the stored rest population so that the cell's stored mass
                             of each colour equals that exact mass up to the final rounding of
                             the rest population and of each decode (rounding losses of the FP32
                             collision and of the 16-bit encode taken back), in every kernel
                             variant */
#define CGEVAP_BF16DEV 3  /* as F16DEV with BF16 deviations                                    */
#define CGEVAP_F32RC 4    /* "recolour on pull": per cell the Q colour-blind post-collision
                             populations and one record (rho_r / rho, V) in FP32, from which the
                             next step forms each colour as Eq. (recolor) does; Q + 4 floats per
                             cell instead of 2Q, FP32 arithmetic.  An imported state (init,
                             set_populations) is held as FP32 pairs until the next step. */
#define CGEVAP_F16RC 5    /* the populations of F32RC stored as FP16 deviations from the
                             lattice-weight rest state of the cell, with FP32 arithmetic: per
                             cell an FP32 rest pair (f_0^r, f_0^b), the FP32 record (rho_r / rho,
                             V), an FP32 rest-state scale Rf and Q - 1 FP16 values
                             s (f_i - r_i Rf) of the colour-blind post-collision populations
                             (f_i^eq(rho, 0) = r_i Rf, r_i = A_i / A_1, s a power of two), which
                             the next step splits into colours as Eq. (recolor) does.  Each
                             step carries each colour's mass exactly: the pulled colour parts
                             are summed without rounding error and the stored rest pair is set
                             so that what a cell passes on of each colour equals its exact
                             post-exchange mass up to the rounding of the rest pair.
                             2 (28 + 2 (Q - 1)) + 1 bytes per lattice update (129 for D3Q19).
                             An imported state is held as FP32 pairs until the next step. */
#define CGEVAP_BF16RC 6   /* as F16RC with BF16 values (s = 1)                                */
#define CGEVAP_F32X 7     /* the FP32 pairs of CGEVAP_F32 with each colour's mass carried
                             exactly through the step: the pulled pairs are summed per colour
                             without rounding error, the exchange's rounding is kept, and the
                             rest pair is stored as the exact post-exchange colour masses less
                             the stored moving pairs.  Same layout and bytes as F32; at small
                             fluxes F32 removes less red mass than the ledger records (the
                             exchange's phi / S-bar is rounded against rest populations of
                             order 0.1 - 1 at every site and step), F32X does not. */

/* ---- element types of caller buffers ---- */
#define CGEVAP_DTYPE_F64 0
#define CGEVAP_DTYPE_F32 1

typedef struct cgevap_params {
  int q;                  /* 9 (D2Q9, nz == 1) or 19 (D3Q19)                                  */
  int nx, ny, nz;         /* lattice size, each >= 1; nx*ny*nz < 2^31                          */
  int periodic[3];        /* per axis x,y,z: 1 periodic, 0 walls just outside both ends        */
  double rho_r_in;        /* initial bulk density of red; alpha_k from these (Sec. II.A)      */
  double rho_b_in;        /* initial bulk density of blue                                     */
  double tau_r, tau_b;    /* component relaxation times, > 1/2 (Sec. II.A)                    */
  double sigma;           /* surface tension; perturbation amplitude (9/4) sigma / tau        */
  double beta;            /* recoloring parameter in [0, 1] (Eq. recolor)                     */
  int site_rule;          /* CGEVAP_SITES_GRADIENT, CGEVAP_SITES_BAND or CGEVAP_SITES_GIVEN     */
  double threshold;       /* Gamma (gradient rule) or theta (band rule)                       */
  double sbar;            /* S-bar > 0 of Eq. (relation); varphi = phi / S-bar                */
  int storage;            /* CGEVAP_F64, F32, F16DEV, BF16DEV, F32RC, F16RC, BF16RC or F32X  */
} cgevap_params;

typedef struct cgevap_ledger {
  double evaporated;      /* cumulative FP64 sum of varphi over (site, step) pairs             */
  double last_removed;    /* FP64 sum of varphi over the sites of the last step                */
  long long site_steps;   /* cumulative number of (site, step) pairs                           */
  long long last_sites;   /* number of sites at the last step                                  */
  long long steps;        /* steps taken since create / reset / load                           */
} cgevap_ledger;

typedef struct cgevap_sim cgevap_sim;

/* Validate p and allocate a simulation on the current CUDA device: two population buffers, two
 * site-mask buffers, the FP64 ledger and its per-block scratch.  Populations start at zero, the
 * flux at zero, the stream is the legacy default stream.  Errors: ARG (invalid p: q not 9/19,
 * nz != 1 with q = 9, a size < 1, tau <= 1/2, beta outside [0,1], densities or S-bar <= 0,
 * unknown rule or storage), OOM, CUDA.  *out is NULL on failure. */
CGEVAP_API int cgevap_create(const cgevap_params* p, cgevap_sim** out);

/* Synchronise the handle's stream and free everything it owns.  NULL is accepted. */
CGEVAP_API int cgevap_destroy(cgevap_sim* sim);

/* Message for the last failure on sim (or of cgevap_create when sim is NULL); never NULL. */
CGEVAP_API const char* cgevap_last_error(const cgevap_sim* sim);

/* Parameters the handle was created with. */
CGEVAP_API int cgevap_get_params(const cgevap_sim* sim, cgevap_params* out);

/* Enqueue all later work on this cudaStream_t (NULL = legacy default stream). */
CGEVAP_API int cgevap_set_stream(cgevap_sim* sim, void* cuda_stream);

/* Copy a per-cell solid flag (uint8, nonzero = solid, [z][y][x]) or clear it (dev_solid NULL).
 * Solid cells hold no populations; fluid links into them bounce back halfway (Sec. III) and
 * they contribute the evaluating cell's rho^N to the colour gradient (neutral wetting).
 * Populations of cells that become solid are zeroed. */
CGEVAP_API int cgevap_set_solid(cgevap_sim* sim, const uint8_t* dev_solid);

/* Evaporative flux phi (Eq. surface_flux): a scalar (dev_phi_field NULL) or a per-cell field
 * [z][y][x] of dtype CGEVAP_DTYPE_F64/F32 that is copied.  Each site loses varphi = phi / S-bar
 * of red rest population per step (Eq. relation, Eq. exchange); negative phi condenses. */
CGEVAP_API int cgevap_set_flux(cgevap_sim* sim, double phi, const void* dev_phi_field, int dtype);

/* Heated-substrate flux (Sec. III.C, Eq. heated): a per-cell flux field
 *   Phi(x) = phi_s / (K + h(x) / length),
 * where h(x) is the liquid height of the column through x along the substrate normal (z in 3D,
 * y in 2D): the sum of rho_r / (rho_r + rho_b) over the column's fluid cells, solid cells
 * excluded.  `length` is the length scale R0 of h* = h / R0, K > 0 the kinetic constant.  The
 * field is computed from the current state now, and again from the state before a step once
 * `every` steps have passed since the last computation (every = 1: before every step); after
 * cgevap_init_equilibrium / cgevap_set_populations the next step recomputes it.  Two kernels of
 * fixed summation order compute it, so runs repeat bit for bit.  The mode stays on until
 * cgevap_set_flux or cgevap_load replaces the flux.  Each site then moves Phi / S-bar (Eq.
 * relation).  Errors: ARG (non-finite phi_s, K <= 0, length <= 0, every < 1, or a periodic
 * substrate-normal axis), OOM, CUDA.  The adjoint entry points reject this mode (UNSUPPORTED). */
CGEVAP_API int cgevap_set_flux_heated(cgevap_sim* sim, double phi_s, double K, double length, int every);

/* Blue pressure outlets for density-contrast runs (Sec. III.B.2; the boundary condition of Zou
 * and He) on the first (rho_lo) and last (rho_hi) plane of the wall-normal axis -- z in 3D, y in
 * 2D, which must have walls.  A density <= 0 leaves that end a halfway bounce-back wall (the
 * default).  Before every step, at each fluid cell of an outlet plane, the blue populations that
 * enter from outside are rebuilt from the cell's known pulled ones so that the blue density is
 * the given one and the blue velocity along the plane is zero (mass and normal momentum balance,
 * bounce-back of the normal non-equilibrium part); red keeps the bounce-back (no red passes).
 * The setting persists across cgevap_init_equilibrium, cgevap_set_populations and cgevap_load and
 * is not written by cgevap_save.  Errors: ARG (non-finite density, a periodic wall-normal axis,
 * two outlets on a single plane).  The adjoint entry points reject it (UNSUPPORTED). */
CGEVAP_API int cgevap_set_outlets(cgevap_sim* sim, double rho_lo, double rho_hi);

/* The flux field the next step reads (FP64 [z][y][x] into dev_out; a scalar flux fills every
 * cell with phi).  With a heated flux it is the field computed at the last recomputation. */
CGEVAP_API int cgevap_get_flux_field(cgevap_sim* sim, double* dev_out);

/* Initial state at rest: rho_r = rho_r_in (1 + rhoN0) / 2, rho_b = rho_b_in (1 - rhoN0) / 2,
 * f_i^k = rho_k phi_i(alpha_k) (Eq. feq with u = 0) plus dev_noise [k][i][z][y][x] if not NULL
 * (dtype noise_dtype).  dev_rhoN0 is FP64 [z][y][x].  Also resets the ledger and, for the
 * gradient rule, sets the first step's sites from |F| of this state. */
CGEVAP_API int cgevap_init_equilibrium(cgevap_sim* sim, const double* dev_rhoN0, const void* dev_noise,
                            int noise_dtype);

/* Replace the state by dev_f [k][i][z][y][x] (dtype F64 or F32), encoded into the storage
 * format; recomputes the gradient-rule sites of the next step from this state. */
CGEVAP_API int cgevap_set_populations(cgevap_sim* sim, const void* dev_f, int dtype);
/* Same from host memory (pageable or pinned); synchronises the stream. */
CGEVAP_API int cgevap_set_populations_host(cgevap_sim* sim, const void* host_f, int dtype);

/* Decode the state into dev_f [k][i][z][y][x] (dtype F64 or F32). */
CGEVAP_API int cgevap_get_populations(cgevap_sim* sim, void* dev_f, int dtype);

/* Advance nsteps >= 0 timesteps (asynchronous; the ledger is updated on the device). */
CGEVAP_API int cgevap_step(cgevap_sim* sim, int nsteps);

/* Local macroscopic fields of the state (FP64, each [z][y][x], u is [3][z][y][x]); any pointer
 * may be NULL.  rho_k = sum_i f_i^k, u = sum_i f_i c_i / rho, rho^N = (rho_r - rho_b) / rho
 * (Sec. II.A); these equal the post-exchange moments of the last step. Solid cells give 0. */
CGEVAP_API int cgevap_get_macros(cgevap_sim* sim, double* dev_rho_r, double* dev_rho_b, double* dev_u,
                      double* dev_rhoN);

/* Site byte per cell [z][y][x] of the last step: bit0 = site at that step, bit1 = gradient
 * rule: |F| > Gamma at that step (site at the next one), bit2 = that step's decision value lay
 * within 1e-6 of the threshold, bit3 = gradient rule: | |F| - Gamma | < 1e-6 at that step. */
CGEVAP_API int cgevap_get_mask(cgevap_sim* sim, uint8_t* dev_mask);

/* Replace the site bytes the next step reads with dev_mask [z][y][x] (copied).  Under
 * CGEVAP_SITES_GIVEN the next step's sites x_I are the cells whose bit0 is set (Eq. exchange with
 * a site set recorded by cgevap_get_mask after each step of an earlier run, so that a run can be
 * repeated with x_I held fixed); under the gradient rule bit1 is the next step's site.
 * Errors: ARG. */
CGEVAP_API int cgevap_set_mask(cgevap_sim* sim, const uint8_t* dev_mask);

/* Liquid volume of the state, V = sum over fluid cells of (1 + rho^N)/2 with rho^N =
 * (rho_r - rho_b)/rho of the stored populations (Sec. II.A; the drop size whose evolution the
 * paper's Sec. III compares with Eq. sphere_r), written as one FP64 value to dev_out[0].
 * Deterministic (fixed reduction order).  Errors: ARG, OOM, CUDA. */
CGEVAP_API int cgevap_volume(cgevap_sim* sim, double* dev_out);

/* Copy the FP64 ledger to the host; synchronises the stream.  Returns CGEVAP_ERR_TIMEOUT (and
 * clears the flag) if a bounded device-side wait of a step since the last call gave up. */
CGEVAP_API int cgevap_get_ledger(cgevap_sim* sim, cgevap_ledger* host_out);

/* The same record, copied asynchronously on the simulation's stream into host_out, which the
 * caller owns: page-locked host memory (else the copy may run synchronously), valid and
 * unread until the stream has passed this point.  A loop of steps can thus read the ledger after
 * every step without waiting for the GPU.  The timeout flag of a device-side wait is neither
 * read nor cleared: cgevap_get_ledger reports it.  Errors: ARG (NULL), CUDA. */
CGEVAP_API int cgevap_get_ledger_async(cgevap_sim* sim, cgevap_ledger* host_out);

/* Zero the ledger (asynchronous). */
CGEVAP_API int cgevap_reset_ledger(cgevap_sim* sim);

/* Health check: CGEVAP_ERR_NAN if any fluid cell has a non-finite population or a non-positive
 * total density, else OK; synchronises the stream. */
CGEVAP_API int cgevap_check_health(cgevap_sim* sim);

/* Write / read a checkpoint: a versioned header, the parameters, the state decoded to FP64,
 * the site bytes, the flux, the solid flags and the ledger.  Loading needs a handle created
 * with the same parameters; running n steps, saving, loading and running m more equals
 * running n + m steps bit for bit.  Both synchronise the stream. Errors: IO, ARG. */
CGEVAP_API int cgevap_save(cgevap_sim* sim, const char* path);
CGEVAP_API int cgevap_load(cgevap_sim* sim, const char* path);

/* Site threshold for a target S-bar (Sec. II.B): the threshold (Gamma for the gradient rule,
 * theta for the band rule) at which an evaporating flat interface loses mass at the prescribed
 * rate, Eq. (satisfy) with Eq. (relation): the time-averaged number of sites per step equals
 * target_sbar x A.  Procedure: a flat interface normal to y on p's box (red below y = 5 ny/8,
 * tanh profile; A = nx nz, or 2 nx nz with a periodic y axis) is equilibrated with the flux off
 * until u changes by less than 1e-7 over 100 steps (at most 5000 steps, Sec. III), then for each
 * trial threshold an evaporation run with flux phi from that state to t* = 1/2 (the interface
 * recedes by half its height) gives the mean site count; the threshold is bisected (30 trials)
 * until that count matches.  p supplies the physics, box, site rule and storage (F64 or F32;
 * p->threshold and p->sbar are not used).  out_threshold: the threshold; out_sbar (may be NULL):
 * the S-bar measured at it.  Synchronous; allocates and frees its own handle.  Errors (message in
 * cgevap_last_error(NULL)): ARG (NULL pointers, phi or target_sbar not > 0, ny < 16, a target
 * outside what any threshold reaches), UNSUPPORTED (16-bit storage), OOM, CUDA. */
CGEVAP_API int cgevap_calibrate_threshold(const cgevap_params* p, double phi, double target_sbar,
                                          double* out_threshold, double* out_sbar);

/* Select the fused-step kernel: family -1 automatic (the default at create: currently the
 * register-pipelined kernel, measured faster), 0 the
 * register-pipelined kernel (every storage, any nx), 1 the bulk-copy pipelined kernel (FP32
 * storage and even nx); variant picks a tile shape / pipeline depth of that family (0 = default);
 * planes_per_chunk > 0 fixes how many planes one CTA marches through (0 = planner).  All
 * choices compute the same result; they differ in speed only.  Errors: ARG, UNSUPPORTED. */
CGEVAP_API int cgevap_tune(cgevap_sim* sim, int family, int variant, int planes_per_chunk);
/* The current choice of cgevap_tune (any output pointer may be NULL). */
CGEVAP_API int cgevap_get_tuning(const cgevap_sim* sim, int* family, int* variant,
                                 int* planes_per_chunk);

/* Bytes the algorithm must move per lattice update of this handle's fused step (populations
 * read and written, site byte read and/or written, flux field read); the numerator of the HBM
 * roofline fraction. */
CGEVAP_API double cgevap_bytes_per_update(const cgevap_sim* sim);

/* Number of fluid cells. */
CGEVAP_API long long cgevap_fluid_cells(const cgevap_sim* sim);

/* ---- adjoint: derivative of a volume-history loss with respect to the flux field -------------
 * Observable: V(t), t = 0..T, the liquid volume (cgevap_volume) after t steps.  The caller forms
 * a loss L(V(0), ..., V(T)); given dL/dV(t), the backward sweep returns dL/dphi(x) for every cell:
 * the exact derivative of the T fused steps (Eq. Stream with bounce-back, Eq. exchange, moments,
 * Eq. cg, Eq. feq, Eq. collision, Eq. perturb, Eq. recolor) with the site sets x_I of all steps
 * held at those of the forward run.  x_I is piecewise constant in phi, so this is the derivative
 * of L wherever no decision value of the run sits exactly on the threshold (and the derivative
 * of the run repeated with its sites replayed, CGEVAP_SITES_GIVEN, everywhere).  Storage F64 or
 * F32 with the register-pipelined step (cgevap_tune family 0); arithmetic in the storage's
 * precision, dL/dphi accumulated in FP64.  The flux may be a scalar or a field (cgevap_set_flux):
 * the scalar derivative is the sum of dL/dphi over cells. */

/* Run T = nsteps steps from the current state exactly as cgevap_step does (state, site bytes and
 * ledger advance) and record what the backward sweep needs: the state and site bytes at every
 * step that is a multiple of K = min(ckpt_every, T).  Device memory held until
 * cgevap_adjoint_release, cgevap_destroy or a forward run of another (T, K):
 * (ceil(T/K) + K + 2) states of the handle's state size plus (ceil(T/K) + K) site arrays and
 * 7 per-cell reals; T/K near sqrt(T) minimises it.  dev_volume: caller-owned FP64 [T + 1],
 * receives V(0), ..., V(T) (NULL: not recorded).  Errors: ARG (nsteps < 1 or ckpt_every < 1),
 * UNSUPPORTED (16-bit storage, or the TMA step selected), OOM (tape), CUDA. */
CGEVAP_API int cgevap_adjoint_forward(cgevap_sim* sim, int nsteps, int ckpt_every,
                                      double* dev_volume);

/* Reverse sweep over the recorded run.  Each segment of K steps is recomputed from its checkpoint
 * with the forward run's step kernel (the handle's own state, site bytes and ledger stay as the
 * forward run left them); the adjoint steps then run from step T-1 down to 0.
 *   dev_dL_dV    caller-owned FP64 [T + 1], dL/dV(t) (entry 0 is not read: V(0) does not depend
 *                on phi); NULL means 0;
 *   dev_dL_dphi  caller-owned FP64 [z][y][x], overwritten with dL/dphi(x): 0 at solid cells and
 *                at cells that were never a site.
 * May be called again for another dL/dV over the same recorded run.  The first sweep over a
 * new tape is the first to write its K recomputed states; on device memory not written before
 * those first writes are slow (about 16 GB/s measured on GB300), so a fit loop's first iteration
 * takes longer than the next ones.  Errors: ARG (no recorded run, NULL dev_dL_dphi, the step's
 * tuning changed since the forward run), CUDA. */
CGEVAP_API int cgevap_adjoint_backward(cgevap_sim* sim, const double* dev_dL_dV,
                                       double* dev_dL_dphi);

/* cgevap_adjoint_forward (without the volume record) then cgevap_adjoint_backward, for a loss
 * whose dL/dV(t) is known before the run (a loss linear in the volume history). */
CGEVAP_API int cgevap_adjoint_run(cgevap_sim* sim, int nsteps, int ckpt_every,
                                  const double* dev_dL_dV, double* dev_dL_dphi);

/* Free the recorded run (synchronises the stream; no-op without one).  Errors: ARG. */
CGEVAP_API int cgevap_adjoint_release(cgevap_sim* sim);

/* ---- ensembles: many independent lattices in one persistent launch ---------------------------
 * An ensemble advances n independent members (D2Q9 and D3Q19 lattices of any sizes, each with its
 * own densities, relaxation times, surface tension, recoloring, site rule, threshold, S-bar,
 * flux and solids; FP32 or FP64 storage, mixed freely, or F32X throughout) by one cooperative
 * persistent kernel
 * launch per call, captured
 * once in a CUDA graph and replayed.  Each member is a full cgevap_sim reachable with
 * cgevap_ensemble_member: set its flux, solids and initial state, read its macros, mask and
 * ledger with the single-lattice calls; cgevap_ensemble_step advances all of them together and
 * gives the same result per member as cgevap_step on that member alone. */
typedef struct cgevap_ens cgevap_ens;

/* Create members[0..n-1] (each validated like cgevap_create; storage must be CGEVAP_F32 or
 * CGEVAP_F64, mixed freely, or CGEVAP_F32X for every member; else UNSUPPORTED) and plan the work
 * list with a default tiling.  An ensemble whose members are all FP32 (or all F32X) runs four
 * CTAs per SM; one with FP64 members runs two (the FP64 step needs more registers).  *out is NULL
 * on failure. */
CGEVAP_API int cgevap_ensemble_create(const cgevap_params* members, int n, cgevap_ens** out);
/* Free the ensemble and all its members.  NULL is accepted. */
CGEVAP_API int cgevap_ensemble_destroy(cgevap_ens* ens);
/* Message for the last failure on ens; never NULL. */
CGEVAP_API const char* cgevap_ensemble_last_error(const cgevap_ens* ens);
/* Number of members / total cells of the active (not paused) members. */
CGEVAP_API int cgevap_ensemble_size(const cgevap_ens* ens);
CGEVAP_API long long cgevap_ensemble_cells(const cgevap_ens* ens);
/* Pause (active = 0) or resume (1) member j: a paused member takes no part in the following
 * cgevap_ensemble_step calls -- its state, site bytes and ledger stay as they are -- so a sweep
 * whose members reach their end at different times stops spending the launch on the finished
 * ones.  The work list is re-planned (the cached graph is rebuilt on the next step).  Errors: ARG
 * (j out of range, active not 0/1, or pausing the last active member). */
CGEVAP_API int cgevap_ensemble_set_active(cgevap_ens* ens, int j, int active);
/* Handle of member j (owned by the ensemble; do not destroy it or change its stream).  Members
 * take a scalar flux or a flux field; cgevap_ensemble_step fails with UNSUPPORTED while a member
 * has outlets (cgevap_set_outlets) or a heated flux (cgevap_set_flux_heated) set. */
CGEVAP_API int cgevap_ensemble_member(cgevap_ens* ens, int j, cgevap_sim** out);
/* Stream for the ensemble and all its members (NULL = legacy default stream). */
CGEVAP_API int cgevap_ensemble_set_stream(cgevap_ens* ens, void* cuda_stream);
/* Advance every member by nsteps >= 0 in one cooperative launch (graph-captured per nsteps and
 * replayed).  Asynchronous; cgevap_ensemble_status reports a grid barrier that gave up. */
CGEVAP_API int cgevap_ensemble_step(cgevap_ens* ens, int nsteps);
/* CGEVAP_ERR_TIMEOUT if a bounded grid barrier gave up since the last call (flag cleared), else
 * OK; synchronises the stream.  After a barrier gave up, the members' states are those of
 * whatever steps their items completed: re-initialise or reload them before trusting them; the
 * next launch starts with a clean barrier. */
CGEVAP_API int cgevap_ensemble_status(cgevap_ens* ens);
/* Limit of one grid-barrier wait of the persistent launch, in milliseconds (default 4000, >= 1).
 * A wait that reaches it sets the status that cgevap_ensemble_status reports and every CTA
 * leaves the launch at its next barrier.  Errors: ARG. */
CGEVAP_API int cgevap_ensemble_set_barrier_timeout(cgevap_ens* ens, int ms);
/* Test hook for the timeout path: in the following launches CTA `cta` (0 <= cta <
 * cgevap_ensemble_grid) does not arrive at the grid barrier after step `step` of the launch, so
 * the other CTAs wait until the barrier limit and the launch ends with CGEVAP_ERR_TIMEOUT; no
 * memory is touched out of turn and every wait stays bounded.  cta = -1 turns it off.
 * Errors: ARG. */
CGEVAP_API int cgevap_ensemble_debug_skip_arrival(cgevap_ens* ens, int cta, int step);
/* CTAs of the persistent launch of the current plan. */
CGEVAP_API int cgevap_ensemble_grid(const cgevap_ens* ens);
/* Tiling of the work list: D2Q9 tiles per CTA (2 or 4, i.e. rows of 128 or 64 cells) and planes
 * per chunk for D3Q19 and D2Q9 members. */
CGEVAP_API int cgevap_ensemble_set_tuning(cgevap_ens* ens, int groups, int planes_3d, int planes_2d);
CGEVAP_API int cgevap_ensemble_get_tuning(const cgevap_ens* ens, int* groups, int* planes_3d,
                                          int* planes_2d);
/* Autotuner: times probe_steps steps of every candidate tiling (groups 4 / 2, D3Q19 chunks of
 * 16-128 planes, D2Q9 chunks of 4-64 rows; only the values that matter for the active members)
 * on the ensemble as it is (its states, site bytes and ledgers are backed up first and restored
 * after), keeps the fastest and writes its time per step to *best_ms (may be NULL).  Needs room
 * for one copy of the states.  Pausing members changes the work: tune again after it. */
CGEVAP_API int cgevap_ensemble_autotune(cgevap_ens* ens, int probe_steps, double* best_ms);

/* ---- one timestep without any allocation -------------------------------------------------
 * No counterpart in the paper; it serves callers that cannot allocate device memory: code running
 * inside a framework that owns every buffer and forbids allocation in its operators (a custom
 * call of an XLA/JAX program, an application arena with a fixed budget), which therefore cannot
 * use cgevap_create.  It advances the state by one step of the same fused kernel as cgevap_step
 * and calls no cudaMalloc, cudaFree or allocating library routine.  The per-block scratch of the
 * FP64 ledger fold lives in a static device array of 256 KiB + 256 B, which every GPU that loads
 * the library holds until the process exits; it fits grids of at most 16384 CTAs (for example
 * 192^3 D3Q19 needs 288 for FP32).
 *   p              lattice and physics, validated like cgevap_create (no solids, no flux field;
 *                  storage CGEVAP_F64, F32, F16DEV or BF16DEV, else ARG);
 *   phi            scalar flux; each site moves phi / S-bar from red to blue rest populations;
 *   dev_state_in   caller-owned state in the handle's internal layout (the raw state bytes of a
 *                  cgevap_save checkpoint).  Populations are stored per direction i on a padded
 *                  grid: pitch P = round_up(nx + 18, 16) elements per row, R = ny + 4 rows per
 *                  plane (D3Q19; R = 1 for D2Q9), nz planes (ny for D2Q9), so one direction
 *                  holds E = planes * R * P elements and cell (x, y, z) sits at element
 *                  (z * R + y + 2) * P + x + 16 (D2Q9: y * P + x + 16); padding and ghost
 *                  elements are neither read nor written by this entry point.  Storage F64/F32: Q arrays of E pairs
 *                  (f_i^r, f_i^b) as double2/float2; F16DEV/BF16DEV: E float2 rest pairs, then
 *                  at byte offset round_up(8 E, 256) Q - 1 arrays of E half2/bfloat162 pairs;
 *   dev_state_out  caller-owned buffer of the same size for the new state (not aliasing _in);
 *   state_bytes    size of each state buffer; must equal that layout's size exactly
 *                  (F64: 16 Q E, F32: 8 Q E, 16-bit: round_up(8 E, 256) + 4 (Q - 1) E bytes);
 *   dev_mask_in    site bytes of the previous step (bits as in cgevap_get_mask), [N];
 *   dev_mask_out   site bytes written for this step, [N];
 *   dev_ledger     device cgevap_ledger updated in place (cumulative fields add up);
 *   cuda_stream    stream to run on (NULL = legacy default stream).
 * Returns ARG for invalid parameters, NULL or aliasing buffers, a wrong state_bytes, or a lattice
 * whose grid exceeds 16384 CTAs; CUDA on a failed runtime call; otherwise OK (asynchronous).
 * A failure's message is cgevap_last_error(NULL) (same thread).
 * The first call on each device resolves the scratch's device address (cudaGetSymbolAddress with
 * that device current); make that first call before any stream capture.  The address is resolved
 * again when the device's current context has changed since (after cudaDeviceReset, for example;
 * the scratch's contents are then new).  Every call on a device
 * shares the scratch: calls that overlap on the GPU (different streams, concurrent threads) race
 * and must be serialised by the caller.  The arrival counter in the scratch is cleared on the
 * stream before each launch; the partial sums need no clearing. */
CGEVAP_API int cgevap_step_static_scratch(const cgevap_params* p, double phi,
                                          const void* dev_state_in, void* dev_state_out,
                                          size_t state_bytes, const uint8_t* dev_mask_in,
                                          uint8_t* dev_mask_out, cgevap_ledger* dev_ledger,
                                          void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CGEVAP_H */
