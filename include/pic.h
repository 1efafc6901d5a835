/*
 * pic.h -- C ABI of the GB300 gauge-conserving spectral PIC library (libgpic.so).
 *
 * The library advances the particle-in-cell method of Christlieb, Sands and White,
 * "A PIC method with a generalized-momentum formulation, Part III: a family of
 * gauge-conserving methods" (arXiv 2410.18414), on a 2-D doubly periodic grid with
 * two velocity components, one time step being Algorithm 1 of section 4.2:
 *
 *   x^{n+1} = x^n + v^n dt                                   (IAEM, section 4.1)
 *   J^{n+1} = sum_p q_p v^n_p S(x - x^{n+1}_p)                (section 2.2, section 4)
 *   rho^{n+1} from the semi-discrete continuity equation     (sections 3.1-3.3, Alg. 1)
 *   phi, A at the new level from the implicit wave solve of the chosen stepper
 *     (CDF-2 implicit: section 3.1; BDF-k: section 3.2; s-stage DIRK: section 3.3)
 *   grad phi~, A, grad A spectrally (section 4), gathered with the same shape S
 *   P^{n+1} = P^n + q(-grad phi~ + grad A . v*) dt, v* = 2 v^n - v^{n-1};
 *   v^{n+1} = c^2 (P - qA) / sqrt(c^2 |P - qA|^2 + (m c^2)^2)  (section 4.1)
 *
 * Conventions shared by every call:
 *   - All work runs on one CUDA device, enqueued on the stream given to pic_init
 *     (0 = the legacy default stream).  Calls that only enqueue work return before
 *     it finishes; calls that return data to the host synchronize that stream.
 *   - Pointers named "src"/"dst" may be host or device memory (unified addressing
 *     decides; pinned host memory is fastest).  The library never keeps them.
 *   - Device memory for the simulation state is owned by the handle and released
 *     by pic_destroy.  No call frees memory it did not allocate.
 *   - Every call returns a pic_status.  Argument errors are reported synchronously
 *     and leave the handle unchanged.  Errors found on the device (non-finite
 *     particle data, fixed-point overflow) are latched in a device word and
 *     reported by the next call that synchronizes (pic_sync, pic_residuals,
 *     pic_read_particles, pic_get_field).  No call aborts the process;
 *     pic_last_error gives a one-line description of the last failure.
 *   - Grid arrays are (nx, ny) row-major with y fastest: node (i, j) at
 *     (i*dx, j*dy) is element i*ny + j.
 */
#ifndef GPIC_PIC_H
#define GPIC_PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_handle pic_handle; /* opaque, owned by the library */

typedef enum {
    PIC_OK = 0,
    PIC_ERR_INVALID_ARG = 1, /* a size, pointer or parameter outside its range     */
    PIC_ERR_UNSUPPORTED = 2, /* a valid request the library does not implement     */
    PIC_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed        */
    PIC_ERR_NONFINITE = 4,   /* a particle momentum or velocity became inf/NaN     */
    PIC_ERR_OVERFLOW = 5,    /* the int64 fixed-point current would overflow       */
    PIC_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                      */
    PIC_ERR_STATE = 7        /* the call needs state that is not available yet     */
} pic_status;

/* Time stepper for the wave equations of phi and A (section 3). */
typedef enum {
    PIC_STEPPER_BDF = 0,  /* BDF-k, k = bdf_order in 1..6 (section 3.2)               */
    PIC_STEPPER_CDF2 = 1, /* implicit centred CDF-2, phi at half levels (section 3.1) */
    PIC_STEPPER_DIRK = 2, /* s-stage DIRK with the tableau in pic_config (section 3.3) */
    PIC_STEPPER_CDF2_SEMI = 3,    /* semi-implicit CDF-2 (section 3.1, second form): the
                                     Laplacian averaged over levels n+1 and n-1, sources
                                     rho^{n+1/2} and J^n */
    PIC_STEPPER_CDF2_EXPLICIT = 4 /* explicit CDF-2 (section 3.1, third form): Laplacian and
                                     sources at level n; stable while (c dt)^2 |k|^2 <= 4 for
                                     every resolved mode */
} pic_stepper;

typedef enum {
    PIC_FP64 = 0,        /* the plain path: everything in FP64                          */
    PIC_FP32_FIX64 = 1   /* FP32 particles and FFT, current summed in int64 fixed point */
} pic_precision;

/* Grid quantities readable with pic_get_field (all real nx*ny arrays, FP64). */
typedef enum {
    PIC_FIELD_JX = 0, PIC_FIELD_JY = 1,      /* J^{n+1} of the last step                  */
    PIC_FIELD_RHO = 2,                        /* newest rho (CDF: rho^{n+3/2})             */
    PIC_FIELD_PHI = 3,                        /* newest phi (CDF: phi^{n+3/2})             */
    PIC_FIELD_AX = 4, PIC_FIELD_AY = 5,      /* A^{n+1}                                   */
    PIC_FIELD_BZ = 6,                         /* dAy/dx - dAx/dy at n+1                    */
    PIC_FIELD_EX = 7, PIC_FIELD_EY = 8,      /* stepper's discrete E (needs diagnostics)  */
    PIC_FIELD_DPHIDX = 9, PIC_FIELD_DPHIDY = 10,  /* the eight fields the particles      */
    PIC_FIELD_GAX = 11, PIC_FIELD_GAY = 12,       /* gather: grad phi~, A, grad A        */
    PIC_FIELD_DAXDX = 13, PIC_FIELD_DAXDY = 14,
    PIC_FIELD_DAYDX = 15, PIC_FIELD_DAYDY = 16,
    /* 2D-3V only (vdim = 3), PIC_ERR_STATE otherwise: */
    PIC_FIELD_JZ = 17,                        /* J_z^{n+1}                                 */
    PIC_FIELD_AZ = 18,                        /* A_z^{n+1}                                 */
    PIC_FIELD_BX = 19, PIC_FIELD_BY = 20,    /* dAz/dy, -dAz/dx at n+1                    */
    PIC_FIELD_DAZDX = 21, PIC_FIELD_DAZDY = 22  /* the in-plane gradient the particles gather */
} pic_field;

typedef struct {
    int32_t nx, ny;          /* grid nodes per direction: even, 8..1024, of the form 2^a 3^b */
    int32_t spline_order;    /* B-spline degree p of the particle shape: 2, 3 or 4          */
    int32_t stepper;         /* pic_stepper                                                 */
    int32_t bdf_order;       /* k for PIC_STEPPER_BDF (1..6)                                */
    int32_t dirk_stages;     /* s for PIC_STEPPER_DIRK (1..4)                               */
    int32_t precision;       /* pic_precision                                               */
    int32_t sort_interval;   /* re-sort particles by tile every this many steps; 0 = never  */
    double lx, ly;           /* periodic domain [0,lx) x [0,ly)                             */
    double c, eps0;          /* speed of light and permittivity; mu0 = 1/(eps0 c^2)         */
    double dt;               /* time step                                                   */
    double q, m;             /* charge and mass of one physical particle                    */
    double weight;           /* macro-particle weight: deposits charge weight*q             */
    double dirk_a[16];       /* s x s Butcher matrix, row-major (lower triangular)          */
    double dirk_b[4];        /* Butcher weights                                             */
    double dirk_c[4];        /* Butcher nodes                                               */
    int32_t charge;          /* pic_charge: where rho^{n+1} comes from (0: continuity)      */
    int32_t vdim;            /* velocity components: 0 or 2 = 2D-2V; 3 = 2D-3V (adds P_z,
                                v_z, J_z and A_z; d/dz = 0, so P_z is constant and A_z
                                obeys its own wave equation with source mu0 J_z)           */
    int32_t nspecies;        /* 0: one species (q, m, weight above); 1..4: each particle
                                carries a species index into species_q/m/w (section 2.1
                                sums the densities over species; section 2.2 writes the
                                equations with each particle's own charge and mass)        */
    int32_t tile;            /* tile width T (cells) of the sorted form's tiles: 4, 8 or 16;
                                0 = from the mean particle density (about 4096 particles a
                                tile); only used with sort_interval > 0                    */
    int32_t reserved[4];     /* must be zero                                                */
    double species_q[4];     /* charge, mass and macro-particle weight of each species     */
    double species_m[4];
    double species_w[4];
} pic_config;

/* Source of the charge rho^{n+1} of each step. */
typedef enum {
    PIC_CHARGE_CONTINUITY = 0, /* the method: the stepper's continuity update from J^{n+1} */
    PIC_CHARGE_DEPOSIT = 1     /* the naive update section 5 compares against: rho mapped to
                                  the mesh from x^{n+1} with the particle shape, like J.
                                  Continuity and the gauge then hold only approximately.
                                  BDF-k and DIRK only (PIC_ERR_UNSUPPORTED for CDF-2, whose
                                  charge lives at half levels) */
} pic_charge;

/* Initial particle state: positions x^0 (wrapped into the domain by pic_init) and
 * velocities v^0 (|v^0| < c).  Arrays of n FP64 values, host or device.  vz (2D-3V) and
 * species (nspecies > 0: int32 indices in 0..nspecies-1; an index out of range is
 * reported as PIC_ERR_NONFINITE) are required when the config uses them, else ignored. */
typedef struct {
    const double *x, *y, *vx, *vy;
    int64_t n;
    const double *vz;
    const int32_t *species;
} pic_particles_in;

/* Diagnostics of the last step that ran with diagnostics enabled (all FP64).
 * *_rms are grid root-mean-square values (Parseval over all modes). */
typedef struct {
    double gauge_rms;      /* Lorenz-gauge residual eps_1 of the stepper (sections 3.1-3.3) */
    double gauss_rms;      /* div E - rho/eps0 with the stepper's E                         */
    double continuity_rms; /* semi-discrete continuity residual                             */
    double gauge_dt_rms;   /* DIRK only: residual of the time-differentiated gauge (eps_2)  */
    double rho_rms;        /* RMS of rho/eps0 (scale for gauss_rms)                         */
    double div_a_rms;      /* RMS of div A^{n+1} (scale for gauge_rms)                      */
    double w_e;            /* eps0/2 sum |E|^2 dx dy (2D-3V: with E_z = -dA_z/dt)          */
    double w_b;            /* 1/(2 mu0) sum |B|^2 dx dy (2D-2V: B_z only)                   */
    double kinetic;        /* sum_p weight m c^2 (gamma_p - 1), per species                 */
    int64_t step;          /* step index n+1 these values belong to                         */
} pic_diagnostics;

/* Create a simulation: validate cfg, copy the initial particles to the device and
 * build the t = 0 state (section 4.2, Algorithm 1 set-up): rho^0 by depositing the
 * charge with its K = 0 modes removed (neutralising background), phi^0 from
 * Poisson's equation, A^0 = 0, P^0 = gamma m v^0, v^{-1} by a first-order Taylor
 * step back in E^0 = -grad phi^0, and every history level at its t = 0 value.
 * On success *out receives the handle.  The stream must outlive the handle.
 * With sort_interval > 0 a species table (2D-2V, FP32 form) runs in the fused binned
 * kernel; 2D-3V runs, and FP64 runs, step their sorted particles with the general kernels.
 * PIC_ERR_INVALID_ARG for a field out of its stated range (tile not
 * 0, 4, 8 or 16; reserved fields not zero; ...).  A tile wider than half the grid is
 * narrowed to fit. */
pic_status pic_init(const pic_config *cfg, const pic_particles_in *init, void *cuda_stream,
                    pic_handle **out);

/* Caller-owned particle state (pic_init_bound): eight device arrays of n values each in
 * the storage type of cfg->precision (double for PIC_FP64, float for PIC_FP32_FIX64),
 * for example torch tensors.  On entry x, y, vx, vy hold x^0 and v^0; px, py, vx_old and
 * vy_old are written by the t = 0 set-up (P^0 and v^{-1}). */
typedef struct {
    void *x, *y, *px, *py, *vx, *vy, *vx_old, *vy_old;
    int64_t n;
} pic_particles_bound;

/* As pic_init, but the handle steps the caller's arrays in place: no copy in, no copy
 * out.  The library never frees them; they must stay allocated until pic_destroy.  Each
 * step writes v^{n+1} over the pair holding v^{n-1}, so the two velocity pairs exchange
 * roles every step: pic_velocity_slot says which pair holds v^n.  Only for unsorted
 * (sort_interval 0), 2D-2V, single-species configurations, else PIC_ERR_UNSUPPORTED;
 * PIC_ERR_INVALID_ARG for NULL arrays (n > 0) or arrays that are not device memory.
 * pic_read_particles, checkpoints, ensembles and the adjoint work as for pic_init. */
pic_status pic_init_bound(const pic_config *cfg, const pic_particles_bound *particles,
                          void *cuda_stream, pic_handle **out);

/* 0 when (vx, vy) of pic_init_bound hold v^n (and (vx_old, vy_old) v^{n-1}), 1 when the
 * roles are exchanged; the same index for handles of pic_init (internal buffers).  -1 for
 * NULL. */
int32_t pic_velocity_slot(const pic_handle *h);

/* Algorithm 1, the position update and deposit: move every particle with v^n
 * (wrapping into the domain) and deposit J^{n+1} with the new positions and v^n.
 * Re-sorts the particles first when sort_interval says so. */
pic_status pic_deposit(pic_handle *h);

/* Algorithm 1, the charge and field steps: FFT of J^{n+1}, rho^{n+1} from continuity,
 * the implicit per-mode wave update of phi and A, and the eight spectral gradient
 * fields on the grid.  Needs a preceding pic_deposit of the same step. */
pic_status pic_field_solve(pic_handle *h);

/* Algorithm 1, the particle update: gather the eight fields at x^{n+1}, IAEM momentum
 * update with v*, new velocity; then shift the time histories (end of the step). */
pic_status pic_gather_push(pic_handle *h);

/* nsteps complete steps (deposit, field solve, gather/push each). */
pic_status pic_step(pic_handle *h, int32_t nsteps);

/* ---- Ensembles: many independent runs in one CUDA-graph launch ----------------------
 *
 * Independent simulations (each its own pic_handle, of any grid size, particle count
 * and form) advance together: pic_ensemble_create captures P steps of every run into
 * one CUDA graph, each run on its own stream so that the runs overlap on the GPU, and
 * pic_ensemble_step replays that graph.  P is the common period of the runs' per-step
 * buffer rotations (history rings, velocity and current buffers, sort buffers: the
 * least common multiple of 2, the BDF ring lengths and twice each sort interval), so
 * every replay finds every buffer where the captured launches expect it.  The results
 * are those of pic_step on each run, bit for bit (both forms sum their deposits as
 * integers, so the order of the additions does not matter).
 *
 * Not a step of the paper: a batching of its step (no counterpart there). */
typedef struct pic_ensemble pic_ensemble; /* opaque, owned by the library */

/* Capture P steps of runs[0..count) into one graph launched on `stream` (a cudaStream_t;
 * not NULL, the legacy default stream cannot be captured).  Every run must be between
 * steps, with diagnostics and kernel timing off, and should have a stream of its own
 * (runs that share a stream are serialised).  Runs nothing on the GPU: the captured
 * steps execute only in pic_ensemble_step.  The runs' host-side state is unchanged on
 * return (on failure as well).  The ensemble keeps the run pointers: destroy it before
 * its runs.  Errors: PIC_ERR_INVALID_ARG (NULL or repeated runs, count < 1 or > 4096,
 * NULL stream), PIC_ERR_STATE (a run mid-step, with diagnostics or timing on),
 * PIC_ERR_CUDA (capture or instantiation failed); the text is in pic_last_error(NULL). */
pic_status pic_ensemble_create(pic_handle *const *runs, int32_t count, void *stream,
                               pic_ensemble **out);

/* Advance every run by nsteps, a multiple of the period (pic_ensemble_period), as
 * nsteps / P graph launches on the ensemble's stream.  The launches wait for work
 * already enqueued on the runs' streams, and later work on a run's stream waits for
 * them, so pic_step, pic_read_particles, pic_get_field... on a run see the result.  A
 * run advanced on its own (pic_step) by a number of steps that is not a multiple of P
 * no longer matches the graph: PIC_ERR_STATE.  Errors: PIC_ERR_INVALID_ARG (NULL,
 * nsteps < 0 or not a multiple of P), PIC_ERR_CUDA; text in pic_last_error(NULL).
 * Device-side errors latch in each run and are reported by pic_sync on that run. */
pic_status pic_ensemble_step(pic_ensemble *e, int32_t nsteps);

/* Steps captured in the graph (the period P), 0 for NULL. */
int32_t pic_ensemble_period(const pic_ensemble *e);

/* Release the graph and the ensemble's events (not the runs).  NULL is allowed. */
void pic_ensemble_destroy(pic_ensemble *e);

/* Compute diagnostics every `every` steps (0 = never, the default).  They cost one
 * extra reduction over modes and particles per diagnosed step, and a device copy of its
 * accumulators into the history ring (pic_diagnostics_history), which the first call
 * with every > 0 allocates (PIC_ERR_CUDA if that fails).  Each call starts a new history:
 * records not yet read are dropped. */
pic_status pic_set_diagnostics(pic_handle *h, int32_t every);

/* Copy the diagnostics of the last diagnosed step to *out (synchronizes).
 * PIC_ERR_STATE if no step has been diagnosed yet. */
pic_status pic_residuals(pic_handle *h, pic_diagnostics *out);

/* The diagnostics of every diagnosed step since the previous call (or since
 * pic_set_diagnostics), oldest first, into out[0..capacity) on the host; *count receives
 * how many were written.  Each diagnosed step's accumulators are copied on the device into
 * a ring of PIC_DIAG_HISTORY records as the step ends, so stepping needs no host
 * synchronisation; when more steps were diagnosed than the ring or capacity holds, the
 * oldest are dropped (the step fields tell).  Synchronizes.  PIC_ERR_INVALID_ARG for NULL
 * pointers or capacity < 0. */
#define PIC_DIAG_HISTORY 4096
pic_status pic_diagnostics_history(pic_handle *h, pic_diagnostics *out, int32_t capacity,
                                   int32_t *count);

/* Copy one real nx*ny grid quantity of the last step into dst (FP64, host or
 * device).  PIC_ERR_STATE for EX/EY unless the last step was diagnosed, and for
 * every field before the first step except RHO and PHI. Synchronizes. */
pic_status pic_get_field(pic_handle *h, int32_t which, double *dst);

/* Copy the particle state, in the order the particles were given to pic_init, into
 * FP64 arrays of n values (host or device).  Any pointer may be NULL to skip it.
 * x, y: x^n; px, py: P^n; vx, vy: v^n; vx_old, vy_old: v^{n-1}.  Synchronizes. */
pic_status pic_read_particles(pic_handle *h, double *x, double *y, double *px, double *py,
                              double *vx, double *vy, double *vx_old, double *vy_old);

/* 2D-3V and species state, as pic_read_particles: pz: P_z (constant), vz, vz_old: v_z^n and
 * v_z^{n-1}; species: each particle's species index (int32).  Any pointer may be NULL.
 * PIC_ERR_STATE when the handle has no such state (vdim 2 for the first three, no species
 * table for the last). */
pic_status pic_read_particles_z(pic_handle *h, double *pz, double *vz, double *vz_old,
                                int32_t *species);

/* Checkpoint and resume.  pic_save_state writes the handle's state between two steps into
 * host memory dst as one byte string: a header of the configuration and the rotation state
 * (step count, which velocity buffer holds v^n, the BDF ring heads) followed by every device
 * buffer a later step reads (particles, the sort's order and tile offsets, the field
 * histories, the last step's J and gather fields).  With dst NULL it only stores the size
 * needed in *size; with *size too small it returns PIC_ERR_INVALID_ARG and the size needed.
 * Synchronizes.  pic_load_state restores such a string into a handle created with the same
 * configuration and particle count (PIC_ERR_INVALID_ARG otherwise; the layout fields and
 * every FP64 parameter a step uses -- lx, ly, c, eps0, dt, q, m, weight, the DIRK tableau
 * and the species table -- are compared bit for bit): the handle then steps exactly as
 * the saved one would have (bit for bit in the FP32 form).  Diagnostics of the last step
 * are not part of the state, and the per-step diagnostics log restarts at the load
 * (pic_diagnostics_history returns no record of a step before it).  A handle that belongs
 * to an ensemble or an adjoint must not be loaded into.  Both: PIC_ERR_STATE inside a
 * step. */
pic_status pic_save_state(pic_handle *h, void *dst, size_t *size);
pic_status pic_load_state(pic_handle *h, const void *src, size_t size);

/* Wait for all work enqueued by this handle; report latched device errors. */
pic_status pic_sync(pic_handle *h);

/* Steps completed since pic_init. */
int64_t pic_step_count(const pic_handle *h);

/* Number of CUDA kernels one step launches (for launch accounting). */
int32_t pic_kernels_per_step(const pic_handle *h);

/* Kernel timing, a measurement aid.  The library brackets each launch group below with
 * a pair of CUDA events on the handle's stream and sums their elapsed times:
 *   PIC_KT_SORT     the particle sort (keys, scan, scatter) of a sorting step
 *   PIC_KT_DEPOSIT  the move + current deposit kernel (not the clearing of J)
 *   PIC_KT_FIELD    all kernels of pic_field_solve
 *   PIC_KT_GATHER   the gather + push kernel
 *   PIC_KT_GATHER_DEPOSIT  the fused kernel of the sorted FP32 form inside pic_step: the
 *                   gather + push of one step with the move + deposit of the next (a step
 *                   that ends with it has no PIC_KT_GATHER launch, the next no
 *                   PIC_KT_DEPOSIT launch)
 * and, in pic_adjoint_backward (one launch group per reversed step):
 *   PIC_KT_ADJ_PUSH     the reverse push + gather kernel (with its field-adjoint deposit)
 *   PIC_KT_ADJ_FIELD    the reverse field solve (transforms and per-mode update)
 *   PIC_KT_ADJ_DEPOSIT  the reverse deposit + move kernel */
typedef enum {
    PIC_KT_SORT = 0,
    PIC_KT_DEPOSIT = 1,
    PIC_KT_FIELD = 2,
    PIC_KT_GATHER = 3,
    PIC_KT_ADJ_PUSH = 4,
    PIC_KT_ADJ_FIELD = 5,
    PIC_KT_ADJ_DEPOSIT = 6,
    PIC_KT_GATHER_DEPOSIT = 7,
    PIC_KT_COUNT = 8
} pic_kernel_timer;

/* max_launches > 0 starts timing: resets every timer and creates max_launches event
 * pairs per timer up front (launches beyond that are not timed; a timer counts only
 * the launches it timed).  max_launches = 0 stops timing and keeps the sums.  Events are
 * created only here, never inside a step.  PIC_ERR_INVALID_ARG for max_launches < 0 or
 * above 2^20; PIC_ERR_CUDA if event creation fails. */
pic_status pic_set_kernel_timing(pic_handle *h, int32_t max_launches);

/* Sum of the timed durations (milliseconds) and the number of timed launches of timer
 * `which` since timing was last started.  Synchronizes the handle's stream.
 * PIC_ERR_INVALID_ARG for an unknown timer or NULL outputs. */
pic_status pic_kernel_time(pic_handle *h, int32_t which, double *total_ms, int64_t *launches);

/* Measurement aid (the paper has no counterpart): the FP64 fused multiply-add rate of the
 * current device in GFLOP/s (an FMA counts two flops), timed with CUDA events on `stream`
 * over a kernel of independent FMA chains filling every SM (best of three runs after a
 * warm-up).  The FP64 path's particle kernels are bound by that rate.  Allocates and frees
 * 8 bytes of device memory; synchronizes the stream.  PIC_ERR_INVALID_ARG for a NULL
 * output, PIC_ERR_CUDA on a runtime failure. */
pic_status pic_measure_fp64_fma(void *stream, double *gflops);

/* One-line description of the last failure on this handle (or of the last failed
 * pic_init when h is NULL).  Valid until the next call on the handle. */
const char *pic_last_error(const pic_handle *h);

/* Release every device allocation of the handle.  NULL is allowed. */
void pic_destroy(pic_handle *h);

/* ---------------------------------------------------------------- adjoint ----
 * Discrete adjoint of the step: the exact gradient of an objective of the final state,
 *     J = sum_ij bz_bar(i, j) B_z(i, j) + sum_p (px_bar_p Px_p + py_bar_p Py_p),
 * B_z = dAy/dx - dAx/dy of the last level and P the last momenta, with respect to the
 * initial velocities v^0 given to pic_init (and, with P^0 = gamma m v^0 taken as the
 * independent variable, with respect to P^0).  For the magnetic energy
 * W_B = 1/2 sum B_z^2 dx dy (section 5) pass bz_bar = B_z dx dy.  The gradient is the
 * transpose of the Jacobian of the forward map that pic_step computes (Algorithm 1 of
 * section 4.2 with any of the field updates -- BDF-k of section 3.2, the three CDF-2 forms of
 * section 3.1, DIRK of section 3.3 -- and the charge from continuity),
 * applied step by step in reverse:
 *   - the transpose of the current deposit is a gather of the current's adjoint with
 *     the shape weights and their derivatives;
 *   - the transpose of the field gather is a deposit of the eight field adjoints;
 *   - per Fourier mode, the stepper's recurrences run backwards with their real
 *     multipliers (DIRK's from its stage recurrence on unit inputs), and i k maps to -i k;
 *   - the IAEM push and the t = 0 set-up (P^0 = gamma m v^0 and the Taylor start
 *     v^{-1}) are transposed per particle.
 * The paper states the forward method only; the adjoint is a derived capability.
 *
 * Precision: for an FP64 handle every step of the reverse sweep is FP64.  For an FP32-form
 * handle (PIC_FP32_FIX64, unsorted) the adjoint is that of the step in exact arithmetic
 * evaluated along the FP32 form's own trajectory: the particle adjoints are FP32 and run
 * through the FP32 weights and push (the fixed-point rounding of the current, piecewise
 * constant, is taken as the identity), and the field adjoints the particles deposit are
 * summed in FP32, while the reverse field solve is FP64 with its own FP64 transforms.  The records and checkpointed particle states are then FP32 (32 n bytes a
 * state, 32 nx ny bytes of gather fields a step); seeds and results stay FP64.
 *
 * Memory: the state (particles and field histories) is checkpointed every
 * `checkpoint_every` steps (K).  The backward pass rebuilds each segment of K steps from
 * its checkpoint -- the particle states (S = 64 n bytes per step of the segment in FP64,
 * 32 n in the FP32 form) and each step's record (see pic_adjoint_mode) -- then runs it
 * backwards.  With G = 64 nx ny bytes of gather fields a step (32 nx ny in the FP32 form):
 * PIC_ADJ_REPLAY (the default) keeps every step's record from the forward pass and replays
 * only the particle move, costing about (nsteps/K + 1 + K) S + nsteps (80 n + G) bytes
 * (PIC_ADJ_REPLAY_LEAN: 32 n in place of 80 n); PIC_ADJ_RECOMPUTE re-runs the segment's
 * full steps, costing about (nsteps/K + 1) S + K (80 n + S + G) bytes.  All hold the
 * adjoint state besides. */
typedef struct pic_adjoint pic_adjoint; /* opaque, owned by the library */

/* What the forward pass keeps between checkpoints. */
typedef enum {
    PIC_ADJ_REPLAY = 0,    /* every step's record: its gather fields, and per particle
                              P^{n+1}, v^{n+1} and the A, grad A its push gathered (80 n + G
                              bytes per step); the backward pass replays the particle
                              states of a segment from its checkpoint with the move alone and
                              the recorded P, v (bit for bit the forward's states) */
    PIC_ADJ_RECOMPUTE = 1, /* nothing: the backward pass re-runs every segment's full forward
                              steps from its checkpoint (least memory) */
    PIC_ADJ_REPLAY_LEAN = 2 /* as PIC_ADJ_REPLAY with per particle only P^{n+1}, v^{n+1}
                              (32 n + G bytes per step): the reverse push gathers A and
                              grad A again from the recorded fields (the same bits, a second
                              pass over the stencil) */
} pic_adjoint_mode;

/* Prepare the adjoint of the next `nsteps` steps of h.  h must be fresh from pic_init
 * (step 0, no step started), of either precision (any stepper), PIC_CHARGE_CONTINUITY and
 * without sorting (sort_interval 0), 2D-2V with one species, else PIC_ERR_UNSUPPORTED (or
 * PIC_ERR_STATE for a handle that has stepped).  checkpoint_every is clamped to 1..nsteps.  Allocates all the
 * adjoint's device memory here (PIC_ERR_CUDA if that fails).  The adjoint keeps h:
 * destroy it before h.  PIC_ERR_INVALID_ARG for NULL pointers or nsteps < 1. */
pic_status pic_adjoint_create(pic_handle *h, int32_t nsteps, int32_t checkpoint_every,
                              pic_adjoint **out);

/* As pic_adjoint_create (which uses PIC_ADJ_REPLAY) with the record mode given:
 * PIC_ERR_INVALID_ARG for an unknown mode. */
pic_status pic_adjoint_create_ex(pic_handle *h, int32_t nsteps, int32_t checkpoint_every,
                                 int32_t mode, pic_adjoint **out);

/* Run the nsteps forward steps on h (as pic_step), keeping the checkpoints.  Once only;
 * PIC_ERR_STATE on a second call. */
pic_status pic_adjoint_forward(pic_adjoint *a);

/* Gradient of J (defined above) after pic_adjoint_forward.  Inputs (device memory, FP64,
 * any may be NULL for a zero term): bz_bar nx*ny (grid layout), px_bar, py_bar n each
 * (the order of pic_init).  Outputs (device memory, FP64, n each, any may be NULL):
 * dJ/dvx^0, dJ/dvy^0, and dJ/dPx^0, dJ/dPy^0 with P^0 independent.  May be called again
 * with other seeds.  h is left with the state of the end of the forward run (particles,
 * histories, J and gather fields of the last step).  Enqueued on h's stream;
 * synchronizes at the end and reports latched device errors.  PIC_ERR_STATE before
 * pic_adjoint_forward. */
pic_status pic_adjoint_backward(pic_adjoint *a, const double *bz_bar, const double *px_bar,
                                const double *py_bar, double *dvx0, double *dvy0,
                                double *dpx0, double *dpy0);

/* Steps between checkpoints after clamping (0 for NULL). */
int32_t pic_adjoint_checkpoint_every(const pic_adjoint *a);

/* Release the adjoint's device memory (not the handle).  NULL is allowed. */
void pic_adjoint_destroy(pic_adjoint *a);

/* Allocation-free move + deposit pass (the position update and deposit of one step, as
 * pic_deposit does them) for callers that cannot let a library allocate device memory:
 * hosts whose GPU memory is owned by their own pool allocator (a hidden cudaMalloc would
 * fail or bypass the pool), and latency-bound loops that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree imply.  The paper has no counterpart; this is a
 * deployment convenience.
 *
 *   cfg     only nx, ny (nx*ny <= 262144, i.e. up to a 512 x 512 grid; each >= 8), lx, ly,
 *           dt, c, spline_order, q, weight and precision (must be PIC_FP64) are used.
 *   x, y    device arrays of n FP64 positions in [0, L), moved in place by v dt and wrapped.
 *   vx, vy  device arrays of n FP64 velocities v^n.
 *   jx, jy  device outputs, nx*ny FP64 each (layout as every grid here): J^{n+1} as a
 *           current density, weight*q*sum_p v_p W W / (dx dy).
 *
 * The only scratch is a fixed 4 MiB array inside the library, resident on every device
 * that loads it until the process exits.  The calls themselves never call cudaMalloc or
 * cudaFree, but the 4 MiB is committed when the CUDA module holding the array is loaded
 * on a device: under CUDA's default lazy module loading that is the first call on that
 * device (which also looks up the array's device address once), outside any pool the
 * caller manages.  A caller whose pool takes the whole GPU should therefore make one call
 * (or load the library with CUDA_MODULE_LOADING=EAGER) before its pool claims the device;
 * otherwise that first call can fail with PIC_ERR_CUDA.  Every call shares the array and
 * clears what it uses; calls that overlap on the GPU (other threads or streams) race on
 * it.  The call enqueues on cuda_stream, reads the device error flag back and
 * synchronizes that stream, so it returns once the pass has finished and cannot be
 * captured into a CUDA graph.  Returns PIC_ERR_INVALID_ARG for a grid above the limit or
 * a bad argument, PIC_ERR_UNSUPPORTED for FP32, PIC_ERR_NONFINITE if a position was
 * outside the domain or not finite (that particle is skipped), PIC_ERR_CUDA on a runtime
 * failure. */
pic_status pic_move_deposit_noalloc(const pic_config *cfg, int64_t n, double *x, double *y,
                                    const double *vx, const double *vy, double *jx, double *jy,
                                    void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GPIC_PIC_H */
