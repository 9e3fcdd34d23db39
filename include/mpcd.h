/*
 * mpcd.h -- C ABI of libmpcd, a GB300 (sm_103a) implementation of the stochastic rotation
 * dynamics (SRD) time step of multi-particle collision dynamics (MPCD).
 *
 * The method (arXiv 2212.11878, Sec. 2): every step the particles stream ballistically, the
 * collision grid is shifted at random, the particles are sorted into the shifted cells
 * (Sec. 3.1, Listing 1), each cell's mass and momentum are summed (Sec. 3.3, Listing 4), and
 * each particle's velocity relative to its cell's centre-of-mass velocity is split along a
 * random axis and its perpendicular part rotated by a fixed angle alpha (Sec. 2, parts
 * (i)-(iii)).  A system is a box of L[0] x L[1] x L[2] cubic cells of edge a holding
 * N = round(ppc * cells) particles of mass m (Sec. 4: N = L^3 <N_c>).
 *
 * Conventions shared by every entry point
 *   - Return value: MPCD_OK (0) or a negative MPCD_ERR_* code.  A failed call leaves a
 *     message readable with mpcd_last_error().  After a CUDA error the handle is poisoned:
 *     every later call except mpcd_last_error / mpcd_destroy returns MPCD_ERR_STATE.
 *   - Ownership: a handle owns all of its device memory; the caller owns every array it
 *     passes in.  Host arrays are plain (pageable or pinned) host memory; "_device" entry
 *     points take device pointers on the handle's GPU.
 *   - Layout: positions and velocities cross the ABI as FP64 arrays of N x 3, row-major
 *     (x, y, z of particle 0, then particle 1, ...), always in particle-id order.
 *   - Asynchrony: mpcd_step only enqueues work on the handle's stream; calls that return
 *     data to the host synchronise that stream first.
 *   - Threads: a handle is used by one host thread at a time.
 */
#ifndef MPCD_H
#define MPCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpcd_s mpcd_t; /* opaque, library-owned */

enum {
  MPCD_OK = 0,
  MPCD_ERR_ARG = -1,     /* invalid argument; nothing was changed */
  MPCD_ERR_CUDA = -2,    /* a CUDA call failed; the handle is now poisoned */
  MPCD_ERR_OOM = -3,     /* device memory ran out (create, or the first call that needs a */
                         /* buffer: host get/set_state, set_masses, record_moments); the    */
                         /* handle is not poisoned and nothing was changed                  */
  MPCD_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up: a grid-wide barrier of the  */
                         /* mixed form's one-launch step waited about a second; the step is */
                         /* incomplete and the handle is poisoned (reported by mpcd_sync and */
                         /* mpcd_get_state)                                                  */
  MPCD_ERR_STATE = -5    /* the handle was poisoned by an earlier error */
};

enum { MPCD_FP64 = 0, MPCD_MIXED = 1 };

/* Parameters of one box.  Readings of points the paper leaves open are noted per field. */
typedef struct {
  int32_t L[3];       /* cells per side (>= 1); box edge L[d] * a                          */
  int32_t precision;  /* MPCD_FP64: FP64 positions and velocities (the paper's `double`,   */
                      /*   Listing 1); MPCD_MIXED: int32 cell + FP32 in-cell offset         */
                      /*   positions, FP32 velocities, FP64 per-cell sums                   */
  double a;           /* cell edge length (> 0)                                             */
  double ppc;         /* mean particles per cell; N = round(ppc * L0 L1 L2)                 */
  double dt;          /* streaming time step (>= 0)                                         */
  double alpha;       /* rotation angle in radians, applied with the right-hand rule        */
  double kT;          /* temperature of the initial Maxwell-Boltzmann velocities (> 0)      */
  double mass;        /* particle mass m (> 0), the same for all particles                  */
  double g[3];        /* constant body-force acceleration (g[2] must be 0 with walls)       */
  uint64_t seed;      /* Philox4x64-10 key word 0 for every random draw of this box         */
  int32_t walls_z;    /* 0: periodic in z; 1: bounce-back walls at z = 0 and z = L[2] a,    */
                      /*   virtual particles in cut cells (Lz + 1 cell layers)               */
  int32_t thermostat; /* 0: none; after each collision, rescale each cell's relative kinetic */
                      /*   energy (n >= 2 real particles) to 1: 3/2 (n-1) kT, or 2: kT G    */
                      /*   with G ~ Gamma(3/2 (n-1)) drawn per (step, cell) (Maxwell-       */
                      /*   Boltzmann scaling, Huang et al. 2010; Philox counter             */
                      /*   (t, cell, 3, attempt), Marsaglia-Tsang).  Other values: ERR_ARG  */
  int32_t resort_k;   /* physically re-order storage by cell every k steps (0: never)       */
  int32_t angular;    /* 1: angular-momentum-conserving collision (the variant Sec. 2       */
                      /*   mentions): after the rotation (and thermostat) each member gets  */
                      /*   omega x rho_i, rho_i its position from the cell's centre of mass */
                      /*   on the shifted grid, omega = I^-1 (L_before - L_after), I the    */
                      /*   cell's inertia tensor (pseudo-inverse for two particles; none    */
                      /*   for a singular one).  Conserves each cell's momentum and angular */
                      /*   momentum, not its energy.  Periodic boxes only (walls: ERR_ARG). */
                      /*   The mixed form takes it through its per-cell kernel.  0: off.    */
} mpcd_params;

/* Create a box and initialise it on the current CUDA device (Sec. 4 workload): positions
 * uniform in the box, velocities N(0, kT/m) per component with the net momentum removed,
 * drawn from Philox counters (i, 0, 0, 0) and (i, 1, 0, 0).  The FP64 form then stores the
 * particles in cell order (see mpcd_set_state).  *out receives the handle, or NULL on
 * failure.  Errors: MPCD_ERR_ARG for invalid params, MPCD_ERR_OOM, MPCD_ERR_CUDA. */
int mpcd_create(const mpcd_params* p, mpcd_t** out);

/* Create an ensemble of nbox independent boxes (each with its own L, ppc, dt, alpha, g,
 * seed) advanced together: one counting sort over the concatenated cell keys and one
 * launch sequence per step (replayed from a CUDA graph).  Boxes use the mixed form
 * (precision MPCD_MIXED) and must share walls_z and thermostat.  Particle and cell data of
 * box b follow those of boxes 0..b-1 (mpcd_box_offsets).  Each box draws its random
 * numbers from its own seed and is advanced exactly as if it were created alone. */
int mpcd_batch_create(int32_t nbox, const mpcd_params* p, mpcd_t** out);

/* First particle and first cell of every box: particle_base[nbox + 1], cell_base[nbox + 1]
 * (either may be NULL).  Particle ids of box b are particle_base[b] .. particle_base[b+1]-1. */
int mpcd_box_offsets(const mpcd_t* h, int64_t* particle_base, int64_t* cell_base);

/* Free every device buffer of the handle.  NULL is accepted. */
int mpcd_destroy(mpcd_t* h);

/* Run all later work on `stream` (a cudaStream_t of the handle's device, e.g. a PyTorch
 * stream); NULL selects the handle's own stream.  Synchronises the previous stream. */
int mpcd_set_stream(mpcd_t* h, void* stream);

/* Enqueue nsteps full SRD steps (Sec. 2): stream, shift, bin, per-cell sums, rotate.
 * Steps are numbered from 1 since creation or the last mpcd_set_state.  Asynchronous. */
int mpcd_step(mpcd_t* h, int64_t nsteps);

/* Wait for all enqueued work (MPCD_ERR_CUDA if a kernel failed). */
int mpcd_sync(mpcd_t* h);

int64_t mpcd_num_particles(const mpcd_t* h); /* N, or -1 for NULL */
int64_t mpcd_num_cells(const mpcd_t* h);     /* collision cells (with walls Lx Ly (Lz+1)) */
int64_t mpcd_steps_done(const mpcd_t* h);    /* steps enqueued since the state was set    */
int32_t mpcd_num_boxes(const mpcd_t* h);     /* 1 for mpcd_create                          */

/* Copy the state to host arrays r[N*3], v[N*3] (FP64, particle-id order).  Mixed-precision
 * positions are returned as (cell index + offset) * a.  Synchronises.  The FP64 form (from
 * 65,536 particles) gathers the state by particle id in eight chunks and copies each chunk to
 * the host on a second stream while the next one is gathered.  The first host
 * get/set_state call allocates a device staging buffer of 6 N doubles, kept until
 * mpcd_destroy; if that allocation fails the call returns MPCD_ERR_OOM, changes nothing and
 * leaves the handle usable. */
int mpcd_get_state(mpcd_t* h, double* r, double* v);

/* Replace the state from host arrays r[n*3], v[n*3] (particle-id order) and set the step
 * counter to t (the next step is t + 1).  n must equal mpcd_num_particles.  Positions must
 * lie in their box ([0, L a) per axis) and velocities be finite; otherwise MPCD_ERR_ARG
 * (the message names the first offending particle) and the state is unchanged.  The check
 * runs on the device.  Storage order afterwards (FP64 form): the particles are stored in
 * cell order of the unshifted grid (cell key of floor(r / a), stable in particle id), the
 * Listing 1 `permute` applied once, so that the first steps already find each cell's members
 * in neighbouring slots; the mixed form keeps id order until its first step.  Storage order
 * is visible only through mpcd_debug_sort.  FP64 form with 65,536 particles or more: the
 * positions are uploaded first, and their check, the cell-order sort and their gather run on
 * a second stream while the velocities are still being copied, into the buffer set that does
 * not hold the current state; a rejected state then still leaves the particles unchanged, but
 * the last step's sort record is gone (mpcd_debug_sort returns MPCD_ERR_STATE until the next
 * step).  Synchronises. */
int mpcd_set_state(mpcd_t* h, int64_t n, const double* r, const double* v, int64_t t);

/* Per-particle masses (the m of the cell sums sum m v and sum m, Sec. 3.3 Listing 4):
 * m[n] in particle-id order, every value finite and > 0, n = mpcd_num_particles.  The mixed
 * form keeps them in FP32 (each value rounded once; mpcd_get_masses returns the rounded
 * values), sums the FP32 products m v exactly, and takes every cell through its per-cell
 * path; with angular-momentum conservation it rejects masses (MPCD_ERR_ARG).
 * They weight the centre-of-mass velocity, the moments, the thermostat's kinetic energy and
 * the angular-momentum correction (whose centre becomes mass-weighted); the rotation of
 * v - u keeps sum m v and sum m v^2 / 2.  Virtual wall particles and the initial velocities
 * keep params.mass.  Masses follow their particles through re-sorts and mpcd_set_state.
 * m = NULL restores the box mass.
 * Errors: MPCD_ERR_ARG (n != N; a mass not finite or <= 0, named in the message; the mixed
 * form with angular-momentum conservation).  Synchronises. */
int mpcd_set_masses(mpcd_t* h, int64_t n, const double* m);
/* The masses in particle-id order (params.mass everywhere when none were set). */
int mpcd_get_masses(mpcd_t* h, double* m);

/* Coupling hook: an external momentum source acting on the fluid between steps, the way an
 * embedded solute (for instance a molecular-dynamics body, the coupling the paper names as
 * future work in Sec. 5) exchanges momentum with the solvent.  Adds dp_i / m_i to the
 * velocity of every particle i, with dp[n * 3] in particle-id order (FP64) and m_i the
 * particle's mass (mpcd_set_masses) or its box's mass.  FP64 form: v + dp / m, each operation
 * rounded once; mixed form: the FP32 velocity becomes the FP32 rounding of v + dp / m.
 * n must equal mpcd_num_particles.  The device variant is enqueued on the handle's stream;
 * the host one copies dp to the device first and synchronises.
 * Errors: MPCD_ERR_ARG (n != N, NULL). */
int mpcd_add_momentum(mpcd_t* h, int64_t n, const double* dp);
int mpcd_add_momentum_device(mpcd_t* h, int64_t n, const double* dp_dev);

/* Same as mpcd_get_state / mpcd_set_state with device arrays.  get_state_device is enqueued
 * on the handle's stream without a host synchronisation; set_state_device checks the state
 * as mpcd_set_state does, which synchronises once. */
int mpcd_get_state_device(mpcd_t* h, double* r_dev, double* v_dev);
int mpcd_set_state_device(mpcd_t* h, int64_t n, const double* r_dev, const double* v_dev, int64_t t);

/* Record per-cell moments during later steps (enable = 1) or stop (0).  Recording costs an
 * extra 40 bytes of HBM traffic per cell per step. */
int mpcd_record_moments(mpcd_t* h, int32_t enable);

/* Per-cell moments of the last recorded step (Listing 4's vcm plus the kinetic energy):
 * out[5*c + 0..4] = M, Px, Py, Pz, E = sum m v^2 / 2 over the real particles of cell c,
 * before the rotation; shift_out[3] = that step's grid shift (may be NULL).
 * MPCD_ERR_STATE if no step was recorded since recording was enabled.  Synchronises. */
int mpcd_cell_moments(mpcd_t* h, double* out, double* shift_out);

/* The sort of the most recent step (Sec. 3.1 linked-cell list as a stable counting sort):
 * keys[N] = cell key of each storage slot at the start of that step, counts[C],
 * offsets[C+1] (exclusive prefix sum), perm[N] = storage slot of the j-th particle in cell
 * order (stable by storage slot), ids[N] = particle id held by each storage slot at the
 * start of that step.  Any pointer may be NULL.  Key of cell (cx, cy, cz) is
 * cx + Lx (cy + Ly cz).  MPCD_ERR_STATE if no step has run.  Synchronises. */
int mpcd_debug_sort(mpcd_t* h, int32_t* keys, int32_t* counts, int32_t* offsets, int32_t* perm,
                    int32_t* ids);

/* Per-kernel timing with CUDA events on the launching stream.  While enabled, mpcd_step
 * launches kernels one by one (no CUDA graph) and brackets each with events.
 * mpcd_timing_read synchronises and returns, for up to nmax kernels, the summed device
 * milliseconds and launch counts since timing was enabled, plus their names
 * (names[k] points into library-owned storage valid until mpcd_destroy).
 * Returns the number of kernels with data (>= 0) or an error. */
int mpcd_timing(mpcd_t* h, int32_t enable);
int mpcd_timing_read(mpcd_t* h, int32_t nmax, const char** names, double* ms, int64_t* launches);

/* Launch and layout parameters that do not change results (the cell sums are exact, so
 * the order in which particles are stored or visited never matters). */
typedef struct {
  int32_t group_target; /* mixed form: mean particles per warp's group of cells (32..224); */
                        /*   per box at most 24 ppc and 192 - ceil(ppc + 4 sqrt(ppc))     */
  int32_t warps;        /* mixed form: warps per collide block (2 or 4) */
  int32_t resort_k;     /* FP64 form: physical re-sort period in steps (0: never) */
  int32_t fuse;         /* 0 or 1 (default 1 in the FP64 form, 0 in the mixed form).  FP64   */
                        /*   periodic boxes without thermostat: 1                             */
                        /*   applies each step's rotation in the same pass as the next step's */
                        /*   streaming and binning (one pass over the state instead of two;   */
                        /*   the last step of every mpcd_step call still ends with its        */
                        /*   rotation).  Mixed form (without masses or angular-momentum       */
                        /*   conservation): 1 runs a whole step as one persistent cooperative */
                        /*   launch whose phases (zeroing, scan, scatter, group table,        */
                        /*   collision, step end) are separated by bounded grid-wide barriers */
                        /*   (MPCD_ERR_TIMEOUT if one waits too long), 0 as eight launches.   */
                        /*   Identical results either way.                                    */
} mpcd_tuning;

int mpcd_get_tuning(const mpcd_t* h, mpcd_tuning* out);
/* Errors: MPCD_ERR_ARG for out-of-range values (fuse must be 0 or 1). */
int mpcd_set_tuning(mpcd_t* h, const mpcd_tuning* t);

/* Autotuner: times each candidate tuning on the handle's own box(es) for trial_steps steps
 * (CUDA events on the handle's stream), keeps the fastest and restores the state, so the
 * simulation is unchanged.  Candidates: group_target in {128, 144, 160, 168, 176} x warps
 * in {2, 4} x fuse in {1, 0} for the mixed form; resort_k in {1, 2, 5, 10, 20, 50} x fuse in
 * {0, 1} for the FP64 form.
 * *best receives the choice and *best_ms its time per step (either may be NULL). */
int mpcd_autotune(mpcd_t* h, int32_t trial_steps, mpcd_tuning* best, double* best_ms);

/* Test hook for the bounded waits (no counterpart in the paper): with enable = 1, the next
 * one-launch mixed step lets one block leave without reaching its grid barriers, so the other
 * blocks' waits run out after about a second; the step then reports MPCD_ERR_TIMEOUT through
 * mpcd_sync and the handle is poisoned.  The GPU context stays usable.  Not for production. */
int mpcd_debug_stall_barrier(mpcd_t* h, int32_t enable);

/* Number of kernels this handle has launched (graph replays count each kernel node). */
int64_t mpcd_launch_count(const mpcd_t* h);

/* Message of the last failure on this handle, or with h = NULL of the calling thread's last
 * failure without a handle (create, mpcd_step_fp64_noalloc).  The string is owned by the
 * library and stays valid until that slot's next failure. */
const char* mpcd_last_error(const mpcd_t* h);

/* Measurement aid (no counterpart in the paper): this GPU's FP64 fused multiply-add rate,
 * in FP64 operations per second counted per thread (one DFMA of one lane = 1), from chains of
 * independent DFMAs on every SM of the current device, best of three timed launches.  The
 * FP64 form's kernels are bound by this rate, not by HBM, and bench reports them against it.
 * Allocates 8 bytes and a stream for the duration of the call.  Errors: MPCD_ERR_ARG for
 * NULL, MPCD_ERR_CUDA. */
int mpcd_measure_fp64_rate(double* instr_per_s);

/* Library build description, e.g. "libmpcd sm_103a". */
const char* mpcd_version(void);

/* One FP64 step for callers that cannot allocate device memory (no counterpart in the
 * paper; it exists for the library's users).  Some programs may not call cudaMalloc at
 * all: code that runs under a fixed device-memory budget owned by a host framework, code
 * that must not take the allocator's locks or latency inside a time-critical loop, or a
 * plug-in that only receives pointers.  Such a caller keeps its particles in its own device
 * arrays and calls this function instead of mpcd_create / mpcd_step.
 *
 * Advances the box described by p (FP64 only; resort_k is ignored: storage order never
 * changes) from step t to t + 1, in place, on structure-of-arrays device arrays x, y, z,
 * vx, vy, vz of n particles, enqueued on `stream` (NULL: the legacy default stream).
 * Positions must already lie in the box: they are not checked (a check would need a host
 * synchronisation), and a position outside it, or a non-finite value, is clamped into an
 * edge cell, which gives wrong physics without an error.
 *
 * Memory: nothing is allocated.  The sort's scratch lives in one static device array of
 * MPCD_NOALLOC_MAX_PARTICLES particles and MPCD_NOALLOC_MAX_CELLS cells (about 7 MB),
 * which every GPU that loads the library holds until the process exits.  Larger n or cell
 * counts are rejected with MPCD_ERR_ARG.  Every call on a device shares that array and
 * leaves its contents behind, so calls that may overlap on a GPU (different streams without
 * ordering between them) race and give wrong results: serialise them.
 *
 * The first call on each device looks up the array's device address (with that device
 * current) and caches it with the id of the current context; make that first call before
 * any stream capture.  After a device reset the next call looks the address up again (the
 * module is loaded anew), so that call, too, must come before any stream capture.
 * Errors: MPCD_ERR_ARG, MPCD_ERR_CUDA (also when a CUDA error from earlier work is already
 * pending on this thread: it is left pending, and nothing is launched).  The message is read
 * with mpcd_last_error(NULL) on the calling thread (one slot per thread). */
#define MPCD_NOALLOC_MAX_PARTICLES (1 << 19)
#define MPCD_NOALLOC_MAX_CELLS (1 << 17)
int mpcd_step_fp64_noalloc(const mpcd_params* p, int64_t t, int64_t n, double* x, double* y, double* z, double* vx,
                           double* vy, double* vz, void* stream);

#ifdef __cplusplus
}
#endif
#endif
