/*
 * mpcd_oracle.h -- FP64 CPU oracle for one stochastic-rotation-dynamics (SRD) time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may load it; the
 * library under paper_2212_11878_gb300/ never does.  It shares no source, header, table or
 * helper with the CUDA path: it has its own Philox, its own key arithmetic and its own
 * rotation.
 *
 * What it computes (arXiv 2212.11878, Sec. 2 "Multi-Particle Collision Dynamics"):
 *   stream every particle ballistically, shift the collision grid randomly, sort the
 *   particles into the shifted cells (Sec. 3.1, Listing 1), sum mass and momentum per cell
 *   (Sec. 3.3, Listing 4), take each particle's velocity relative to its cell's centre-of-mass
 *   velocity, split it along a random axis and rotate the perpendicular part by a fixed
 *   angle (Sec. 2, parts (i)-(iii)).
 *
 * Where the paper is silent, the oracle takes these readings:
 *   R1 stream then collide inside step t; steps are counted from 1.
 *   R2 shift s uniform in [-a/2, a/2)^3, cell = floor((r - s)/a) mod L.
 *   R3 a wrapped coordinate that rounds to L becomes 0.
 *   R4 with walls the z shift is taken in [0, a) and the z layer is floor((z - s)/a) + 1,
 *      so there are Lz + 1 layers.
 *   R5 key = cx + Lx*(cy + Ly*cz).
 *   R6 inside a cell, particles keep their storage order (stable counting sort).
 *   R7 centre-of-mass velocity u = (sum m v) / (sum m).
 *   R8 rotation by +alpha (right-hand rule about the axis).
 *   R9 random numbers: Philox4x64-10, key (seed, 0), counter (a, b, tag, 0).
 *   R12 cells with fewer than two particles (real + virtual) are left unchanged.
 *   R13 bounce-back walls at z = 0 and z = Lz*a, virtual particles in cut cells.
 *   R14 optional cell-level velocity-rescaling thermostat.
 *   R22 optional Maxwell-Boltzmann-scaling (MBS) thermostat: the target of the R14 rescale
 *       is drawn per cell from the Gamma distribution of the relative kinetic energy of
 *       3(n_c - 1) degrees of freedom (Huang et al. 2010, cited in Sec. 2 and Sec. 4),
 *       with Marsaglia and Tsang's method (ACM TOMS 26(3), 2000).
 *   R23 optional angular-momentum-conserving collision (the variants Sec. 2 mentions, from
 *       the Gompper et al. review it cites): after the rotation (and the thermostat), every
 *       member of a cell gets omega x rho_i, rho_i its position relative to the cell's centre
 *       of mass and omega = I^-1 (L_before - L_after), I the cell's inertia tensor; cells of
 *       two particles use I's pseudo-inverse, cells whose inertia tensor is singular
 *       otherwise are left uncorrected.  Positions within a cell are taken on the shifted
 *       grid (the fractional part of (r - s)/a), so a cell cut by the periodic boundary is
 *       whole.  Not with walls: virtual particles have no positions.
 *   R24 optional per-particle masses (the masses Listing 4 sums): M = sum m_i,
 *       P = sum m_i v_i, E = sum m_i v_i^2 / 2, the thermostat's kinetic energy and the
 *       angular-momentum correction weighted by m_i, the centre of mass of R23 mass-weighted.
 *       The rotation of v - u is unchanged; it conserves sum m_i v_i and sum m_i |v_i|^2 / 2.
 *   R25 before a run the storage may be put in cell order once (orc_presort): a stable sort
 *       by the cell of each position on the unshifted grid, the Listing 1 `permute` applied
 *       to a state that was given in particle-id order.  It moves particles between storage
 *       slots only; the stable in-cell order of R6 then follows the new storage order.
 */
#ifndef MPCD_ORACLE_H
#define MPCD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox counter "tags" (third counter word), reading R9. */
enum { ORC_TAG_INIT = 0, ORC_TAG_SHIFT = 1, ORC_TAG_AXIS = 2, ORC_TAG_THERMO = 3, ORC_TAG_WALL = 4 };

typedef struct {
  int32_t L[3];       /* cells per side */
  int32_t resort_k;   /* physically re-order storage every k steps (0: never) */
  double a;           /* cell edge length */
  double dt;          /* time step */
  double alpha;       /* rotation angle, radians */
  double kT;          /* temperature (energy units) */
  double mass;        /* particle mass, the same for every particle */
  double ppc;         /* mean particles per cell: sets N and fills wall cells */
  double g[3];        /* body-force acceleration */
  uint64_t seed;      /* Philox key word 0 */
  int32_t walls_z;    /* 0: periodic in z; 1: bounce-back walls at z = 0 and z = Lz*a */
  int32_t thermostat; /* 0: none; 1: cell-level rescale of the relative kinetic energy to
                         * 3/2 (n_c - 1) kT; 2: to kT times a Gamma(3/2 (n_c - 1)) draw (R22) */
  int32_t angular;    /* 1: angular-momentum-conserving collision (R23); periodic boxes only */
} orc_params;

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = bijection(ctr) under key. */
void orc_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* (w >> 11) * 2^-53: uniform on [0, 1), exact in FP64. */
double orc_u53(uint64_t w);

int64_t orc_num_cells(const orc_params* p);
/* Grid shift of step t (R2; with walls the z component is folded into [0, a), R4). */
void orc_shift(const orc_params* p, int64_t t, double s[3]);
/* Cell key of position r on the grid shifted by s (R2, R4, R5). */
int64_t orc_cell_key(const orc_params* p, const double r[3], const double s[3]);
/* Random rotation axis of cell `cell` in step t, uniform on the unit sphere (R9). */
void orc_axis(const orc_params* p, int64_t t, int64_t cell, double n[3]);
/* Gamma(shape, 1) variate of cell `cell` in step t for the MBS thermostat (R22), shape >= 1:
 * Marsaglia-Tsang, attempt k on Philox counter (t, cell, THERMO, k); at most 64 attempts,
 * after which it returns shape - 1/3. */
double orc_mbs_gamma(const orc_params* p, int64_t t, int64_t cell, double shape);
/* Position of r inside its cell on the grid shifted by s, in cell units: the fractional
 * part of (r - s)/a per axis (R23). */
void orc_cell_local(const orc_params* p, const double r[3], const double s[3], double l[3]);
/* v <- u + rotation of (v - u) by alpha about unit axis n (Sec. 2, parts (ii)-(iii)). */
void orc_rotate(const double n[3], double alpha, const double u[3], double v[3]);

/* Initial state (positions uniform in the box, velocities Gaussian N(0, kT/m) per
 * component with the mean removed).  r, v: N x 3, row-major. */
void orc_init(const orc_params* p, int64_t n, double* r, double* v);

/* One full step t (t >= 1) on the state (r, v: N x 3 row-major; id: N).
 * Optional outputs (NULL to skip), all describing this step's collision grid:
 *   keys[N]      cell key of each storage slot (storage order at the start of the step)
 *   counts[C]    particles per cell
 *   offsets[C+1] exclusive prefix sum of counts
 *   perm[N]      storage slot of the j-th particle in cell order (stable, R6)
 *   moments[5C]  per cell: M, Px, Py, Pz, E = sum m v^2 / 2 of the real particles, before
 *                the rotation
 *   shift[3]     the grid shift used
 * Returns 0, or -1 on invalid arguments, -2 if memory ran out. */
int orc_step(const orc_params* p, int64_t n, int64_t t, double* r, double* v, int32_t* id,
             int32_t* keys, int32_t* counts, int32_t* offsets, int32_t* perm,
             double* moments, double* shift);
/* orc_step with per-particle masses (R24): mass[N] in storage order (> 0; NULL: every
 * particle has p->mass), permuted with the state on re-sort steps.  The cell sums, the
 * thermostat's kinetic energy and the angular-momentum correction weight by it; virtual wall
 * particles keep p->mass. */
int orc_step_m(const orc_params* p, int64_t n, int64_t t, double* r, double* v, int32_t* id, double* mass,
               int32_t* keys_out, int32_t* counts_out, int32_t* offsets_out, int32_t* perm_out,
               double* moments_out, double* shift_out);

/* Put the storage in cell order before a run (reading R25): a stable sort of the storage
 * slots by the cell key of each position on the unshifted grid (s = 0), the Listing 1
 * `permute` applied once, so that particles of one cell sit together from the first step on.
 * r, v (N x 3), id (N) and mass (N, may be NULL) are permuted together.  0 on success. */
int orc_presort(const orc_params* p, int64_t n, double* r, double* v, int32_t* id, double* mass);

#ifdef __cplusplus
}
#endif
#endif
