// mpcd_internal.h -- data structures shared by the libmpcd host runtime (api.cu) and the
// kernel translation units.  Not part of the public ABI (include/mpcd.h).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mpcd {

// One box as the kernels see it.  All values derived on the host from mpcd_params.  (16-byte
// aligned so that kernels can copy it into shared memory in 16-byte pieces.)
struct alignas(16) Geom {
  int32_t L[3];
  int32_t walls;       // bounce-back walls in z
  int32_t thermostat;  // cell-level rescale of the relative kinetic energy: 1 fixed, 2 MBS
  int32_t resort_k;    // physical re-sort period (0: never)
  int32_t pow2a;       // a is a power of two: (r - s) * (1/a) == (r - s) / a exactly
  int32_t force;       // any g component non-zero
  int32_t log2a;       // a = 2^log2a when pow2a
  int32_t angular;     // angular-momentum-conserving collision (periodic boxes)
  double a, inv_a;
  double B[3];         // box edge lengths L[d] * a
  double dt;
  double g[3];         // body-force acceleration
  double h[3];         // g dt^2 / 2, evaluated as ((0.5 * g) * dt) * dt
  double cos_a, sin_a; // rotation by alpha
  double mass, kT, ppc;
  uint64_t seed;
  int64_t n;           // particles
  int64_t ncell;       // collision cells (walls: Lx Ly (Lz + 1))
  int64_t pbase;       // first particle of the box in the concatenated arrays (batched)
  int64_t cbase;       // first cell key of the box (batched)
  // mixed form: positions in cell units (int cell coordinate + FP32 offset in [0, 1))
  float dta;           // dt / a
  float ha[3];         // g dt^2 / (2 a)
  float gdt[3];        // g dt
  float cos_af, sin_af;
  // FP32 copies of dt, 1/a, g (0 where g is 0), kT and m: a double -> float conversion or a
  // double compare in a kernel would occupy the narrow FP64 pipe
  float dtf, inv_af, gf[3], kTf, massf;
  int32_t bits[3];     // bits of each packed cell coordinate
};

// Device-resident step control, read by every kernel of a step so that one captured CUDA
// graph can replay any step.
struct Ctl {
  int64_t t;            // completed steps; the step in flight is t + 1
  int32_t cur;          // particle buffer set holding the state (0 or 1)
  int32_t err;          // set by a kernel whose bounded grid-barrier wait ran out (one-launch mixed step)
  double shift[3];      // grid shift of step t + 1 (the next step to run)
  double shift_next[3]; // grid shift of step t + 2
  double shift_last[3]; // grid shift of step t (the last completed step)
  double mean[3];       // scratch for the initial-momentum removal
  float sf[3];          // shift of step t + 1 in cell units (mixed form)
  float sf_next[3];     // shift of step t + 2 in cell units (mixed form)
};

// FP64 particle state, structure of arrays, two buffer sets for out-of-place re-sorting.  In
// a handle each set is one allocation, r[k][d] = r[k][0] + d n and v[k][d] = r[k][0] + (3 + d) n
// (the fused rotate-and-stream pass addresses all six from r[k][0]); the allocation-free step
// passes the caller's six arrays and never runs that pass.
struct Fp64Bufs {
  double* r[2][3];
  double* v[2][3];
  int32_t* id[2];
};

// Per-particle masses of the FP64 form in storage order, per buffer set (null: every particle
// has the box mass).  Passed as a separate, last kernel argument, and only to the kernels
// that read it, so the argument layout of every other kernel stays as it is.
struct Fp64Mass {
  double* m[2];
};

// Mixed-precision particle record, 32 bytes (one DRAM sector): in-cell offsets in cell
// units [0, 1), the home cell's coordinates packed as cx | cy << bits[0] | cz << (bits[0] +
// bits[1]), FP32 velocity and the particle id.
struct alignas(32) MixRec {
  float ox, oy, oz;
  int32_t cell;
  float vx, vy, vz;
  int32_t id;
};

// Two record buffers: every mixed step reads one and writes the other in cell order.
struct MixBufs {
  MixRec* rec[2];
};

// Per-particle masses of the mixed form (FP32) in the storage order of each record buffer
// (null: every particle has its box's mass).  A separate, last kernel argument, like Fp64Mass.
struct MixMass {
  float* m[2];
};

// Scratch of the mixed step.  key/count are double-buffered: step t's collide kernel writes
// the keys and counts of step t + 1 for the records it writes; the scatter takes each
// particle's place in its cell from the per-cell cursor.
struct MixScratch {
  int32_t* key[2];
  int32_t* count[2];
  int32_t* cursor;
  int32_t* offset;
  int32_t* perm;
  int32_t* partial;
  double* moments;
};

// Per-step scratch of the counting sort and the cell reduction.
struct Scratch {
  int32_t* key;      // [N] cell key per storage slot (of even steps where key2 is separate)
  int32_t* key2;     // [N] keys of odd steps for the dense pair's fused pass; else == key
  int32_t* rank;     // [N] arrival rank inside the cell (from the counting atomics)
  int32_t* cursor;   // [C] per-cell place cursor of the scatter; null: the scatter uses rank
  int32_t* perm;     // [N] storage slot of the j-th particle in cell order
  int32_t* count;    // [C] particles per cell
  int32_t* offset;   // [C + 1] exclusive prefix sum of count
  int32_t* partial;  // scan partial sums
  double* moments;   // [5 C] per-cell M, Px, Py, Pz, E (only when recording)
  double* frame;     // [16 C] per-cell record: R (9), b (3), rotate flag, 3 unused
  double* red;       // [3 * reduce blocks] partial sums for the initial mean removal
};

// ---- kernel launchers (kernels_*.cu).  All are asynchronous on `st`. ----
int scan_tiles(int64_t count);
void launch_zero_i32(int32_t* p, int64_t n, cudaStream_t st);
void launch_zero_i32_pair(int32_t* p, int32_t* q, int64_t n, cudaStream_t st);  // both arrays, one launch
void launch_scan(const int32_t* count, int32_t* offset, int32_t* partial, int64_t n, cudaStream_t st);

void launch_init_fp64(const Geom& g, Fp64Bufs b, double* red, int red_blocks, Ctl* ctl, cudaStream_t st);
void launch_stream_bin_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, cudaStream_t st);
// perm from keys and ranks: the keys of step ctl->t + 1, or s.key when ctl is null
void launch_scatter(const Geom& g, Scratch s, const Ctl* ctl, cudaStream_t st);
// periodic boxes without thermostat or angular-momentum correction (fp64_dense_collide):
// cell_frame here, then launch_rotate_fp64; otherwise one thread per cell here and no
// rotate launch
bool fp64_dense_collide(const Geom& g, const Scratch& s);
// dst[j] = m_by_id[id[j]]: particle masses into storage order
void launch_gather_masses(int64_t n, const double* m_by_id, const int32_t* id, double* dst, cudaStream_t st);
void launch_collide_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, bool moments, cudaStream_t st, Fp64Mass ms);
// The dense pair's rotation of step ctl->t, launched after that step's end_step (so ctl->cur
// is the buffer set the particles end in); the last step of every mpcd_step call.
void launch_rotate_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, cudaStream_t st, Fp64Mass ms);
// The rotation of step ctl->t fused with the streaming and binning of step ctl->t + 1 (dense
// pair, every step of an mpcd_step call after its first).
void launch_rotate_stream_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, cudaStream_t st, Fp64Mass ms);
// one thread per cell for every box kind (no frame buffer needed)
void launch_collide_fp64_generic(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, bool moments, cudaStream_t st,
                                 Fp64Mass ms = Fp64Mass{});
void launch_end_step(const Geom& g, Ctl* ctl, cudaStream_t st);
void launch_sort_segments(const Geom& g, Scratch s, cudaStream_t st);
// Storage of buffer set 0 into cell order of the unshifted grid (stable by slot), written to
// buffer set 1 with the ids and masses; returns the number of kernels launched.
int launch_presort_fp64(const Geom& g, Fp64Bufs b, Scratch s, Fp64Mass ms, cudaStream_t st);
// A state in particle-id order (N x 3 arrays r, v; masses m_by_id or null) written straight
// into buffer set 1 in that cell order (m_dst: the masses in storage order); returns launches.
// The two halves of launch_set_state_sorted_fp64: the cell order from the positions alone
// (scratch arrays only), then the gather of the state into buffer set 1.
int launch_sort_positions_fp64(const Geom& g, Scratch s, const double* r, cudaStream_t st);
int launch_gather_state_fp64(const Geom& g, Fp64Bufs b, Scratch s, const double* r, const double* v,
                             const double* m_by_id, double* m_dst, cudaStream_t st);
// The gather's two halves into buffer set `set`: positions and ids; velocities and masses.
int launch_gather_positions_fp64(const Geom& g, Fp64Bufs b, Scratch s, const double* r, int set, cudaStream_t st);
int launch_gather_velocities_fp64(const Geom& g, Fp64Bufs b, Scratch s, const double* v, int set,
                                  const double* m_by_id, double* m_dst, cudaStream_t st);
int launch_set_state_sorted_fp64(const Geom& g, Fp64Bufs b, Scratch s, const double* r, const double* v,
                                 const double* m_by_id, double* m_dst, cudaStream_t st);
void launch_get_state_fp64(const Geom& g, Fp64Bufs b, int cur, double* r, double* v, cudaStream_t st);
// slot_of[id] = storage slot (N ints), then the state of particles p0 .. p1 - 1 by id into
// N x 3 arrays: lets a host copy of the state run in chunks beside the gathers
void launch_slot_of(const Geom& g, Fp64Bufs b, int cur, int32_t* slot_of, cudaStream_t st);
void launch_gather_by_id(int64_t p0, int64_t p1, const int32_t* slot_of, Fp64Bufs b, int cur, double* r, double* v,
                         cudaStream_t st);
// v += dp / m per particle (dp[3 N] by particle id, m its mass or the box mass)
void launch_add_momentum_fp64(const Geom& g, Fp64Bufs b, int cur, Fp64Mass ms, const double* dp, cudaStream_t st);

// ---- mixed form (kernels_mixed.cu); one box or an ensemble of independent boxes ----
// A group of consecutive cells of one box, handled by one warp; rewritten every step
// (k_group_bounds) so that each group holds about the target number of records.
struct MixGroup {
  int64_t c0;      // first cell (global key)
  int32_t box;
  int32_t ncells;  // groups of more than 32 cells take the per-cell path
};

// The fixed part of a group: it starts at the first cell of its box whose record offset
// reaches rec0 (the box's first group starts at the box's first cell).
struct MixGroupSpec {
  int64_t rec0;   // first record of the group's range (global, cell order)
  int64_t rec1;   // first record of the next group of the box, or -1 for the box's last group
  int32_t box;
  int32_t pad;
};

// Grid shifts of one box (each box draws its own from its seed).
struct BoxShift {
  double s[3];       // step t + 1
  double s_next[3];  // step t + 2
  double s_last[3];  // step t
  float sf[3];       // step t + 1, cell units
  float sf_next[3];  // step t + 2, cell units
};

// Device tables of the mixed form.  Box b owns particles [pbase[b], pbase[b+1]) and cells
// [boxes[b].cbase, boxes[b].cbase + boxes[b].ncell) of the concatenated arrays.
struct MixBatch {
  const Geom* boxes;
  BoxShift* shifts;
  const MixGroup* groups;
  const int64_t* pbase;
  int32_t nbox;
  int32_t ngroups;
  int64_t n;      // particles of all boxes
  int64_t ncell;  // cells of all boxes
  int32_t walls, force, thermostat, warps;  // uniform over boxes; warps per collide block
  int32_t angular, pad;                     // uniform over boxes: every group takes the per-cell path
};

constexpr int kMixCap = 192;  // records one warp stages (larger groups take the per-cell path)
void mixed_box_shifts(const Geom& g, int64_t t, BoxShift* out);  // host: shifts of steps t+1, t+2
void launch_init_mixed_box(const Geom& g, MixBufs b, double* red, int red_blocks, Ctl* ctl, cudaStream_t st);
void launch_bin_mixed(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, cudaStream_t st);
// Set up the collide kernels on the current device (shared-memory limit, persistent grid);
// call once per device before the first launch, outside stream capture.
cudaError_t prepare_collide_mixed();
// With masses (ms.m[0] non-null) every group takes the per-cell path with mass-weighted sums.
void launch_collide_stream_mixed(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, bool moments, cudaStream_t st,
                                 MixMass ms = MixMass{});
void launch_end_step_mixed(const MixBatch& mb, Ctl* ctl, cudaStream_t st);
// The whole mixed step (staged path: no masses, no angular-momentum correction) in one
// cooperative persistent launch: zeroing, scan, scatter, group table, collision, step end.
// bar: two device counters, 0 between steps; stall (tests only): block 0 skips the barriers
// so the others' bounded waits run out and ctl->err is set.
// Tile sums the one-launch step needs at most (its tiles hold 32 x warps x 8 cells): the
// size of MixScratch::partial, with the three-kernel scan's scan_tiles.
int64_t step_scan_tiles(int64_t ncell);
cudaError_t launch_step_mixed(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, bool moments,
                              const MixGroupSpec* spec, MixGroup* groups, unsigned* bar, int stall, cudaStream_t st);
void launch_scatter_cursor(int64_t n, const int32_t* key, const int32_t* offset, int32_t* cursor, int32_t* perm,
                           cudaStream_t st);
// Rewrite the group table from this step's offsets.
void launch_group_bounds(const MixBatch& mb, const MixGroupSpec* spec, const int32_t* offset, MixGroup* groups,
                         cudaStream_t st);
void launch_get_state_mixed(const MixBatch& mb, MixBufs b, int cur, double* r, double* v, cudaStream_t st);
// masses by particle id into the FP32 storage-order array of record buffer rec
void launch_gather_masses_mixed(int64_t n, const MixRec* rec, const double* m_by_id, float* dst, cudaStream_t st);
void launch_add_momentum_mixed(const MixBatch& mb, MixBufs b, int cur, MixMass ms, const double* dp, cudaStream_t st);
void launch_set_state_mixed(const MixBatch& mb, MixBufs b, const double* r, const double* v, cudaStream_t st);
// First invalid particle of a state (position outside its box, non-finite velocity) into
// *bad, which the caller sets to ~0 first: per box of *mb, or for the single box g if mb is NULL.
void launch_check_positions(const Geom& g, int64_t n, const double* r, unsigned long long* bad, cudaStream_t st);
void launch_check_velocities(int64_t n, const double* v, unsigned long long* bad, cudaStream_t st);
void launch_check_state(const MixBatch* mb, const Geom& g, int64_t n, const double* r, const double* v,
                        unsigned long long* bad, cudaStream_t st);

}  // namespace mpcd
