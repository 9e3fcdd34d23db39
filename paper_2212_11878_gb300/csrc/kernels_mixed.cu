// kernels_mixed.cu -- the mixed-precision form of the SRD step.
//
// State: one 32-byte record per particle (MixRec): position as the home cell's integer
// coordinates plus an FP32 offset in [0, 1) cell units, FP32 velocity, particle id.
//
// Step t (after the first step, three launches plus the scan):
//   scatter         perm[offset[key] + cursor[key]++] = slot (keys were written by step t-1)
//   collide_stream  one warp per group of cells.  The warp gathers its cells' records
//                   through perm into shared memory and
//                     1. streams each particle from r_{t-1} to r_t (FP32, in cell units);
//                     2. per cell: exact momentum sum, centre-of-mass velocity u, random
//                        axis, rotation of v - u by alpha (paper Sec. 2 (ii)-(iii)), a
//                        rescale that restores the cell's relative kinetic energy (the
//                        rotation conserves it exactly; FP32 rounding does not) and a
//                        correction that restores the cell's exact momentum;
//                     3. streams each particle once more to r_{t+1} to get its cell key on
//                        the grid of step t+1 and counts it there (no-return atomics);
//                     4. writes (r_t, v_t) in cell order to the other record buffer, so the
//                        storage is re-sorted every step at no extra traffic.
// Lanes take records for the per-particle work (gather, stream, rotation, write-out) and
// cells for the per-cell work (sums, frame), with the per-cell data in shared memory.
// Every per-cell sum is an exact integer (fixed point, order-independent), so the result
// does not depend on the order in which the atomics delivered a cell's members and is a
// function of the state alone.  No FP64 arithmetic runs per particle or per cell (except
// for the virtual particles of wall cells).
#include "cellmath.cuh"
#include "device_common.cuh"
#include "mpcd_internal.h"

namespace mpcd {

namespace {
constexpr int kThreads = 256;


unsigned grid_for(int64_t n, int per_thread = 1) {
  int64_t blocks = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 64) blocks = 152 * 64;
  return static_cast<unsigned>(blocks);
}

// ------------------------------------------------------------ packed coordinates ----
__device__ __forceinline__ void unpack_cell(const Geom& g, int32_t c, int cc[3]) {
  cc[0] = c & ((1 << g.bits[0]) - 1);
  cc[1] = (c >> g.bits[0]) & ((1 << g.bits[1]) - 1);
  cc[2] = c >> (g.bits[0] + g.bits[1]);
}

__device__ __forceinline__ int32_t pack_cell(const Geom& g, const int cc[3]) {
  return cc[0] | (cc[1] << g.bits[0]) | (cc[2] << (g.bits[0] + g.bits[1]));
}

// ----------------------------------------------------------------- FP32 streaming ----
// Carry whole cells from the offset x into the coordinate c.
__device__ __forceinline__ void carry(float& x, int& c, int L, bool periodic) {
  if (x >= 1.0f || x < 0.0f) {
    const float fl = floorf(x);
    int k = static_cast<int>(fl);
    x = __fsub_rn(x, fl);
    if (x >= 1.0f) {  // a value just below an integer rounded onto it
      x = 0.0f;
      k += 1;
    }
    c += k;
    if (periodic && (c < 0 || c >= L)) {
      c %= L;
      if (c < 0) c += L;
    }
  }
}

// Ballistic move over dt in cell units (v in length/time), with the body force and, when
// WALLS, bounce-back at z = 0 and z = Lz (velocity reversed at the crossing time).
template <int WALLS, int FORCE>
__device__ __forceinline__ void stream_mixed(const Geom& g, float f[3], int cc[3], float v[3]) {
  if (!WALLS) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (FORCE) {
        f[d] = __fadd_rn(fmaf(v[d], g.dta, f[d]), g.ha[d]);
        v[d] = __fadd_rn(v[d], g.gdt[d]);
      } else {
        f[d] = fmaf(v[d], g.dta, f[d]);
      }
      carry(f[d], cc[d], g.L[d], true);
    }
    return;
  }
  const float inv_a = static_cast<float>(g.inv_a);
  const int Lz = g.L[2];
  float left = static_cast<float>(g.dt);
  for (int bounce = 0; bounce < 8 && left > 0.0f; ++bounce) {
    const float vz_c = v[2] * inv_a;  // cells per unit time
    const float zrel = fmaf(vz_c, left, f[2]);
    float tau = left;
    int wall = 0;
    if (zrel < -static_cast<float>(cc[2])) {
      tau = -(static_cast<float>(cc[2]) + f[2]) / vz_c;
      wall = -1;
    } else if (zrel >= static_cast<float>(Lz - cc[2])) {
      tau = (static_cast<float>(Lz - cc[2]) - f[2]) / vz_c;
      wall = 1;
    }
    if (!(tau > 0.0f)) tau = 0.0f;
    if (tau > left) tau = left;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const float gt = g.g[d] != 0.0 ? static_cast<float>(g.g[d]) : 0.0f;
      f[d] = fmaf(fmaf(0.5f * gt, tau, v[d]), tau * inv_a, f[d]);
      v[d] = fmaf(gt, tau, v[d]);
      carry(f[d], cc[d], g.L[d], true);
    }
    if (wall == 0) {
      f[2] = fmaf(vz_c, tau, f[2]);
      carry(f[2], cc[2], Lz, false);
      left = 0.0f;
    } else {
      if (wall < 0) {
        cc[2] = 0;
        f[2] = 0.0f;
      } else {
        cc[2] = Lz - 1;
        f[2] = 1.0f;  // on the top wall; the reversed velocity moves it back inside
      }
      v[0] = -v[0];
      v[1] = -v[1];
      v[2] = -v[2];
      left = __fsub_rn(left, tau);
    }
  }
  if (cc[2] < 0) {
    cc[2] = 0;
    f[2] = 0.0f;
  }
  if (cc[2] >= Lz) {
    cc[2] = Lz - 1;
    f[2] = 0.99999994f;
  }
  if (f[2] >= 1.0f) f[2] = 0.99999994f;
  if (f[2] < 0.0f) f[2] = 0.0f;
}

// Cell key on the grid shifted by sf (cell units); with walls sf[2] lies in [0, 1).
template <int WALLS>
__device__ __forceinline__ int mixed_key(const Geom& g, const float f[3], const int cc[3], const float sf[3]) {
  int k[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int c = cc[d];
    if (WALLS && d == 2) {
      c += (f[2] < sf[2]) ? 0 : 1;  // layers 0 .. Lz
      c = c < 0 ? 0 : (c > g.L[2] ? g.L[2] : c);
    } else {
      const float x = __fsub_rn(f[d], sf[d]);
      c += (x < 0.0f) ? -1 : (x >= 1.0f ? 1 : 0);
      if (c < 0) c += g.L[d];
      else if (c >= g.L[d]) c -= g.L[d];
    }
    k[d] = c;
  }
  return k[0] + g.L[0] * (k[1] + g.L[1] * k[2]);
}

// Axis and rotation in FP32 from the same Philox draw as the FP64 form.
__device__ __forceinline__ void frame_f32(const Geom& g, int64_t t1, int64_t cell, float R[9]) {
  const u64x4 w = draw(g.seed, static_cast<uint64_t>(t1), static_cast<uint64_t>(cell), kTagAxis);
  const float z = fmaf(2.0f, static_cast<float>(w.x >> 40) * 0x1.0p-24f, -1.0f);
  float sp, cp;
  sincospif(2.0f * (static_cast<float>(w.y >> 40) * 0x1.0p-24f), &sp, &cp);
  const float rho = sqrtf((1.0f - z) * (1.0f + z));
  const float n0 = rho * cp, n1 = rho * sp, n2 = z;
  const float c = g.cos_af, s = g.sin_af, om = 1.0f - g.cos_af;
  const float wx = om * n0, wy = om * n1, wz = om * n2;
  R[0] = fmaf(wx, n0, c);
  R[1] = fmaf(wx, n1, -s * n2);
  R[2] = fmaf(wx, n2, s * n1);
  R[3] = fmaf(wy, n0, s * n2);
  R[4] = fmaf(wy, n1, c);
  R[5] = fmaf(wy, n2, -s * n0);
  R[6] = fmaf(wz, n0, -s * n1);
  R[7] = fmaf(wz, n1, s * n0);
  R[8] = fmaf(wz, n2, c);
}

// ---------------------------------------------------------------- per-cell collision ----
// Member access for the cell routine, in particle-id order: records already streamed to
// r_t; their velocity slots receive the collided velocity.


// Exact sum of FP32 values in fixed point with F fractional bits: x * 2^F (an exact FP32
// product) is truncated to an int64 and added (exact when x's ulp is at least 2^-F).
// Returns false, leaving the sum unchanged, if |x| >= 2^LIM.  Integer addition is
// associative, so the total does not depend on the order of the terms.
template <int F, int LIM>
__device__ __forceinline__ bool fxf_add(long long& a, float x) {
  if (!(fabsf(x) < static_cast<float>(1ull << (LIM + 24)) * 0x1.0p-24f)) return false;  // also rejects NaN
  a += __float2ll_rz(x * static_cast<float>(1ull << (F > 62 ? 62 : F)) *
                     (F > 62 ? static_cast<float>(1ull << (F - 62)) : 1.0f));
  return true;
}

// Velocities and squared lengths: 2^-36 grid, |x| < 2^14, up to 2^13 terms.
__device__ __forceinline__ bool fx_v(long long& a, float x) { return fxf_add<36, 14>(a, x); }
// Energy differences of order 1e-7: 2^-56 grid, |x| < 2^-2, up to 2^9 terms.
__device__ __forceinline__ bool fx_de(long long& a, float x) { return fxf_add<56, -2>(a, x); }

// Per-cell data the particle passes need.
struct CellFrame {
  float u[3];
  float R[9];
  float df;
  int rot;
};

// The per-cell step before the rotation, from the exact momentum sums S (2^-36 fixed
// point): centre-of-mass velocity (with the virtual particles of a cut wall cell), whether
// the cell rotates, and its rotation.
template <int WALLS>
__device__ __forceinline__ void cell_prologue(const Geom& g, const long long S[3], int n, int64_t c, int64_t t1,
                                              double shift_z, CellFrame& f) {
  f.rot = 0;
  f.df = 0.0f;
  if (n == 0) return;
  const float scale = 0x1.0p-36f / static_cast<float>(n);
  f.u[0] = __ll2float_rn(S[0]) * scale;
  f.u[1] = __ll2float_rn(S[1]) * scale;
  f.u[2] = __ll2float_rn(S[2]) * scale;
  bool virt = false;
  if (WALLS) {
    const int64_t layer = c / ((int64_t)g.L[0] * g.L[1]);
    if (shift_z > 0.0 && (layer == 0 || layer == g.L[2]) && (double)n < g.ppc) {
      // R13: virtual particles fill the cut cell to ppc, at rest on average (FP64, wall cells only)
      const double m = g.mass;
      const double Mv = (g.ppc - (double)n) * m;
      const u64x4 w = draw(g.seed, static_cast<uint64_t>(t1), static_cast<uint64_t>(c), kTagWall);
      double g0, g1, g2, g3;
      gauss_pair(w.x, w.y, g0, g1);
      gauss_pair(w.z, w.w, g2, g3);
      const double sd = sqrt(Mv * g.kT);
      const double Mt = (double)n * m + Mv;
      f.u[0] = static_cast<float>((m * __ll2double_rn(S[0]) * 0x1.0p-36 + sd * g0) / Mt);
      f.u[1] = static_cast<float>((m * __ll2double_rn(S[1]) * 0x1.0p-36 + sd * g1) / Mt);
      f.u[2] = static_cast<float>((m * __ll2double_rn(S[2]) * 0x1.0p-36 + sd * g2) / Mt);
      virt = true;
    }
  }
  if (n < 2 && !virt) return;
  f.rot = 1;
  frame_f32(g, t1, c, f.R);
}

// w = R (v - u) for one particle, and |v - u|^2 - |w|^2.
__device__ __forceinline__ float rotate_relative(const CellFrame& f, float v[3]) {
  const float d0 = __fsub_rn(v[0], f.u[0]), d1 = __fsub_rn(v[1], f.u[1]), d2 = __fsub_rn(v[2], f.u[2]);
  const float w0 = fmaf(f.R[0], d0, fmaf(f.R[1], d1, f.R[2] * d2));
  const float w1 = fmaf(f.R[3], d0, fmaf(f.R[4], d1, f.R[5] * d2));
  const float w2 = fmaf(f.R[6], d0, fmaf(f.R[7], d1, f.R[8] * d2));
  const float eb = fmaf(d0, d0, fmaf(d1, d1, __fmul_rn(d2, d2)));
  v[0] = w0;
  v[1] = w1;
  v[2] = w2;
  return __fsub_rn(eb, fmaf(w0, w0, fmaf(w1, w1, __fmul_rn(w2, w2))));
}

__device__ __forceinline__ float sq3(const float w[3]) { return fmaf(w[0], w[0], fmaf(w[1], w[1], __fmul_rn(w[2], w[2]))); }

// Scale factor 1 + df of the rotated relative velocities.  The rotation keeps |v - u|
// exactly; in FP32 the squared lengths drift by about 1e-7, so df = sum(|v-u|^2 - |w|^2) /
// (2 sum |w|^2): the sum of the small differences is accurate on its own, and the cell's
// relative kinetic energy is restored to FP32 rounding of the stored velocities.  With the
// thermostat, df sets it to 3/2 (n - 1) kT instead.  dE: 2^-56 fixed point, Ea: 2^-36.
template <int THERMO>
__device__ __forceinline__ float cell_df(const Geom& g, int n, long long dE, long long Ea, bool ok) {
  if (!ok || Ea <= 0) return 0.0f;
  const float ea = __ll2float_rn(Ea) * 0x1.0p-36f;
  if (THERMO && n >= 2)
    return sqrtf(3.0f * static_cast<float>(n - 1) * static_cast<float>(g.kT) / (static_cast<float>(g.mass) * ea)) -
           1.0f;
  return 0.5f * (__ll2float_rn(dE) * 0x1.0p-56f) / ea;
}

__device__ __forceinline__ void write_moments_mixed(const Geom& g, double* moments, int64_t c, int n, const long long S[3],
                                                    long long E2) {
  double* mo = moments + 5 * c;
  mo[0] = static_cast<double>(n) * g.mass;
  mo[1] = g.mass * __ll2double_rn(S[0]) * 0x1.0p-36;
  mo[2] = g.mass * __ll2double_rn(S[1]) * 0x1.0p-36;
  mo[3] = g.mass * __ll2double_rn(S[2]) * 0x1.0p-36;
  mo[4] = 0.5 * g.mass * __ll2double_rn(E2) * 0x1.0p-36;
}

// Velocities of a cell's members: SoA arrays in shared memory (stride 1) or AoS records in
// global memory (stride 8 floats).
struct V3 {
  float* x;
  float* y;
  float* z;
  int stride;
  __device__ __forceinline__ float& vx(int j) const { return x[j * stride]; }
  __device__ __forceinline__ float& vy(int j) const { return y[j * stride]; }
  __device__ __forceinline__ float& vz(int j) const { return z[j * stride]; }
};

// Exact sums over a cell's velocities (and v.v for the moments).
template <int MOMENTS>
__device__ __forceinline__ bool cell_sums_mixed(const V3& v, int n, long long S[3], long long& E2) {
  S[0] = S[1] = S[2] = 0;
  E2 = 0;
  bool ok = n < 8192;
  for (int j = 0; j < n; ++j) {
    const float a = v.vx(j), b = v.vy(j), c = v.vz(j);
    ok &= fx_v(S[0], a) & fx_v(S[1], b) & fx_v(S[2], c);
    if (MOMENTS) ok &= fx_v(E2, fmaf(a, a, fmaf(b, b, __fmul_rn(c, c))));
  }
  return ok;
}

// Exact energy sums over a cell's rotated relative velocities w and their terms
// |v - u|^2 - |w|^2, then the scale factor.
template <int THERMO>
__device__ __forceinline__ float cell_energy(const Geom& g, const V3& w, const float* term, int tstride, int n) {
  long long dE = 0, Ea = 0;
  bool oke = n < 512;
  for (int j = 0; j < n; ++j) {
    const float ww[3] = {w.vx(j), w.vy(j), w.vz(j)};
    oke &= fx_de(dE, term[j * tstride]) & fx_v(Ea, sq3(ww));
  }
  return cell_df<THERMO>(g, n, dE, Ea, oke);
}

// The whole collision of one cell by one thread over AoS records rec[0..n-1] in global
// memory (crowded cells).  Its energy sums are accumulated during the rotation instead of
// from stored terms; being exact integer sums they equal the staged path's bit for bit.
template <int WALLS, int THERMO, int MOMENTS>
__device__ void mixed_collide_cell(const Geom& g, MixRec* rec, int n, int64_t c, int64_t t1, double shift_z,
                                   double* moments) {
  const V3 v{&rec[0].vx, &rec[0].vy, &rec[0].vz, 8};
  long long S[3], E2;
  const bool ok = cell_sums_mixed<MOMENTS>(v, n, S, E2);
  if (MOMENTS) write_moments_mixed(g, moments, c, n, S, E2);
  CellFrame f;
  cell_prologue<WALLS>(g, S, n, c, t1, shift_z, f);
  if (!f.rot || !ok) return;
  long long dE = 0, Ea = 0;
  bool oke = n < 512;
  for (int j = 0; j < n; ++j) {
    float w[3] = {v.vx(j), v.vy(j), v.vz(j)};
    const float term = rotate_relative(f, w);
    v.vx(j) = w[0];
    v.vy(j) = w[1];
    v.vz(j) = w[2];
    oke &= fx_de(dE, term) & fx_v(Ea, sq3(w));
  }
  const float df = cell_df<THERMO>(g, n, dE, Ea, oke);
  for (int j = 0; j < n; ++j) {
    v.vx(j) = __fadd_rn(f.u[0], fmaf(df, v.vx(j), v.vx(j)));
    v.vy(j) = __fadd_rn(f.u[1], fmaf(df, v.vy(j), v.vy(j)));
    v.vz(j) = __fadd_rn(f.u[2], fmaf(df, v.vz(j), v.vz(j)));
  }
}

// Stream one record from r_{t-1} to r_t in place.
template <int WALLS, int FORCE>
__device__ __forceinline__ void stream_record(const Geom& g, MixRec& r) {
  float f[3] = {r.ox, r.oy, r.oz};
  float v[3] = {r.vx, r.vy, r.vz};
  int cc[3];
  unpack_cell(g, r.cell, cc);
  stream_mixed<WALLS, FORCE>(g, f, cc, v);
  r.ox = f[0];
  r.oy = f[1];
  r.oz = f[2];
  r.vx = v[0];
  r.vy = v[1];
  r.vz = v[2];
  r.cell = pack_cell(g, cc);
}

// Key of a record's position after one more stream (the grid of the next step).
template <int WALLS, int FORCE>
__device__ __forceinline__ int next_key(const Geom& g, const MixRec& r, const float sf[3]) {
  float f[3] = {r.ox, r.oy, r.oz};
  float v[3] = {r.vx, r.vy, r.vz};
  int cc[3];
  unpack_cell(g, r.cell, cc);
  stream_mixed<WALLS, FORCE>(g, f, cc, v);
  return mixed_key<WALLS>(g, f, cc, sf);
}

__device__ __forceinline__ MixRec load_rec(const MixRec* __restrict__ p) {
  const float4* q = reinterpret_cast<const float4*>(p);
  const float4 a = __ldg(q), b = __ldg(q + 1);
  MixRec r;
  r.ox = a.x;
  r.oy = a.y;
  r.oz = a.z;
  r.cell = __float_as_int(a.w);
  r.vx = b.x;
  r.vy = b.y;
  r.vz = b.z;
  r.id = __float_as_int(b.w);
  return r;
}

__device__ __forceinline__ void store_rec(MixRec* __restrict__ p, const MixRec& r) {
  float4* q = reinterpret_cast<float4*>(p);
  q[0] = make_float4(r.ox, r.oy, r.oz, __int_as_float(r.cell));
  q[1] = make_float4(r.vx, r.vy, r.vz, __int_as_float(r.id));
}

// ----------------------------------------------------------------------- kernels ----
// Box of particle i (pbase is sorted; nbox + 1 entries).
__device__ __forceinline__ int box_of(const int64_t* __restrict__ pbase, int nbox, int64_t i) {
  int lo = 0, hi = nbox;  // pbase[lo] <= i < pbase[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pbase[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int WALLS, int FORCE>
__global__ void __launch_bounds__(kThreads) k_bin_mixed(MixBatch mb, MixBufs b, MixScratch s, Ctl* __restrict__ ctl) {
  const int cur = ctl->cur;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mb.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int bx = box_of(mb.pbase, mb.nbox, i);
    const Geom& g = mb.boxes[bx];
    const float sf[3] = {mb.shifts[bx].sf[0], mb.shifts[bx].sf[1], mb.shifts[bx].sf[2]};
    const MixRec r = load_rec(b.rec[cur] + i);
    const int k = static_cast<int>(g.cbase) + next_key<WALLS, FORCE>(g, r, sf);
    s.key[cur][i] = k;
    atomicAdd(&s.count[cur][k], 1);
  }
}

// Shared-memory staging of one warp's records, structure of arrays: lanes that walk
// different cells read different banks.
struct MixStage {
  float ox[kMixCap], oy[kMixCap], oz[kMixCap];
  int32_t cell[kMixCap];
  float vx[kMixCap], vy[kMixCap], vz[kMixCap];
  int32_t id[kMixCap];
  float term[kMixCap];  // |v-u|^2 - |w|^2 of each record
  uint8_t seg[kMixCap]; // cell of each record within the group
  float fr[14][32];     // per cell: u (3), R (9), df, rotate flag
};

__device__ __forceinline__ void stage_put(MixStage& st, int e, const MixRec& r) {
  st.ox[e] = r.ox;
  st.oy[e] = r.oy;
  st.oz[e] = r.oz;
  st.cell[e] = r.cell;
  st.vx[e] = r.vx;
  st.vy[e] = r.vy;
  st.vz[e] = r.vz;
  st.id[e] = r.id;
}

__device__ __forceinline__ MixRec stage_get(const MixStage& st, int e) {
  MixRec r;
  r.ox = st.ox[e];
  r.oy = st.oy[e];
  r.oz = st.oz[e];
  r.cell = st.cell[e];
  r.vx = st.vx[e];
  r.vy = st.vy[e];
  r.vz = st.vz[e];
  r.id = st.id[e];
  return r;
}

// One warp per group of cells of one box (the group table never straddles boxes).  The
// per-cell random axis is keyed on the cell's index inside its box, so a box advanced in
// an ensemble reproduces the same box advanced alone.
template <int WARPS, int WALLS, int FORCE, int THERMO, int MOMENTS>
__global__ void __launch_bounds__(WARPS * 32) k_collide_stream_mixed(MixBatch mb, MixBufs b, MixScratch s,
                                                                    Ctl* __restrict__ ctl) {
  __shared__ MixStage stage[WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gi = (int64_t)blockIdx.x * WARPS + warp;
  if (gi >= mb.ngroups) return;
  const MixGroup grp = mb.groups[gi];
  const Geom& g = mb.boxes[grp.box];
  const BoxShift& sh = mb.shifts[grp.box];
  const int64_t t1 = ctl->t + 1;
  const int cur = ctl->cur, nxt = cur ^ 1;
  const float sf[3] = {sh.sf_next[0], sh.sf_next[1], sh.sf_next[2]};  // grid of the next step
  const double shz = sh.s[2];                                        // grid of this step
  const int cbase = static_cast<int>(g.cbase);
  const int64_t c0 = grp.c0;
  const int64_t cend = c0 + grp.ncells;
  const int64_t c = c0 + lane;
  const bool live = lane < grp.ncells;
  const int64_t cl = c - cbase;  // cell index inside the box
  const int E0 = s.offset[c0];
  const int E1 = s.offset[cend];
  const int E = E1 - E0;
  const MixRec* __restrict__ src = b.rec[cur];
  MixRec* __restrict__ dst = b.rec[nxt];
  int32_t* __restrict__ knext = s.key[nxt];
  int32_t* __restrict__ cnext = s.count[nxt];
  if (E > kMixCap) {
    // too many records to stage: one cell per lane, in place in the destination buffer
    if (live) {
      const int o = s.offset[c];
      const int n = s.offset[c + 1] - o;
      const int32_t* pm = s.perm + o;
      for (int j = 0; j < n; ++j) {
        MixRec r = load_rec(src + pm[j]);
        stream_record<WALLS, FORCE>(g, r);
        dst[o + j] = r;
      }
      mixed_collide_cell<WALLS, THERMO, MOMENTS>(g, dst + o, n, cl, t1, shz, MOMENTS ? s.moments + 5 * cbase : nullptr);
      for (int j = 0; j < n; ++j) {
        const int k = cbase + next_key<WALLS, FORCE>(g, dst[o + j], sf);
        knext[o + j] = k;
        atomicAdd(&cnext[k], 1);
      }
    }
    return;
  }
  MixStage& st = stage[warp];
  const int o = live ? s.offset[c] : E1;
  const int n = live ? s.offset[c + 1] - o : 0;
  const int lo = o - E0;
  // 1. gather (a batch of loads in flight per lane) and stream to r_t (lane = record); tag
  //    each staged record with its cell (lane = cell)
  constexpr int kBatch = 4;
  for (int base = 0; base < E; base += 32 * kBatch) {
    int slot[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const int e = base + lane + 32 * k;
      slot[k] = e < E ? s.perm[E0 + e] : 0;
    }
    MixRec rec[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const int e = base + lane + 32 * k;
      if (e < E) rec[k] = load_rec(src + slot[k]);
    }
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const int e = base + lane + 32 * k;
      if (e < E) {
        stream_record<WALLS, FORCE>(g, rec[k]);
        stage_put(st, e, rec[k]);
      }
    }
  }
  for (int j = 0; j < n; ++j) st.seg[lo + j] = static_cast<uint8_t>(lane);
  __syncwarp();
  // 2. per cell (lane = cell): exact momentum sums, centre-of-mass velocity, frame
  if (live) {
    const V3 v{st.vx + lo, st.vy + lo, st.vz + lo, 1};
    long long S[3], E2;
    const bool ok = cell_sums_mixed<MOMENTS>(v, n, S, E2);
    if (MOMENTS) write_moments_mixed(g, s.moments, c, n, S, E2);
    CellFrame f;
    cell_prologue<WALLS>(g, S, n, cl, t1, shz, f);
#pragma unroll
    for (int k = 0; k < 3; ++k) st.fr[k][lane] = f.u[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) st.fr[3 + k][lane] = f.R[k];
    st.fr[13][lane] = (f.rot && ok) ? 1.0f : 0.0f;
  }
  __syncwarp();
  // 3. rotate (lane = record): w = R (v - u) and the energy term of each particle
  for (int e = lane; e < E; e += 32) {
    const int j = st.seg[e];
    if (st.fr[13][j] != 0.0f) {
      CellFrame f;
#pragma unroll
      for (int k = 0; k < 3; ++k) f.u[k] = st.fr[k][j];
#pragma unroll
      for (int k = 0; k < 9; ++k) f.R[k] = st.fr[3 + k][j];
      float w[3] = {st.vx[e], st.vy[e], st.vz[e]};
      st.term[e] = rotate_relative(f, w);
      st.vx[e] = w[0];
      st.vy[e] = w[1];
      st.vz[e] = w[2];
    }
  }
  __syncwarp();
  // 4. per cell: exact energy sums, scale factor
  if (live && st.fr[13][lane] != 0.0f) {
    const V3 w{st.vx + lo, st.vy + lo, st.vz + lo, 1};
    st.fr[12][lane] = cell_energy<THERMO>(g, w, st.term + lo, 1, n);
  }
  __syncwarp();
  // 5. new velocities, keys and counts of the next step, write-out in cell order
  for (int e = lane; e < E; e += 32) {
    MixRec r = stage_get(st, e);
    const int j = st.seg[e];
    if (st.fr[13][j] != 0.0f) {
      const float df = st.fr[12][j];
      r.vx = __fadd_rn(st.fr[0][j], fmaf(df, r.vx, r.vx));
      r.vy = __fadd_rn(st.fr[1][j], fmaf(df, r.vy, r.vy));
      r.vz = __fadd_rn(st.fr[2][j], fmaf(df, r.vz, r.vz));
    }
    const int k = cbase + next_key<WALLS, FORCE>(g, r, sf);
    store_rec(dst + E0 + e, r);
    knext[E0 + e] = k;
    atomicAdd(&cnext[k], 1);
  }
}

__global__ void __launch_bounds__(kThreads) k_scatter_cursor(int64_t n, const int32_t* __restrict__ key,
                                                             const int32_t* __restrict__ offset, int32_t* __restrict__ cursor,
                                                             int32_t* __restrict__ perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
    const int64_t j = i + stride;
    const int k0 = key[i];
    const int k1 = j < n ? key[j] : 0;
    const int p0 = offset[k0] + atomicAdd(&cursor[k0], 1);
    const int p1 = j < n ? offset[k1] + atomicAdd(&cursor[k1], 1) : 0;
    perm[p0] = static_cast<int32_t>(i);
    if (j < n) perm[p1] = static_cast<int32_t>(j);
  }
}

__device__ __forceinline__ void box_shifts(const Geom& g, int64_t t, BoxShift& b) {
  grid_shift(g.seed, t + 1, g.a, g.walls, b.s);
  grid_shift(g.seed, t + 2, g.a, g.walls, b.s_next);
  shift_in_cells(g, b.s, b.sf);
  shift_in_cells(g, b.s_next, b.sf_next);
}

__global__ void k_end_step_mixed(MixBatch mb, Ctl* ctl) {
  const int64_t t = ctl->t + 1;  // completed steps after this one
  for (int bx = blockIdx.x * blockDim.x + threadIdx.x; bx < mb.nbox; bx += gridDim.x * blockDim.x) {
    BoxShift& sh = mb.shifts[bx];
    for (int d = 0; d < 3; ++d) sh.s_last[d] = sh.s[d];
    box_shifts(mb.boxes[bx], t, sh);
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->t = t;
    ctl->cur ^= 1;
  }
}

// ---- initial state, the same Philox draws as the FP64 form (one box per launch) ----
__device__ __forceinline__ void init_draw(const Geom& g, int64_t i, double r[3], double v[3]) {
  const double sigma = sqrt(g.kT / g.mass);
  const u64x4 w = draw(g.seed, static_cast<uint64_t>(i), 0, kTagInit);
  r[0] = unit53(w.x) * g.B[0];
  r[1] = unit53(w.y) * g.B[1];
  r[2] = unit53(w.z) * g.B[2];
  const u64x4 q = draw(g.seed, static_cast<uint64_t>(i), 1, kTagInit);
  double g0, g1, g2, g3;
  gauss_pair(q.x, q.y, g0, g1);
  gauss_pair(q.z, q.w, g2, g3);
  v[0] = sigma * g0;
  v[1] = sigma * g1;
  v[2] = sigma * g2;
}

__device__ __forceinline__ MixRec to_record(const Geom& g, const double r[3], const double v[3], int32_t id) {
  MixRec rec;
  float f[3];
  int cc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double q = g.pow2a ? r[d] * g.inv_a : r[d] / g.a;
    double fl = floor(q);
    float x = static_cast<float>(q - fl);
    int c = static_cast<int>(fl);
    if (x >= 1.0f) {
      x = 0.0f;
      c += 1;
    }
    if (c >= g.L[d]) c -= g.L[d];
    if (c < 0) c = 0;
    f[d] = x;
    cc[d] = c;
  }
  rec.ox = f[0];
  rec.oy = f[1];
  rec.oz = f[2];
  rec.cell = pack_cell(g, cc);
  rec.vx = static_cast<float>(v[0]);
  rec.vy = static_cast<float>(v[1]);
  rec.vz = static_cast<float>(v[2]);
  rec.id = id;
  return rec;
}

__device__ __forceinline__ double block_sum_fixed(double v, double* sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads) k_init_mixed_sum(Geom g, double* __restrict__ red) {
  __shared__ double sm[kThreads];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    double r[3], v[3];
    init_draw(g, i, r, v);
    acc[0] += v[0];
    acc[1] += v[1];
    acc[2] += v[2];
  }
  for (int d = 0; d < 3; ++d) {
    const double tot = block_sum_fixed(acc[d], sm);
    if (threadIdx.x == 0) red[3 * blockIdx.x + d] = tot;
  }
}

__global__ void __launch_bounds__(kThreads) k_init_mixed_mean(const double* __restrict__ red, int nblk, int64_t n,
                                                              Ctl* ctl) {
  __shared__ double sm[kThreads];
  for (int d = 0; d < 3; ++d) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) acc += red[3 * k + d];
    const double tot = block_sum_fixed(acc, sm);
    if (threadIdx.x == 0) ctl->mean[d] = n > 0 ? tot / (double)n : 0.0;
  }
}

__global__ void __launch_bounds__(kThreads) k_init_mixed_write(Geom g, MixBufs b, const Ctl* __restrict__ ctl) {
  const double m0 = ctl->mean[0], m1 = ctl->mean[1], m2 = ctl->mean[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    double r[3], v[3];
    init_draw(g, i, r, v);
    v[0] -= m0;
    v[1] -= m1;
    v[2] -= m2;
    store_rec(b.rec[0] + g.pbase + i, to_record(g, r, v, static_cast<int32_t>(g.pbase + i)));
  }
}

__global__ void __launch_bounds__(kThreads) k_set_state_mixed(MixBatch mb, MixBufs b, const double* __restrict__ r,
                                                              const double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mb.n; i += (int64_t)gridDim.x * blockDim.x) {
    const Geom& g = mb.boxes[box_of(mb.pbase, mb.nbox, i)];
    const double ri[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]};
    const double vi[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
    store_rec(b.rec[0] + i, to_record(g, ri, vi, static_cast<int32_t>(i)));
  }
}

__global__ void __launch_bounds__(kThreads) k_get_state_mixed(MixBatch mb, const MixRec* __restrict__ rec,
                                                              double* __restrict__ r, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mb.n; i += (int64_t)gridDim.x * blockDim.x) {
    const MixRec q = load_rec(rec + i);
    const int64_t p = q.id;
    const Geom& g = mb.boxes[box_of(mb.pbase, mb.nbox, p)];
    int cc[3];
    unpack_cell(g, q.cell, cc);
    r[3 * p + 0] = ((double)cc[0] + (double)q.ox) * g.a;
    r[3 * p + 1] = ((double)cc[1] + (double)q.oy) * g.a;
    r[3 * p + 2] = ((double)cc[2] + (double)q.oz) * g.a;
    v[3 * p + 0] = q.vx;
    v[3 * p + 1] = q.vy;
    v[3 * p + 2] = q.vz;
  }
}
}  // namespace

int mixed_cells_per_group(double ppc, int target) {
  int gc = ppc > 0.0 ? static_cast<int>(target / ppc) : 32;
  if (gc > 32) gc = 32;
  if (gc < 1) gc = 1;
  return gc;
}

void mixed_box_shifts(const Geom& g, int64_t t, BoxShift* out) {
  grid_shift(g.seed, t + 1, g.a, g.walls, out->s);
  grid_shift(g.seed, t + 2, g.a, g.walls, out->s_next);
  for (int d = 0; d < 3; ++d) out->s_last[d] = 0.0;
  shift_in_cells(g, out->s, out->sf);
  shift_in_cells(g, out->s_next, out->sf_next);
}

void launch_init_mixed_box(const Geom& g, MixBufs b, double* red, int red_blocks, Ctl* ctl, cudaStream_t st) {
  k_init_mixed_sum<<<red_blocks, kThreads, 0, st>>>(g, red);
  k_init_mixed_mean<<<1, kThreads, 0, st>>>(red, red_blocks, g.n, ctl);
  k_init_mixed_write<<<grid_for(g.n), kThreads, 0, st>>>(g, b, ctl);
}

void launch_bin_mixed(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, cudaStream_t st) {
  if (mb.walls)
    k_bin_mixed<1, 1><<<grid_for(mb.n), kThreads, 0, st>>>(mb, b, s, ctl);
  else if (mb.force)
    k_bin_mixed<0, 1><<<grid_for(mb.n), kThreads, 0, st>>>(mb, b, s, ctl);
  else
    k_bin_mixed<0, 0><<<grid_for(mb.n), kThreads, 0, st>>>(mb, b, s, ctl);
}

template <int WARPS>
void launch_collide_w(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, bool moments, cudaStream_t st) {
  const unsigned grid = static_cast<unsigned>((mb.ngroups + WARPS - 1) / WARPS);
  if (grid == 0) return;
  const int sel = (mb.walls ? 8 : (mb.force ? 4 : 0)) | (mb.thermostat ? 2 : 0) | (moments ? 1 : 0);
  switch (sel) {
    case 0: k_collide_stream_mixed<WARPS, 0, 0, 0, 0><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 1: k_collide_stream_mixed<WARPS, 0, 0, 0, 1><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 2: k_collide_stream_mixed<WARPS, 0, 0, 1, 0><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 3: k_collide_stream_mixed<WARPS, 0, 0, 1, 1><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 4: k_collide_stream_mixed<WARPS, 0, 1, 0, 0><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 5: k_collide_stream_mixed<WARPS, 0, 1, 0, 1><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 6: k_collide_stream_mixed<WARPS, 0, 1, 1, 0><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 7: k_collide_stream_mixed<WARPS, 0, 1, 1, 1><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 8: k_collide_stream_mixed<WARPS, 1, 1, 0, 0><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 9: k_collide_stream_mixed<WARPS, 1, 1, 0, 1><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    case 10: k_collide_stream_mixed<WARPS, 1, 1, 1, 0><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
    default: k_collide_stream_mixed<WARPS, 1, 1, 1, 1><<<grid, WARPS * 32, 0, st>>>(mb, b, s, ctl); break;
  }
}

void launch_collide_stream_mixed(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, bool moments, cudaStream_t st) {
  if (mb.warps == 2)
    launch_collide_w<2>(mb, b, s, ctl, moments, st);
  else
    launch_collide_w<4>(mb, b, s, ctl, moments, st);
}

void launch_end_step_mixed(const MixBatch& mb, Ctl* ctl, cudaStream_t st) { k_end_step_mixed<<<1, 256, 0, st>>>(mb, ctl); }

void launch_scatter_cursor(int64_t n, const int32_t* key, const int32_t* offset, int32_t* cursor, int32_t* perm,
                           cudaStream_t st) {
  k_scatter_cursor<<<grid_for(n, 2), kThreads, 0, st>>>(n, key, offset, cursor, perm);
}

void launch_get_state_mixed(const MixBatch& mb, MixBufs b, int cur, double* r, double* v, cudaStream_t st) {
  k_get_state_mixed<<<grid_for(mb.n), kThreads, 0, st>>>(mb, b.rec[cur], r, v);
}

void launch_set_state_mixed(const MixBatch& mb, MixBufs b, const double* r, const double* v, cudaStream_t st) {
  k_set_state_mixed<<<grid_for(mb.n), kThreads, 0, st>>>(mb, b, r, v);
}

}  // namespace mpcd
