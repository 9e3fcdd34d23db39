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
#include <mutex>

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

// carry() for a periodic coordinate c in [0, L) and x in [-1, 2) (a move of at most one
// cell): the same result without a branch.
__device__ __forceinline__ void carry_near(float& x, int& c, int L) {
  // k = +1 for x in [1, 2), -1 for x in [-1, 0), 0 otherwise; x - k is exact for k = +1 and
  // rounds like x + 1 for k = -1 (both as in carry()); all selects, no branches
  const int up = x >= 1.0f, dn = x < 0.0f;
  const float y = __fsub_rn(x, up ? 1.0f : (dn ? -1.0f : 0.0f));
  const int onto = y >= 1.0f;  // a value just below an integer rounded onto it
  x = onto ? 0.0f : y;
  c += up - dn + onto;
  c += (c < 0) ? L : 0;
  c -= (c >= L) ? L : 0;
}

__device__ __forceinline__ void carry_periodic(float& x, int& c, int L) {
  if (x >= -1.0f && x < 2.0f)
    carry_near(x, c, L);
  else
    carry(x, c, L, true);
}

// Ballistic move over dt in cell units (v in length/time), with the body force and, when
// WALLS, bounce-back at z = 0 and z = Lz (velocity reversed at the crossing time).
// NEAR: the caller has checked (moves_near) that no coordinate moves by a cell or more and,
// with walls, (stays_inside) that the particle reaches no wall within dt, so the carry needs
// no test and there is no bounce; the result is the same as without NEAR.
template <int WALLS, int FORCE, int NEAR = 0>
__device__ __forceinline__ void stream_mixed(const Geom& g, float f[3], int cc[3], float v[3]) {
  if (WALLS && NEAR) {
    // the first pass of the bounce loop below when it finds no wall: tau = dt
    const float inv_a = g.inv_af;
    const float tau = g.dtf;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const float gt = g.gf[d];
      f[d] = fmaf(fmaf(0.5f * gt, tau, v[d]), tau * inv_a, f[d]);
      v[d] = fmaf(gt, tau, v[d]);
      carry_near(f[d], cc[d], g.L[d]);
    }
    f[2] = fmaf(v[2] * inv_a, tau, f[2]);
    carry_near(f[2], cc[2], g.L[2]);  // stays in [0, Lz): the wrap never applies
    return;
  }
  if (!WALLS && NEAR) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (FORCE) {
        f[d] = __fadd_rn(fmaf(v[d], g.dta, f[d]), g.ha[d]);
        v[d] = __fadd_rn(v[d], g.gdt[d]);
      } else {
        f[d] = fmaf(v[d], g.dta, f[d]);
      }
      carry_near(f[d], cc[d], g.L[d]);
    }
    return;
  }
  if (!WALLS) {
    bool near = true;  // every coordinate moved by at most one cell
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (FORCE) {
        f[d] = __fadd_rn(fmaf(v[d], g.dta, f[d]), g.ha[d]);
        v[d] = __fadd_rn(v[d], g.gdt[d]);
      } else {
        f[d] = fmaf(v[d], g.dta, f[d]);
      }
      near = near && f[d] >= -1.0f && f[d] < 2.0f;
    }
    if (near) {
#pragma unroll
      for (int d = 0; d < 3; ++d) carry_near(f[d], cc[d], g.L[d]);
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) carry(f[d], cc[d], g.L[d], true);
    }
    return;
  }
  const float inv_a = g.inv_af;
  const int Lz = g.L[2];
  float left = g.dtf;
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
      const float gt = g.gf[d];
      f[d] = fmaf(fmaf(0.5f * gt, tau, v[d]), tau * inv_a, f[d]);
      v[d] = fmaf(gt, tau, v[d]);
      carry_periodic(f[d], cc[d], g.L[d]);
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
      c += static_cast<int>(x >= 1.0f) - static_cast<int>(x < 0.0f);
      c += (c < 0) ? g.L[d] : 0;
      c -= (c >= g.L[d]) ? g.L[d] : 0;
    }
    k[d] = c;
  }
  return k[0] + g.L[0] * (k[1] + g.L[1] * k[2]);
}

// A 53-bit integer 0 <= m < 2^53 times 2^-53, rounded to FP32 from its two halves (no 64-bit
// conversion, which would use the FP64 pipe).
__device__ __forceinline__ float u53_f32(uint64_t m) {
  const float hi = static_cast<float>(static_cast<uint32_t>(m >> 21));           // exact below 2^24, else RN
  const float lo = static_cast<float>(static_cast<uint32_t>(m & 0x1FFFFFull));   // exact
  return fmaf(hi, 0x1.0p-32f, lo * 0x1.0p-53f);
}

// Gamma(shape, 1) variate of the Maxwell-Boltzmann-scaling thermostat in FP32: the same
// Marsaglia-Tsang steps and Philox counters (t, cell, THERMO, k) as the FP64 form, with the
// uniforms rounded from their 53-bit integers.  Not inlined: it runs once per cell, only in
// the kernels instantiated for this thermostat (THERMO = 2).
__device__ __noinline__ float mbs_gamma_f32(uint64_t seed, int64_t t, int64_t cell, float shape) {
  const float d = shape - (1.0f / 3.0f);
  const float c = rsqrtf(9.0f * d);
  for (uint64_t k = 0; k < 64; ++k) {
    const u64x4 w = philox4x64_10(static_cast<uint64_t>(t), static_cast<uint64_t>(cell), kTagThermo, k, seed, 0);
    const uint64_t m0 = w.x >> 11, m2 = w.z >> 11;
    const float u1 = m0 ? u53_f32((1ull << 53) - m0) : 1.0f;  // (0, 1]
    const float x = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u53_f32(w.y >> 11));
    const float tt = fmaf(c, x, 1.0f);
    if (tt <= 0.0f) continue;
    const float v = tt * tt * tt;
    const float u = m2 ? u53_f32((1ull << 53) - m2) : 1.0f;
    const float x2 = x * x;
    if (u < 1.0f - 0.0331f * (x2 * x2)) return d * v;
    if (logf(u) < 0.5f * x2 + d * ((1.0f - v) + logf(v))) return d * v;
  }
  return d;
}

// Axis and rotation in FP32 from the same Philox draw as the FP64 form: U = U53(w0), the
// axis z = 2U - 1 = U - (1 - U) and rho = sqrt(1 - z^2) = 2 sqrt(U (1 - U)), with U and
// 1 - U each taken from the 53-bit integer, so that rho keeps full FP32 accuracy near the
// poles (1 - z from a rounded z would lose it); phi = 2 pi U53(w1).
__device__ __forceinline__ void frame_f32(const Geom& g, int64_t t1, int64_t cell, float R[9]) {
  const u64x4 w = draw(g.seed, static_cast<uint64_t>(t1), static_cast<uint64_t>(cell), kTagAxis);
  const uint64_t mz = w.x >> 11;
  const float U = u53_f32(mz), Uc = mz ? u53_f32((1ull << 53) - mz) : 1.0f;  // U in [0, 1), 1 - U in (0, 1]
  const float z = __fsub_rn(U, Uc);
  float sp, cp;
  sincospif(2.0f * u53_f32(w.y >> 11), &sp, &cp);
  const float rho = 2.0f * sqrtf(U * Uc);
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


// Exact sums of FP32 values on the fixed-point grid 2^-F.  A value is split into two int32
// parts, x = (h 2^23 + lo) 2^-F to the nearest grid point: h = x 2^(F-23) rounded to an
// integer and lo the remainder in units of 2^-F.  Both come from FP32 fused multiply-adds
// whose result lands on the integer grid of the constant 1.5 * 2^23 (|h| <= 2^21, |lo| <=
// 2^22), so the split costs a few FMA-pipe instructions (GB300's 64-bit conversions share its
// narrow FP64 pipe).  Returns false, with both parts 0, for |x| >= 2^(44-F) or a non-finite
// x.  Integer sums of the parts do not depend on the order of the terms; the sums of up to
// 256 terms fit in int32.
template <int F>
__device__ __forceinline__ bool fix_split(float x, int& h, int& lo) {
  static_assert(F >= 23 && F <= 44, "grid");
  constexpr float kScale = static_cast<float>(1ull << (F - 23));
  constexpr float kLimit = static_cast<float>(1ull << (44 - F));
  constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
  const bool ok = fabsf(x) < kLimit;
  const float t = fmaf(x, kScale, kRound);
  const float rem = fmaf(x, kScale, -__fsub_rn(t, kRound));  // exact: x 2^(F-23) - h
  const float t2 = fmaf(rem, 8388608.0f, kRound);
  h = ok ? __float_as_int(t) - 0x4B400000 : 0;
  lo = ok ? __float_as_int(t2) - 0x4B400000 : 0;
  return ok;
}

// The fixed-point value h 2^23 + lo of a split (or of sums of splits).
__device__ __forceinline__ long long fix_join(int h, int lo) {
  return static_cast<long long>(h) * 8388608LL + static_cast<long long>(lo);
}

// a += x on the grid 2^-F (int64 accumulator, for cells of any size).
template <int F>
__device__ __forceinline__ bool fx_add(long long& a, float x) {
  int h, lo;
  const bool ok = fix_split<F>(x, h, lo);
  a += fix_join(h, lo);
  return ok;
}

// Grids of the per-cell sums: velocities 2^-32 (|v| < 2^12), squared lengths 2^-30 (< 2^14),
// energy differences 2^-44 (|x| < 1).
constexpr int kFixV = 32, kFixV2 = 30, kFixDE = 44;

// An int64 rounded to the nearest FP32 (ties to even), on the integer pipe; the same value
// as __ll2float_rn.
__device__ __forceinline__ float ll_to_float(long long s) {
  const unsigned long long a = s < 0 ? 0ull - static_cast<unsigned long long>(s) : static_cast<unsigned long long>(s);
  if (a == 0ull) return 0.0f;
  const int lz = __clzll(static_cast<long long>(a));
  const unsigned long long nrm = a << lz;                 // leading one at bit 63
  unsigned mant = static_cast<unsigned>(nrm >> 40);      // 24 bits
  const unsigned long long rem = nrm & 0xFFFFFFFFFFull;  // 40 bits below
  if (rem > 0x8000000000ull || (rem == 0x8000000000ull && (mant & 1u))) ++mant;
  unsigned ex = static_cast<unsigned>(63 - lz + 127);
  if (mant == 0x1000000u) {
    mant >>= 1;
    ++ex;
  }
  return __uint_as_float((s < 0 ? 0x80000000u : 0u) | (ex << 23) | (mant & 0x7FFFFFu));
}

// Per-cell data the particle passes need.
struct CellFrame {
  float u[3];
  float R[9];
  float df;
  int rot;
};

// The per-cell step before the rotation, from the exact momentum sums S (2^-36 fixed
// point): centre-of-mass velocity (with the virtual particles of a cut wall cell) and
// whether the cell rotates.  The rotation itself (frame_f32) needs no particle data.
template <int WALLS>
__device__ __forceinline__ void cell_prologue_u(const Geom& g, const long long S[3], int n, int64_t c, int64_t t1,
                                                double shift_z, CellFrame& f) {
  f.rot = 0;
  f.df = 0.0f;
  if (n == 0) return;
  const float scale = 0x1.0p-32f / static_cast<float>(n);
  f.u[0] = ll_to_float(S[0]) * scale;
  f.u[1] = ll_to_float(S[1]) * scale;
  f.u[2] = ll_to_float(S[2]) * scale;
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
      f.u[0] = static_cast<float>((m * __ll2double_rn(S[0]) * 0x1.0p-32 + sd * g0) / Mt);
      f.u[1] = static_cast<float>((m * __ll2double_rn(S[1]) * 0x1.0p-32 + sd * g1) / Mt);
      f.u[2] = static_cast<float>((m * __ll2double_rn(S[2]) * 0x1.0p-32 + sd * g2) / Mt);
      virt = true;
    }
  }
  f.rot = (n >= 2 || virt) ? 1 : 0;
}

template <int WALLS>
__device__ __forceinline__ void cell_prologue(const Geom& g, const long long S[3], int n, int64_t c, int64_t t1,
                                              double shift_z, CellFrame& f) {
  cell_prologue_u<WALLS>(g, S, n, c, t1, shift_z, f);
  if (f.rot) frame_f32(g, t1, c, f.R);
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
// thermostat, df sets it to 3/2 (n - 1) kT instead, or with the Maxwell-Boltzmann-scaling
// thermostat to kT times a Gamma(3/2 (n - 1)) draw for (step t1, cell).  dE: 2^-44 fixed
// point, Ea: 2^-30.
template <int THERMO>
__device__ __forceinline__ float cell_df(const Geom& g, int n, long long dE, long long Ea, bool ok, int64_t t1,
                                         int64_t cell) {
  if (!ok || Ea <= 0) return 0.0f;
  const float ea = ll_to_float(Ea) * 0x1.0p-30f;
  if (THERMO && n >= 2) {
    const float dof = THERMO == 2 ? 2.0f * mbs_gamma_f32(g.seed, t1, cell, 1.5f * static_cast<float>(n - 1))
                                  : 3.0f * static_cast<float>(n - 1);
    return sqrtf(dof * g.kTf / (g.massf * ea)) - 1.0f;
  }
  return 0.5f * (ll_to_float(dE) * 0x1.0p-44f) / ea;
}

__device__ __forceinline__ void write_moments_mixed(const Geom& g, double* moments, int64_t c, int n, const long long S[3],
                                                    long long E2) {
  double* mo = moments + 5 * c;
  mo[0] = static_cast<double>(n) * g.mass;
  mo[1] = g.mass * __ll2double_rn(S[0]) * 0x1.0p-32;
  mo[2] = g.mass * __ll2double_rn(S[1]) * 0x1.0p-32;
  mo[3] = g.mass * __ll2double_rn(S[2]) * 0x1.0p-32;
  mo[4] = 0.5 * g.mass * __ll2double_rn(E2) * 0x1.0p-30;
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
    ok &= fx_add<kFixV>(S[0], a) & fx_add<kFixV>(S[1], b) & fx_add<kFixV>(S[2], c);
    if (MOMENTS) ok &= fx_add<kFixV2>(E2, fmaf(a, a, fmaf(b, b, __fmul_rn(c, c))));
  }
  return ok;
}

// Position of a streamed record inside its cell of this step's grid (shift sf, cell units),
// exact in FP64: the offset less the shift less the whole cells that the key counted.
__device__ __forceinline__ void mixed_local(const MixRec& r, const float sf[3], double l[3]) {
  const float f[3] = {r.ox, r.oy, r.oz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float x = __fsub_rn(f[d], sf[d]);
    const int k = static_cast<int>(x >= 1.0f) - static_cast<int>(x < 0.0f);
    l[d] = static_cast<double>(f[d]) - static_cast<double>(sf[d]) - static_cast<double>(k);
  }
}

// Angular-momentum-conserving collision (the variant the paper mentions in Sec. 2), mixed
// form, from the cell's moments: with in-cell positions l (exact in FP64) and velocities v
// before the collision, A = sum l, Q = sum l l^T, B = sum l v^T and P = sum v, accumulated as
// exact fixed-point sums of the FP64 products (two FP32 factors), so the member order does
// not matter.  The moments about the centre are M = a (B - lbar P^T) and S = a^2 (Q - n lbar
// lbar^T); L_before = eps : M and, after w = R (v - u) and the rescale by 1 + df,
// L_after = (1 + df) eps : (M R^T); I = tr(S) 1 - S; omega = I^-1 (L_before - L_after) as
// in the FP64 form.  Each member then gets (a omega) x (l - lbar).
struct CellMoments {
  Fx128 A[3], Q[6], B[9], P[3];
};

__device__ __forceinline__ void moments_zero(CellMoments& cm) {
  for (int k = 0; k < 3; ++k) fx_zero(cm.A[k]), fx_zero(cm.P[k]);
  for (int k = 0; k < 6; ++k) fx_zero(cm.Q[k]);
  for (int k = 0; k < 9; ++k) fx_zero(cm.B[k]);
}

// Adds a streamed record; false if a term left the exact range (the cell is then not corrected).
__device__ __forceinline__ bool moments_add(CellMoments& cm, const MixRec& r, const float sf[3]) {
  double l[3];
  mixed_local(r, sf, l);
  const double v[3] = {r.vx, r.vy, r.vz};
  bool ok = true;
  for (int d = 0; d < 3; ++d) ok &= fx_add(cm.A[d], l[d]) & fx_add(cm.P[d], v[d]);
  ok &= fx_add(cm.Q[0], l[0] * l[0]) & fx_add(cm.Q[1], l[1] * l[1]) & fx_add(cm.Q[2], l[2] * l[2]);
  ok &= fx_add(cm.Q[3], l[0] * l[1]) & fx_add(cm.Q[4], l[0] * l[2]) & fx_add(cm.Q[5], l[1] * l[2]);
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) ok &= fx_add(cm.B[3 * x + y], l[x] * v[y]);
  return ok;
}

// a omega and lbar of a cell of n >= 2 members (aw = 0 when I is singular); l0: the in-cell
// position of one member (the two-particle case needs their separation).
__device__ __noinline__ void mixed_omega(const Geom* __restrict__ gp, const CellMoments* __restrict__ cm, const float* Rf,
                                         float df, int n, const double* l0, double* aw, double* lbar) {
  const double a = gp->a;
  double R[9], A[3], Q[6], B[9], P[3];
  for (int k = 0; k < 9; ++k) R[k] = Rf[k], B[k] = fx_value(cm->B[k]);
  for (int k = 0; k < 3; ++k) A[k] = fx_value(cm->A[k]), P[k] = fx_value(cm->P[k]);
  for (int k = 0; k < 6; ++k) Q[k] = fx_value(cm->Q[k]);
  aw[0] = aw[1] = aw[2] = 0.0;
  for (int d = 0; d < 3; ++d) lbar[d] = A[d] / n;
  double Mm[3][3], S[3][3], N[3][3];
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) Mm[x][y] = a * (B[3 * x + y] - lbar[x] * P[y]);
  const int qi[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) S[x][y] = a * a * (Q[qi[x][y]] - n * lbar[x] * lbar[y]);
  const double sc = 1.0 + static_cast<double>(df);
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) N[x][y] = sc * (Mm[x][0] * R[3 * y] + Mm[x][1] * R[3 * y + 1] + Mm[x][2] * R[3 * y + 2]);
  const double dL[3] = {(Mm[1][2] - Mm[2][1]) - (N[1][2] - N[2][1]), (Mm[2][0] - Mm[0][2]) - (N[2][0] - N[0][2]),
                        (Mm[0][1] - Mm[1][0]) - (N[0][1] - N[1][0])};
  const double tr = S[0][0] + S[1][1] + S[2][2];
  double I[3][3], w[3] = {0.0, 0.0, 0.0};
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) I[x][y] = (x == y ? tr : 0.0) - S[x][y];
  if (n == 2) {  // the pair lies on one line: I acts as tr(S) normal to it
    const double q[3] = {a * (l0[0] - lbar[0]), a * (l0[1] - lbar[1]), a * (l0[2] - lbar[2])};
    const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    if (!(qq > 0.0) || !(tr > 0.0)) return;
    const double along = (q[0] * dL[0] + q[1] * dL[1] + q[2] * dL[2]) / qq;
    for (int d = 0; d < 3; ++d) w[d] = (dL[d] - along * q[d]) / tr;
  } else {
    double cof[3][3];
    for (int x = 0; x < 3; ++x)
      for (int y = 0; y < 3; ++y) {
        const int x1 = (x + 1) % 3, x2 = (x + 2) % 3, y1 = (y + 1) % 3, y2 = (y + 2) % 3;
        cof[x][y] = I[x1][y1] * I[x2][y2] - I[x1][y2] * I[x2][y1];
      }
    const double det = I[0][0] * cof[0][0] + I[0][1] * cof[0][1] + I[0][2] * cof[0][2];
    const double t3 = (I[0][0] + I[1][1] + I[2][2]) / 3.0;
    if (!(det > 1e-12 * t3 * t3 * t3)) return;
    for (int x = 0; x < 3; ++x) w[x] = (cof[x][0] * dL[0] + cof[x][1] * dL[1] + cof[x][2] * dL[2]) / det;
  }
  for (int d = 0; d < 3; ++d) aw[d] = a * w[d];
}

// The whole collision of one cell by one thread over AoS records rec[0..n-1] in global
// memory (crowded cells, and every cell with angular-momentum conservation, which also gets
// this step's shift sf in cell units and the cell's moments cm).  Its sums accumulate the
// same fixed-point parts in int64, so they equal the staged path's bit for bit.
template <int WALLS, int THERMO, int MOMENTS, int ANG = 0>
__device__ void mixed_collide_cell(const Geom& g, MixRec* rec, int n, int64_t c, int64_t t1, double shift_z,
                                   double* moments, const float* sf, const CellMoments* cm = nullptr,
                                   bool cm_ok = false) {
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
    oke &= fx_add<kFixDE>(dE, term) & fx_add<kFixV2>(Ea, sq3(w));
  }
  const float df = cell_df<THERMO>(g, n, dE, Ea, oke, t1, c);
  float aw[3] = {0.0f, 0.0f, 0.0f}, lb[3] = {0.0f, 0.0f, 0.0f};
  const bool spin = ANG && !WALLS && n >= 2 && cm_ok;
  if (spin) {
    double l0[3], awd[3], lbd[3];
    mixed_local(rec[0], sf, l0);
    mixed_omega(&g, cm, f.R, df, n, l0, awd, lbd);
    for (int d = 0; d < 3; ++d) aw[d] = static_cast<float>(awd[d]), lb[d] = static_cast<float>(lbd[d]);
  }
  for (int j = 0; j < n; ++j) {
    float nx = __fadd_rn(f.u[0], fmaf(df, v.vx(j), v.vx(j)));
    float ny = __fadd_rn(f.u[1], fmaf(df, v.vy(j), v.vy(j)));
    float nz = __fadd_rn(f.u[2], fmaf(df, v.vz(j), v.vz(j)));
    if (ANG && spin) {  // + (a omega) x (l - lbar), in FP32
      float q[3];
      for (int d = 0; d < 3; ++d) {
        const float x = __fsub_rn((&rec[j].ox)[d], sf[d]);
        q[d] = __fsub_rn(x, static_cast<float>(static_cast<int>(x >= 1.0f) - static_cast<int>(x < 0.0f))) - lb[d];
      }
      nx += aw[1] * q[2] - aw[2] * q[1];
      ny += aw[2] * q[0] - aw[0] * q[2];
      nz += aw[0] * q[1] - aw[1] * q[0];
    }
    v.vx(j) = nx;
    v.vy(j) = ny;
    v.vz(j) = nz;
  }
}

// True when streaming a particle with velocity v moves each in-cell offset f in [0, 1) by
// less than 0.99 cells (with the body-force term): f + v dt / a then stays in (-1, 2) after
// rounding, which is all that carry_near needs.
template <int FORCE>
__device__ __forceinline__ bool moves_near(const Geom& g, const MixRec& r) {
  float m = fmaxf(fabsf(r.vx), fmaxf(fabsf(r.vy), fabsf(r.vz))) * g.dta;  // NaN: not near
  if (FORCE) m += fmaxf(fabsf(g.ha[0]), fmaxf(fabsf(g.ha[1]), fabsf(g.ha[2])));
  return m < 0.99f;
}

// With walls: true when streaming the record over dt > 0 reaches neither wall, by the same
// test as the first pass of the bounce loop in stream_mixed (NaN: false).
__device__ __forceinline__ bool stays_inside(const Geom& g, const MixRec& r) {
  const int cz = r.cell >> (g.bits[0] + g.bits[1]);
  const float tau = g.dtf;
  const float zrel = fmaf(r.vz * g.inv_af, tau, r.oz);
  return tau > 0.0f && zrel >= -static_cast<float>(cz) && zrel < static_cast<float>(g.L[2] - cz);
}

// Stream one record from r_{t-1} to r_t in place.
template <int WALLS, int FORCE, int NEAR = 0>
__device__ __forceinline__ void stream_record(const Geom& g, MixRec& r) {
  float f[3] = {r.ox, r.oy, r.oz};
  float v[3] = {r.vx, r.vy, r.vz};
  int cc[3];
  unpack_cell(g, r.cell, cc);
  stream_mixed<WALLS, FORCE, NEAR>(g, f, cc, v);
  r.ox = f[0];
  r.oy = f[1];
  r.oz = f[2];
  r.vx = v[0];
  r.vy = v[1];
  r.vz = v[2];
  r.cell = pack_cell(g, cc);
}

// Out-of-line general forms, for the rare warps holding a particle that moves a cell or more
// (records pass by value, so calling them stores nothing to memory).
template <int WALLS, int FORCE>
__device__ __noinline__ MixRec stream_record_general(const Geom* __restrict__ g, MixRec r) {
  stream_record<WALLS, FORCE>(*g, r);
  return r;
}

// Key of a record's position after one more stream (the grid of the next step).
template <int WALLS, int FORCE, int NEAR = 0>
__device__ __forceinline__ int next_key(const Geom& g, const MixRec& r, const float sf[3]) {
  float f[3] = {r.ox, r.oy, r.oz};
  float v[3] = {r.vx, r.vy, r.vz};
  int cc[3];
  unpack_cell(g, r.cell, cc);
  stream_mixed<WALLS, FORCE, NEAR>(g, f, cc, v);
  return mixed_key<WALLS>(g, f, cc, sf);
}

template <int WALLS, int FORCE>
__device__ __noinline__ int next_key_general(const Geom* __restrict__ g, MixRec r, float sf0, float sf1, float sf2) {
  const float sf[3] = {sf0, sf1, sf2};
  return next_key<WALLS, FORCE>(*g, r, sf);
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

// ------------------------------------------------------------- collide + stream ----
// Each warp runs a loop over groups of cells (groups w, w + W, w + 2W, ... for warp w of W).
// Its records move HBM -> shared memory (cp.async, issued one group ahead) -> registers
// (one record per lane and chunk of 32) -> HBM, so the gather of the next group is in flight
// while the current group is computed.  Per-record work runs one lane per record; the
// per-cell sums run one or two lanes per cell over the velocities in shared memory.
constexpr int kPer = kMixCap / 32;  // records per lane

template <int NQ>
struct MixWarpStage {
  MixRec rec[kMixCap];      // landing zone of the next group's records (as stored in HBM)
  int2 q[NQ][kMixCap];      // fixed-point parts (h, lo) of each record's terms of the cell sums
  alignas(16) float cf[32][16];  // per cell: u (3), df | R[0..3] | R[4..7] | R[8], rotate flag, 2 unused
  uint8_t seg[kMixCap];     // cell of each record within the group
  int32_t bad[2][32];       // per cell: a momentum / energy term outside its fixed-point range
  Geom box[2];              // the box of the current / next group (copied with its records)
  BoxShift shift[2];
};

// A group's cells and records; lo / n describe the cell that this lane works on in the
// per-cell phases: lanes 4j .. 4j + 3 share cell j when the group has at most 8 cells, lanes
// 2j and 2j + 1 when it has at most 16, else lane j alone.
struct Span {
  int64_t c0;
  int box, ncells, lsh;
  int E0, E;  // first record (cell order), records
  int lo, n;  // this lane's cell: first record relative to E0, members
};

// Whether a group goes through the shared-memory stage.
__device__ __forceinline__ bool stages(const Span& sp) { return sp.E > 0 && sp.E <= kMixCap && sp.ncells <= 32; }

__device__ __forceinline__ MixGroup group_desc(const MixBatch& mb, int64_t gi) {
  if (gi < mb.ngroups) return mb.groups[gi];
  MixGroup d;
  d.c0 = 0;
  d.box = 0;
  d.ncells = 0;
  return d;
}

__device__ __forceinline__ Span group_span(const int32_t* __restrict__ offset, const MixGroup& d, int lane) {
  Span sp;
  sp.c0 = d.c0;
  sp.box = d.box;
  sp.ncells = d.ncells;
  sp.lsh = d.ncells <= 8 ? 2 : (d.ncells <= 16 ? 1 : 0);
  const int j = lane >> sp.lsh;
  const int ja = j < d.ncells ? j : d.ncells;
  const int jb = j < d.ncells ? j + 1 : d.ncells;
  const int a = offset[d.c0 + ja], bnd = offset[d.c0 + jb];
  sp.E0 = offset[d.c0];
  sp.E = offset[d.c0 + d.ncells] - sp.E0;
  sp.lo = a - sp.E0;
  sp.n = bnd - a;
  return sp;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(__cvta_generic_to_global(gmem)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Start copying a group's records (slots pm) and its box's constants into the stage.
template <typename Stage>
__device__ __forceinline__ void gather_async(Stage& st, const MixRec* __restrict__ src, const Span& sp, const int pm[kPer],
                                             const MixBatch& mb, int slot, int lane) {
  const int E = sp.E, box = sp.box;
  static_assert(sizeof(Geom) % 16 == 0 && sizeof(BoxShift) % 16 == 0, "16-byte pieces");
  constexpr int kGeomPieces = sizeof(Geom) / 16, kShiftPieces = sizeof(BoxShift) / 16;
  static_assert(kGeomPieces + kShiftPieces <= 32, "one piece per lane");
  if (lane < kGeomPieces)
    cp_async16(reinterpret_cast<float4*>(&st.box[slot]) + lane, reinterpret_cast<const float4*>(mb.boxes + box) + lane);
  else if (lane < kGeomPieces + kShiftPieces)
    cp_async16(reinterpret_cast<float4*>(&st.shift[slot]) + (lane - kGeomPieces),
               reinterpret_cast<const float4*>(mb.shifts + box) + (lane - kGeomPieces));
  if (stages(sp)) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = lane + 32 * i;
      if (e < E) {
        cp_async16(&st.rec[e], src + pm[i]);
        cp_async16(reinterpret_cast<float4*>(&st.rec[e]) + 1, reinterpret_cast<const float4*>(src + pm[i]) + 1);
      }
    }
  }
  cp_async_commit();
}

__device__ __forceinline__ void load_perm(const int32_t* __restrict__ perm, const Span& sp, int pm[kPer], int lane) {
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int e = lane + 32 * i;
    pm[i] = (stages(sp) && e < sp.E) ? perm[sp.E0 + e] : 0;
  }
}

// A staged record from shared memory.  Lanes with bit 2 set read the second 16-byte half
// first, so that the eight lanes of each quarter-warp cover all 32 banks (the 32-byte record
// stride would otherwise put lanes l and l + 4 on the same banks).
__device__ __forceinline__ MixRec lds_rec(const MixRec* p, int lane) {
  const float4* q = reinterpret_cast<const float4*>(p);
  const int h = (lane >> 2) & 1;
  const float4 x = q[h], y = q[h ^ 1];
  const float4 a = h ? y : x, b = h ? x : y;
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

// A group too large for the stage (more than kMixCap records or 32 cells): one lane per
// cell, in passes of 32 cells, records in place in the destination.
// (Arguments are plain values and pointers so that calling it stores nothing to the stack.)
template <int WALLS, int FORCE, int THERMO, int MOMENTS, int ANG = 0>
__device__ __noinline__ void collide_group_direct(const Geom* __restrict__ gp, const BoxShift* __restrict__ shp,
                                                  int64_t c0, int ncells, const int32_t* __restrict__ offset,
                                                  const int32_t* __restrict__ perm, double* moments,
                                                  const MixRec* __restrict__ src, MixRec* __restrict__ dst,
                                                  int32_t* __restrict__ knext, int32_t* __restrict__ cnext, int64_t t1,
                                                  int lane) {
  const Geom& g = *gp;
  const float sf[3] = {shp->sf_next[0], shp->sf_next[1], shp->sf_next[2]};
  const int cbase = static_cast<int>(g.cbase);
  for (int64_t c = c0 + lane; c < c0 + ncells; c += 32) {
    const int o = offset[c];
    const int n = offset[c + 1] - o;
    const int32_t* pm = perm + o;
    CellMoments cm;
    bool cm_ok = true;
    if (ANG) moments_zero(cm);
    for (int j = 0; j < n; ++j) {
      MixRec r = load_rec(src + pm[j]);
      stream_record<WALLS, FORCE>(g, r);
      dst[o + j] = r;
      if (ANG) cm_ok &= moments_add(cm, r, shp->sf);
    }
    mixed_collide_cell<WALLS, THERMO, MOMENTS, ANG>(g, dst + o, n, c - cbase, t1, shp->s[2],
                                                    MOMENTS ? moments + 5 * (int64_t)cbase : nullptr, shp->sf,
                                                    ANG ? &cm : nullptr, cm_ok);
    for (int j = 0; j < n; ++j) {
      const int k = cbase + next_key<WALLS, FORCE>(g, dst[o + j], sf);
      knext[o + j] = k;
      atomicAdd(&cnext[k], 1);
    }
  }
}

// Phase 1 of a staged group (lane = record): stream to r_t and split each velocity into the
// fixed-point parts of the momentum sums.  Returns the lane's records with a term out of
// range (bit i: chunk i).  All chunks run; records past the end repeat the last one and
// store nothing.
template <int WALLS, int FORCE, int NEAR, int MOMENTS, typename Stage>
__device__ __forceinline__ unsigned stream_split(const Geom& g, const Geom* __restrict__ gp, MixRec (&r)[kPer],
                                                 Stage& st, int E, int lane) {
  constexpr int NQ = 3 + MOMENTS;
  unsigned badm = 0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int e = lane + 32 * i;
    {
      const bool valid = e < E;
      if (NEAR)
        stream_record<WALLS, FORCE, 1>(g, r[i]);
      else
        r[i] = stream_record_general<WALLS, FORCE>(gp, r[i]);
      int h0, l0, h1, l1, h2, l2;
      bool o = fix_split<kFixV>(r[i].vx, h0, l0) & fix_split<kFixV>(r[i].vy, h1, l1) &
               fix_split<kFixV>(r[i].vz, h2, l2);
      if (valid) {
        st.q[0][e] = make_int2(h0, l0);
        st.q[1][e] = make_int2(h1, l1);
        st.q[2][e] = make_int2(h2, l2);
      }
      if (MOMENTS) {
        const float v2 = fmaf(r[i].vx, r[i].vx, fmaf(r[i].vy, r[i].vy, __fmul_rn(r[i].vz, r[i].vz)));
        o &= fix_split<kFixV2>(v2, h0, l0);
        if (valid) st.q[NQ - 1][e] = make_int2(h0, l0);
      }
      if (valid && !o) badm |= 1u << i;
    }
  }
  return badm;
}

// Phase 5 tail (lane = record): keys of the next step, counts, write-out in cell order.
template <int WALLS, int FORCE, int NEAR>
__device__ __forceinline__ void key_store(const Geom& g, const Geom* __restrict__ gp, const MixRec (&r)[kPer],
                                          const float sf[3], int E,
                                          MixRec* __restrict__ dst, int32_t* __restrict__ knext,
                                          int32_t* __restrict__ cnext, int cbase, int lane) {
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int e = lane + 32 * i;
    {
      const int k = cbase + (NEAR ? next_key<WALLS, FORCE, 1>(g, r[i], sf)
                                  : next_key_general<WALLS, FORCE>(gp, r[i], sf[0], sf[1], sf[2]));
      if (e < E) {
        store_rec(dst + e, r[i]);
        knext[e] = k;
        atomicAdd(&cnext[k], 1);
      }
    }
  }
}

// The per-cell random axis is keyed on the cell's index inside its box, so a box advanced in
// an ensemble reproduces the same box advanced alone; every per-cell sum is an exact integer,
// so neither the grouping nor the lanes per cell change any result.
// The collision of every group of a warp (gi, gi + W, ...), shared by the collide kernel and
// the one-launch step kernel: t1 is the step, cur the record buffer it starts from.
template <int WARPS, int WALLS, int FORCE, int THERMO, int MOMENTS>
__device__ __forceinline__ void collide_groups(const MixBatch& mb, const MixBufs& b, const MixScratch& s, int64_t t1,
                                               int cur, unsigned char* smem_raw) {
  constexpr int NQ = 3 + MOMENTS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  MixWarpStage<NQ>& st = reinterpret_cast<MixWarpStage<NQ>*>(smem_raw)[warp];
  const int64_t W = (int64_t)gridDim.x * WARPS;
  int64_t gi = (int64_t)blockIdx.x * WARPS + warp;
  if (gi >= mb.ngroups) return;
  const int nxt = cur ^ 1;
  const MixRec* __restrict__ src = b.rec[cur];
  MixRec* __restrict__ dst = b.rec[nxt];
  const int32_t* __restrict__ perm = s.perm;
  const int32_t* __restrict__ offset = s.offset;
  int32_t* __restrict__ knext = s.key[nxt];
  int32_t* __restrict__ cnext = s.count[nxt];

  // prologue: the first group's records into the stage, the second group's slots into registers
  Span sp = group_span(offset, group_desc(mb, gi), lane);
  int pm[kPer];
  load_perm(perm, sp, pm, lane);
  int slot = 0;  // stage slot of the current group's box constants
  gather_async(st, src, sp, pm, mb, slot, lane);
  Span sp1 = group_span(offset, group_desc(mb, gi + W), lane);
  load_perm(perm, sp1, pm, lane);
  cp_async_wait_all();
  __syncwarp();

  for (;;) {
    const bool staged = stages(sp);  // empty and oversized groups take the per-cell path
    MixRec r[kPer];
    if (staged) {
      // every lane takes kPer records; those past the end of the group repeat the last one,
      // so all chunks run without branches and only their stores are predicated
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int e = lane + 32 * i;
        r[i] = lds_rec(&st.rec[e < sp.E ? e : sp.E - 1], lane);
      }
    }
    __syncwarp();
    gather_async(st, src, sp1, pm, mb, slot ^ 1, lane);  // group k + 1: HBM -> stage
    const MixGroup d2 = group_desc(mb, gi + 2 * W);       // group k + 2: descriptor
    Span sp2;
    if (!staged) {
      collide_group_direct<WALLS, FORCE, THERMO, MOMENTS>(mb.boxes + sp.box, mb.shifts + sp.box, sp.c0, sp.ncells,
                                                          offset, perm, s.moments, src, dst, knext, cnext, t1, lane);
      sp2 = group_span(offset, d2, lane);
      load_perm(perm, sp2, pm, lane);
    } else {
      const Geom* gbox = mb.boxes + sp.box;
      const Geom g = st.box[slot];  // a register copy: the stores below cannot alias it
      const BoxShift& sh = st.shift[slot];
      const float sf[3] = {sh.sf_next[0], sh.sf_next[1], sh.sf_next[2]};  // grid of the next step
      const double shz = sh.s[2];                                        // grid of this step
      const int cbase = static_cast<int>(g.cbase);
      const int E = sp.E, E0 = sp.E0;
      const int lsh = sp.lsh, j = lane >> lsh, p = lane & ((1 << lsh) - 1), step = 1 << lsh;
      const bool cl_live = j < sp.ncells;
      const int lo = sp.lo, n = sp.n;
      const int64_t cl = sp.c0 + j - cbase;  // cell index inside the box

      // 1. stream to r_t and split the velocities into fixed-point parts (lane = record);
      //    tag records with their cell and draw the rotation (lane = cell)
      bool near = true;
#pragma unroll
      for (int i = 0; i < kPer; ++i)
        near = near & moves_near<FORCE>(g, r[i]) & (!WALLS || stays_inside(g, r[i]));
      unsigned badm = __all_sync(0xffffffffu, near) ? stream_split<WALLS, FORCE, 1, MOMENTS>(g, gbox, r, st, E, lane)
                                                     : stream_split<WALLS, FORCE, 0, MOMENTS>(g, gbox, r, st, E, lane);
      for (int k = p; k < n; k += step) st.seg[lo + k] = static_cast<uint8_t>(j);
      st.bad[0][j] = 0;
      st.bad[1][j] = 0;
      float R8 = 0.0f;  // kept for the per-cell record written after the sums
      if (cl_live && p == 0 && n >= 1) {
        float R[9];
        frame_f32(g, t1, cl, R);
        float4* q = reinterpret_cast<float4*>(st.cf[j]);
        q[1] = make_float4(R[0], R[1], R[2], R[3]);
        q[2] = make_float4(R[4], R[5], R[6], R[7]);
        R8 = R[8];
      }
      sp2 = group_span(offset, d2, lane);  // group k + 2: record range
      __syncwarp();
      if (__any_sync(0xffffffffu, badm != 0u)) {  // rare: mark the cells of out-of-range terms
#pragma unroll
        for (int i = 0; i < kPer; ++i)
          if ((badm >> i) & 1u) st.bad[0][st.seg[lane + 32 * i]] = 1;
        __syncwarp();
      }
      // 2. per cell: exact momentum sums, centre-of-mass velocity, whether the cell rotates
      long long S[3], E2 = 0;
      {
        int hs[NQ], ls[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) hs[c] = ls[c] = 0;
        for (int k = p; k < n; k += step) {
#pragma unroll
          for (int c = 0; c < NQ; ++c) {
            const int2 v = st.q[c][lo + k];
            hs[c] += v.x;
            ls[c] += v.y;
          }
        }
        for (int m = 1; m < step; m <<= 1) {  // warp-uniform: lsh is the group's
#pragma unroll
          for (int c = 0; c < NQ; ++c) {
            hs[c] += __shfl_xor_sync(0xffffffffu, hs[c], m);
            ls[c] += __shfl_xor_sync(0xffffffffu, ls[c], m);
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) S[c] = fix_join(hs[c], ls[c]);
        if (MOMENTS) E2 = fix_join(hs[NQ - 1], ls[NQ - 1]);
      }
      if (cl_live && p == 0) {
        const bool ok = st.bad[0][j] == 0;
        if (MOMENTS) write_moments_mixed(g, s.moments, sp.c0 + j, n, S, E2);
        CellFrame f;
        cell_prologue_u<WALLS>(g, S, n, cl, t1, shz, f);
        float4* q = reinterpret_cast<float4*>(st.cf[j]);
        q[0] = make_float4(f.u[0], f.u[1], f.u[2], 0.0f);
        q[3] = make_float4(R8, (f.rot && ok) ? 1.0f : 0.0f, 0.0f, 0.0f);
      }
      __syncwarp();
      // 3. rotate (lane = record): w = R (v - u), and the fixed-point parts of the energy terms
      badm = 0;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int e = lane + 32 * i;
        {
          const bool valid = e < E;
          const float4* q = reinterpret_cast<const float4*>(st.cf[st.seg[valid ? e : E - 1]]);
          const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
          const bool rot = q3.y != 0.0f;
          CellFrame f;
          f.u[0] = q0.x;
          f.u[1] = q0.y;
          f.u[2] = q0.z;
          f.R[0] = q1.x;
          f.R[1] = q1.y;
          f.R[2] = q1.z;
          f.R[3] = q1.w;
          f.R[4] = q2.x;
          f.R[5] = q2.y;
          f.R[6] = q2.z;
          f.R[7] = q2.w;
          f.R[8] = q3.x;
          float w[3] = {r[i].vx, r[i].vy, r[i].vz};
          const float term = rotate_relative(f, w);
          r[i].vx = rot ? w[0] : r[i].vx;
          r[i].vy = rot ? w[1] : r[i].vy;
          r[i].vz = rot ? w[2] : r[i].vz;
          int h0, l0, h1, l1;
          const bool o = fix_split<kFixDE>(term, h0, l0) & fix_split<kFixV2>(sq3(w), h1, l1);
          if (valid && rot) {
            st.q[0][e] = make_int2(h0, l0);
            st.q[1][e] = make_int2(h1, l1);
            if (!o) badm |= 1u << i;
          }
        }
      }
      load_perm(perm, sp2, pm, lane);  // group k + 2: slots
      __syncwarp();
      if (__any_sync(0xffffffffu, badm != 0u)) {
#pragma unroll
        for (int i = 0; i < kPer; ++i)
          if ((badm >> i) & 1u) st.bad[1][st.seg[lane + 32 * i]] = 1;
        __syncwarp();
      }
      // 4. per cell: exact energy sums, scale factor
      {
        const bool rot = cl_live && st.cf[j][13] != 0.0f;
        int hd = 0, ld = 0, ha = 0, la = 0;
        if (rot)
          for (int k = p; k < n; k += step) {
            const int2 d = st.q[0][lo + k], a = st.q[1][lo + k];
            hd += d.x;
            ld += d.y;
            ha += a.x;
            la += a.y;
          }
        for (int m = 1; m < step; m <<= 1) {
          hd += __shfl_xor_sync(0xffffffffu, hd, m);
          ld += __shfl_xor_sync(0xffffffffu, ld, m);
          ha += __shfl_xor_sync(0xffffffffu, ha, m);
          la += __shfl_xor_sync(0xffffffffu, la, m);
        }
        if (rot && p == 0)
          st.cf[j][3] = cell_df<THERMO>(g, n, fix_join(hd, ld), fix_join(ha, la), st.bad[1][j] == 0, t1, cl);
      }
      __syncwarp();
      // 5. new velocities; keys and counts of the next step; write-out in cell order
      near = true;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int e = lane + 32 * i;
        {
          const float* cf = st.cf[st.seg[e < E ? e : E - 1]];
          const float4 q0 = *reinterpret_cast<const float4*>(cf);
          const bool rot = cf[13] != 0.0f;
          const float df = q0.w;
          const float nx = __fadd_rn(q0.x, fmaf(df, r[i].vx, r[i].vx));
          const float ny = __fadd_rn(q0.y, fmaf(df, r[i].vy, r[i].vy));
          const float nz = __fadd_rn(q0.z, fmaf(df, r[i].vz, r[i].vz));
          r[i].vx = rot ? nx : r[i].vx;
          r[i].vy = rot ? ny : r[i].vy;
          r[i].vz = rot ? nz : r[i].vz;
          near = near & moves_near<FORCE>(g, r[i]) & (!WALLS || stays_inside(g, r[i]));
        }
      }
      if (__all_sync(0xffffffffu, near))
        key_store<WALLS, FORCE, 1>(g, gbox, r, sf, E, dst + E0, knext + E0, cnext, cbase, lane);
      else
        key_store<WALLS, FORCE, 0>(g, gbox, r, sf, E, dst + E0, knext + E0, cnext, cbase, lane);
    }
    cp_async_wait_all();  // group k + 1 has landed
    __syncwarp();
    gi += W;
    if (gi >= mb.ngroups) break;
    slot ^= 1;
    sp = sp1;
    sp1 = sp2;
  }
}

template <int WARPS, int WALLS, int FORCE, int THERMO, int MOMENTS>
__global__ void __launch_bounds__(WARPS * 32, 12 / WARPS) k_collide_stream_mixed(MixBatch mb, MixBufs b, MixScratch s,
                                                                    Ctl* __restrict__ ctl) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  collide_groups<WARPS, WALLS, FORCE, THERMO, MOMENTS>(mb, b, s, ctl->t + 1, ctl->cur, smem_raw);
}

// perm[offset[key] + rank] = slot, the rank from a per-cell cursor.  Neighbouring slots mostly
// share a key, so each warp groups equal keys (match.any) and one lane per group takes the
// group's ranks with a single atomic.  The order inside a cell is whatever the atomics give;
// every per-cell sum downstream is exact, so it does not matter.  A warp takes 8 chunks of
// 32 consecutive slots per iteration, so that eight load-atomic-store chains are in flight.
__global__ void __launch_bounds__(kThreads) k_scatter_cursor(int64_t n, const int32_t* __restrict__ key,
                                                             const int32_t* __restrict__ offset, int32_t* __restrict__ cursor,
                                                             int32_t* __restrict__ perm) {
  constexpr int kChunks = 8;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 * kChunks); base < n;
       base += warps * 32 * kChunks) {  // warp-uniform
    int k[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const int64_t i = base + 32 * c + lane;
      k[c] = i < n ? key[i] : -1 - lane;  // distinct sentinels: lanes past the end stay alone
    }
    unsigned peers[kChunks];
    int rank[kChunks], first[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      peers[c] = __match_any_sync(0xffffffffu, k[c]);
      rank[c] = __popc(peers[c] & below);
      first[c] = 0;
      if (k[c] >= 0 && rank[c] == 0) first[c] = atomicAdd(&cursor[k[c]], __popc(peers[c]));
    }
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const int start = __shfl_sync(0xffffffffu, first[c], __ffs(peers[c]) - 1);
      const int64_t i = base + 32 * c + lane;
      if (k[c] >= 0) perm[offset[k[c]] + start + rank[c]] = static_cast<int32_t>(i);
    }
  }
}

// First cell c in [lo, hi] with offset[c] >= rec (offset[hi] is the box's end).
__device__ __forceinline__ int64_t first_cell(const int32_t* __restrict__ offset, int64_t lo, int64_t hi, int64_t rec) {
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (offset[mid] >= rec)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// Group g of a box starts at the first cell whose records start at or after its rec0, and
// ends where the next group starts (the last one at the box's end): the groups tile the box
// and each holds about the target number of records, within one cell's worth.
__global__ void __launch_bounds__(kThreads) k_group_bounds(int64_t ngroups, const Geom* __restrict__ boxes,
                                                           const MixGroupSpec* __restrict__ spec,
                                                           const int32_t* __restrict__ offset,
                                                           MixGroup* __restrict__ groups) {
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < ngroups; gi += (int64_t)gridDim.x * blockDim.x) {
    const MixGroupSpec q = spec[gi];
    const int64_t cb = boxes[q.box].cbase, ce = cb + boxes[q.box].ncell;
    const int64_t c0 = first_cell(offset, cb, ce, q.rec0);
    const int64_t c1 = q.rec1 < 0 ? ce : first_cell(offset, cb, ce, q.rec1);
    MixGroup d;
    d.c0 = c0;
    d.box = q.box;
    d.ncells = static_cast<int32_t>(c1 - c0);
    groups[gi] = d;
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

// ---- one persistent launch per step (the mixed form's staged path; ensembles included) ----
// Every phase of a step in one cooperative launch of the persistent collide grid, the phases
// separated by grid-wide barriers: (1) zero the next step's counts and the scatter cursors,
// sum this step's counts per tile; (2) block 0 scans the tile sums; (3) the offsets inside
// each tile; (4) the scatter (perm from the cursors) and the group table; (5) the collision
// (collide_groups); (6) the last block to finish ends the step.  A cooperative launch has all
// blocks resident, so every barrier is reached; each wait is still bounded: a block that
// waits longer than about a second sets the control block's error flag and returns, and
// every block that sees the flag returns too, so a failed step ends with an error that the
// host reads (MPCD_ERR_TIMEOUT) instead of a hang.
constexpr int kStepScanItems = 8;
constexpr unsigned kBarrierSpins = 1u << 22;  // polls of about 0.25 us each

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on bar[0]: returns false (every thread of the block) if the wait ran out or
// another block had already given up.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    for (unsigned spin = 0;; ++spin) {
      if (ld_acquire_u32(bar) >= target) break;
      if (*reinterpret_cast<volatile int*>(err) != 0 || spin >= kBarrierSpins) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum over the block (every thread gets it); red holds one int per warp.
template <int NT>
__device__ __forceinline__ int block_sum_i32(int v, int* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int t = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// Exclusive scan over the block; *total receives the block's sum.
template <int NT>
__device__ __forceinline__ int block_scan_i32(int v, int* red, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) red[wid] = incl;
  __syncthreads();
  int before = 0, t = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    if (w < wid) before += red[w];
    t += red[w];
  }
  __syncthreads();
  *total = t;
  return before + incl - v;
}

struct StepAux {
  const MixGroupSpec* spec;  // the fixed part of the group table
  MixGroup* groups;          // rewritten in phase 4 (mb.groups points at the same table)
  unsigned* bar;             // [2]: barrier arrivals, blocks finished; both 0 between steps
  int stall;                 // test hook: block 0 leaves without arriving at any barrier
};

template <int WARPS, int WALLS, int FORCE, int THERMO, int MOMENTS>
__global__ void __launch_bounds__(WARPS * 32, 12 / WARPS) k_step_mixed(MixBatch mb, MixBufs b, MixScratch s,
                                                                 Ctl* __restrict__ ctl, StepAux aux) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NT = WARPS * 32;
  constexpr int kTileCells = NT * kStepScanItems;
  __shared__ int red[NT / 32];
  __shared__ int s_last;
  if (aux.stall && blockIdx.x == 0) return;
  const int64_t t1 = ctl->t + 1;
  const int cur = ctl->cur, nxt = cur ^ 1;
  const int64_t C = mb.ncell;
  const int64_t tiles = (C + kTileCells - 1) / kTileCells;
  const int64_t gthreads = (int64_t)gridDim.x * NT, gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
  int* err = &ctl->err;
  unsigned gen = 0;

  // 1. next step's counts and the cursors to zero; this step's counts summed per tile
  for (int64_t i = gtid; i < C; i += gthreads) {
    s.count[nxt][i] = 0;
    s.cursor[i] = 0;
  }
  for (int64_t tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
    int v = 0;
#pragma unroll
    for (int k = 0; k < kStepScanItems; ++k) {
      const int64_t i = tl * kTileCells + k * NT + threadIdx.x;
      if (i < C) v += s.count[cur][i];
    }
    v = block_sum_i32<NT>(v, red);
    if (threadIdx.x == 0) s.partial[tl] = v;
  }
  if (!grid_barrier(aux.bar, ++gen * gridDim.x, err)) return;

  // 2. block 0: exclusive scan of the tile sums, in place; the total closes the offsets
  if (blockIdx.x == 0) {
    int carry = 0;
    for (int64_t base = 0; base < tiles; base += NT) {
      const int64_t i = base + threadIdx.x;
      const int v = i < tiles ? s.partial[i] : 0;
      int total;
      const int ex = block_scan_i32<NT>(v, red, &total);
      if (i < tiles) s.partial[i] = carry + ex;
      carry += total;
    }
    if (threadIdx.x == 0) s.offset[C] = carry;
  }
  if (!grid_barrier(aux.bar, ++gen * gridDim.x, err)) return;

  // 3. offsets inside each tile (thread = kStepScanItems consecutive cells)
  for (int64_t tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
    const int64_t i0 = tl * kTileCells + (int64_t)threadIdx.x * kStepScanItems;
    int vals[kStepScanItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kStepScanItems; ++k) {
      vals[k] = i0 + k < C ? s.count[cur][i0 + k] : 0;
      sum += vals[k];
    }
    int total;
    int run = block_scan_i32<NT>(sum, red, &total) + s.partial[tl];
#pragma unroll
    for (int k = 0; k < kStepScanItems; ++k) {
      if (i0 + k < C) s.offset[i0 + k] = run;
      run += vals[k];
    }
  }
  if (!grid_barrier(aux.bar, ++gen * gridDim.x, err)) return;

  // 4. perm from the cursors (equal keys of a warp take their places with one atomic), and
  //    the cell boundaries of every group
  {
    constexpr int kChunks = 8;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int64_t warps = (int64_t)gridDim.x * WARPS;
    const int32_t* __restrict__ key = s.key[cur];
    for (int64_t base = ((int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5)) * (32 * kChunks); base < mb.n;
         base += warps * 32 * kChunks) {
      int k[kChunks], first[kChunks], rank[kChunks];
      unsigned peers[kChunks];
#pragma unroll
      for (int c = 0; c < kChunks; ++c) {
        const int64_t i = base + 32 * c + lane;
        k[c] = i < mb.n ? key[i] : -1 - lane;
      }
#pragma unroll
      for (int c = 0; c < kChunks; ++c) {
        peers[c] = __match_any_sync(0xffffffffu, k[c]);
        rank[c] = __popc(peers[c] & below);
        first[c] = 0;
        if (k[c] >= 0 && rank[c] == 0) first[c] = atomicAdd(&s.cursor[k[c]], __popc(peers[c]));
      }
#pragma unroll
      for (int c = 0; c < kChunks; ++c) {
        const int start = __shfl_sync(0xffffffffu, first[c], __ffs(peers[c]) - 1);
        const int64_t i = base + 32 * c + lane;
        if (k[c] >= 0) s.perm[s.offset[k[c]] + start + rank[c]] = static_cast<int32_t>(i);
      }
    }
    for (int64_t gi = gtid; gi < mb.ngroups; gi += gthreads) {
      const MixGroupSpec q = aux.spec[gi];
      const int64_t cb = mb.boxes[q.box].cbase, ce = cb + mb.boxes[q.box].ncell;
      MixGroup d;
      d.c0 = first_cell(s.offset, cb, ce, q.rec0);
      d.box = q.box;
      d.ncells = static_cast<int32_t>((q.rec1 < 0 ? ce : first_cell(s.offset, cb, ce, q.rec1)) - d.c0);
      aux.groups[gi] = d;
    }
  }
  if (!grid_barrier(aux.bar, ++gen * gridDim.x, err)) return;

  // 5. the collision of this block's groups
  collide_groups<WARPS, WALLS, FORCE, THERMO, MOMENTS>(mb, b, s, t1, cur, smem_raw);

  // 6. the last block to finish advances the step (shifts of every box, step counter, buffer)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(aux.bar + 1, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int bx = threadIdx.x; bx < mb.nbox; bx += NT) {
    BoxShift& sh = mb.shifts[bx];
    for (int d = 0; d < 3; ++d) sh.s_last[d] = sh.s[d];
    box_shifts(mb.boxes[bx], t1, sh);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->t = t1;
    ctl->cur = nxt;
    aux.bar[0] = 0u;  // every block has left its last barrier
    aux.bar[1] = 0u;
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
    if (!(fl >= 0.0 && fl < static_cast<double>(g.L[d]))) {
      // outside the box (the state entry points reject such input): fold into range, so
      // that no cell index can leave the key space
      const double Ld = static_cast<double>(g.L[d]);
      fl = (fl == fl && fabs(fl) < 9.0e15) ? fl - Ld * floor(fl / Ld) : 0.0;
      if (!(fl >= 0.0 && fl < Ld)) fl = 0.0;
      if (!(x >= 0.0f && x < 1.0f)) x = 0.0f;
    }
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

// Validation of a state on the device: the smallest index i with a position outside
// [0, B_d) of its box or a non-finite velocity goes to *bad (left as is when all are valid).
__device__ __forceinline__ bool state_ok(const double* r, const double* v, const double B[3]) {
  bool ok = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) ok = ok && r[d] >= 0.0 && r[d] < B[d] && isfinite(v[d]);
  return ok;
}

__global__ void __launch_bounds__(kThreads) k_check_state_batch(MixBatch mb, const double* __restrict__ r,
                                                                const double* __restrict__ v,
                                                                unsigned long long* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mb.n; i += (int64_t)gridDim.x * blockDim.x)
    if (!state_ok(r + 3 * i, v + 3 * i, mb.boxes[box_of(mb.pbase, mb.nbox, i)].B))
      atomicMin(bad, static_cast<unsigned long long>(i));
}

__global__ void __launch_bounds__(kThreads) k_check_state_box(int64_t n, Geom g, const double* __restrict__ r,
                                                              const double* __restrict__ v,
                                                              unsigned long long* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!state_ok(r + 3 * i, v + 3 * i, g.B)) atomicMin(bad, static_cast<unsigned long long>(i));
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
// Masses (by particle id, FP64) into the storage order of a record buffer, rounded to FP32.
__global__ void __launch_bounds__(kThreads) k_gather_masses_mixed(int64_t n, const MixRec* __restrict__ rec,
                                                                  const double* __restrict__ m_by_id,
                                                                  float* __restrict__ dst) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = __double2float_rn(m_by_id[rec[j].id]);
}

// v += dp / m for every record (dp by particle id); the FP32 velocity becomes the FP32
// rounding of the FP64 sum.
__global__ void __launch_bounds__(kThreads) k_add_momentum_mixed(MixBatch mb, MixRec* __restrict__ rec,
                                                                 const float* __restrict__ m,
                                                                 const double* __restrict__ dp) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < mb.n; j += (int64_t)gridDim.x * blockDim.x) {
    MixRec r = load_rec(rec + j);
    const int64_t i = r.id;
    const double mi = m ? static_cast<double>(m[j]) : mb.boxes[box_of(mb.pbase, mb.nbox, i)].mass;
    r.vx = __double2float_rn(static_cast<double>(r.vx) + dp[3 * i] / mi);
    r.vy = __double2float_rn(static_cast<double>(r.vy) + dp[3 * i + 1] / mi);
    r.vz = __double2float_rn(static_cast<double>(r.vz) + dp[3 * i + 2] / mi);
    store_rec(rec + j, r);
  }
}

}  // namespace

void launch_gather_masses_mixed(int64_t n, const MixRec* rec, const double* m_by_id, float* dst, cudaStream_t st) {
  if (n > 0) k_gather_masses_mixed<<<grid_for(n), kThreads, 0, st>>>(n, rec, m_by_id, dst);
}

void launch_add_momentum_mixed(const MixBatch& mb, MixBufs b, int cur, MixMass ms, const double* dp, cudaStream_t st) {
  if (mb.n > 0) k_add_momentum_mixed<<<grid_for(mb.n), kThreads, 0, st>>>(mb, b.rec[cur], ms.m[cur], dp);
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

namespace {
// prepare: raise the kernel's dynamic shared-memory limit on the current device and record
// how many of its blocks are resident at once (the persistent grid); runs outside capture.
template <int WARPS, int WALLS, int FORCE, int THERMO, int MOMENTS>
cudaError_t launch_collide_t(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, cudaStream_t st, bool prepare) {
  auto kern = k_collide_stream_mixed<WARPS, WALLS, FORCE, THERMO, MOMENTS>;
  const int smem = WARPS * static_cast<int>(sizeof(MixWarpStage<3 + MOMENTS>));
  static int resident = 0;
  if (prepare) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) resident = per_sm * sms;
    return e;
  }
  int64_t grid = (mb.ngroups + WARPS - 1) / WARPS;
  if (grid == 0) return cudaSuccess;
  if (resident > 0 && grid > resident) grid = resident;
  kern<<<static_cast<unsigned>(grid), WARPS * 32, smem, st>>>(mb, b, s, ctl);
  return cudaSuccess;
}

// A group of at most kMixCap records with angular-momentum conservation: the warp gathers and
// streams the records into its stage st (lane = record), each lane collides its cells there
// (lane = cell; the same per-cell arithmetic and member order as collide_group_direct, so the
// same results), and the warp writes them out in cell order with the next step's keys.
template <int FORCE, int THERMO, int MOMENTS>
__device__ __noinline__ void collide_group_staged_ang(const Geom* __restrict__ gp, const BoxShift* __restrict__ shp,
                                                      int64_t c0, int ncells, int E0, int E,
                                                      const int32_t* __restrict__ offset,
                                                      const int32_t* __restrict__ perm, double* moments,
                                                      const MixRec* __restrict__ src, MixRec* __restrict__ dst,
                                                      int32_t* __restrict__ knext, int32_t* __restrict__ cnext,
                                                      int64_t t1, int lane, MixRec* st) {
  const Geom& g = *gp;
  const float sf[3] = {shp->sf_next[0], shp->sf_next[1], shp->sf_next[2]};
  const int cbase = static_cast<int>(g.cbase);
  for (int e = lane; e < E; e += 32) {
    MixRec r = load_rec(src + perm[E0 + e]);
    stream_record<0, FORCE>(g, r);
    st[e] = r;
  }
  __syncwarp();
  for (int64_t c = c0 + lane; c < c0 + ncells; c += 32) {
    const int o = offset[c] - E0;
    const int n = offset[c + 1] - offset[c];
    CellMoments cm;
    moments_zero(cm);
    bool ok = true;
    for (int j = 0; j < n; ++j) ok &= moments_add(cm, st[o + j], shp->sf);
    mixed_collide_cell<0, THERMO, MOMENTS, 1>(g, st + o, n, c - cbase, t1, shp->s[2],
                                              MOMENTS ? moments + 5 * (int64_t)cbase : nullptr, shp->sf, &cm, ok);
  }
  __syncwarp();
  for (int e = lane; e < E; e += 32) {
    const MixRec r = st[e];
    store_rec(dst + E0 + e, r);
    const int k = cbase + next_key<0, FORCE>(g, r, sf);
    knext[E0 + e] = k;
    atomicAdd(&cnext[k], 1);
  }
  __syncwarp();  // the stage is reused by the warp's next group
}

// Angular-momentum-conserving collision: a warp per group, only these paths compiled with the
// correction, so the staged kernel's code is untouched.  Groups of at most kMixCap records
// are staged in shared memory; larger ones go through collide_group_direct.  Periodic boxes
// only.
template <int FORCE, int THERMO, int MOMENTS>
__global__ void __launch_bounds__(128) k_collide_direct_mixed(MixBatch mb, MixBufs b, MixScratch s,
                                                              Ctl* __restrict__ ctl) {
  __shared__ MixRec stage[4][kMixCap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int64_t t1 = ctl->t + 1;
  const int cur = ctl->cur, nxt = cur ^ 1;
  for (int64_t gi = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; gi < mb.ngroups; gi += warps) {
    const MixGroup d = mb.groups[gi];
    const int E0 = s.offset[d.c0], E = s.offset[d.c0 + d.ncells] - E0;
    if (E <= kMixCap)
      collide_group_staged_ang<FORCE, THERMO, MOMENTS>(mb.boxes + d.box, mb.shifts + d.box, d.c0, d.ncells, E0, E,
                                                       s.offset, s.perm, s.moments, b.rec[cur], b.rec[nxt],
                                                       s.key[nxt], s.count[nxt], t1, lane, stage[warp]);
    else
      collide_group_direct<0, FORCE, THERMO, MOMENTS, 1>(mb.boxes + d.box, mb.shifts + d.box, d.c0, d.ncells,
                                                         s.offset, s.perm, s.moments, b.rec[cur], b.rec[nxt],
                                                         s.key[nxt], s.count[nxt], t1, lane);
  }
}

// ---- per-particle masses in the mixed form (Listing 4 sums m v and m; reading R24) ----
// The masses are FP32 values in storage order beside the records (two buffer sets, moved with
// them).  Each product m_j v_j is rounded once in FP32 and summed exactly on the fixed-point
// grids, as are the m_j, so the member order does not matter: P = sum m v, M = sum m,
// u = P / M (with the virtual wall particles of a cut cell, which keep the box mass), and
// the energy-restoring rescale and the thermostats weight each member's terms by m_j.
template <int THERMO>
__device__ __forceinline__ float cell_df_mass(const Geom& g, int n, long long dE, long long Ea, bool ok, int64_t t1,
                                              int64_t cell) {
  if (!ok || Ea <= 0) return 0.0f;
  const float ea = ll_to_float(Ea) * 0x1.0p-30f;  // sum m |w|^2
  if (THERMO && n >= 2) {
    const float dof = THERMO == 2 ? 2.0f * mbs_gamma_f32(g.seed, t1, cell, 1.5f * static_cast<float>(n - 1))
                                  : 3.0f * static_cast<float>(n - 1);
    return sqrtf(dof * g.kTf / ea) - 1.0f;
  }
  return 0.5f * (ll_to_float(dE) * 0x1.0p-44f) / ea;
}

template <int WALLS, int THERMO, int MOMENTS>
__device__ void mixed_collide_cell_mass(const Geom& g, MixRec* rec, const float* __restrict__ m, int n, int64_t c,
                                        int64_t t1, double shift_z, double* moments) {
  long long P[3] = {0, 0, 0}, M = 0, E2 = 0;
  bool ok = n < 8192;
  for (int j = 0; j < n; ++j) {
    const float mj = m[j], a = rec[j].vx, b = rec[j].vy, cz = rec[j].vz;
    ok &= fx_add<kFixV>(P[0], __fmul_rn(mj, a)) & fx_add<kFixV>(P[1], __fmul_rn(mj, b)) &
          fx_add<kFixV>(P[2], __fmul_rn(mj, cz)) & fx_add<kFixV>(M, mj);
    if (MOMENTS) ok &= fx_add<kFixV2>(E2, __fmul_rn(mj, fmaf(a, a, fmaf(b, b, __fmul_rn(cz, cz)))));
  }
  if (MOMENTS) {
    double* mo = moments + 5 * c;
    mo[0] = __ll2double_rn(M) * 0x1.0p-32;
    mo[1] = __ll2double_rn(P[0]) * 0x1.0p-32;
    mo[2] = __ll2double_rn(P[1]) * 0x1.0p-32;
    mo[3] = __ll2double_rn(P[2]) * 0x1.0p-32;
    mo[4] = 0.5 * __ll2double_rn(E2) * 0x1.0p-30;
  }
  if (n == 0 || M <= 0) return;
  CellFrame f;
  f.df = 0.0f;
  const float Mf = ll_to_float(M);
  f.u[0] = ll_to_float(P[0]) / Mf;
  f.u[1] = ll_to_float(P[1]) / Mf;
  f.u[2] = ll_to_float(P[2]) / Mf;
  bool virt = false;
  if (WALLS) {
    const int64_t layer = c / ((int64_t)g.L[0] * g.L[1]);
    if (shift_z > 0.0 && (layer == 0 || layer == g.L[2]) && (double)n < g.ppc) {
      // R13: virtual particles of the box mass fill the cut cell to ppc (FP64, wall cells only)
      const double Mv = (g.ppc - (double)n) * g.mass;
      const u64x4 w = draw(g.seed, static_cast<uint64_t>(t1), static_cast<uint64_t>(c), kTagWall);
      double g0, g1, g2, g3;
      gauss_pair(w.x, w.y, g0, g1);
      gauss_pair(w.z, w.w, g2, g3);
      const double sd = sqrt(Mv * g.kT);
      const double Mt = __ll2double_rn(M) * 0x1.0p-32 + Mv;
      f.u[0] = static_cast<float>((__ll2double_rn(P[0]) * 0x1.0p-32 + sd * g0) / Mt);
      f.u[1] = static_cast<float>((__ll2double_rn(P[1]) * 0x1.0p-32 + sd * g1) / Mt);
      f.u[2] = static_cast<float>((__ll2double_rn(P[2]) * 0x1.0p-32 + sd * g2) / Mt);
      virt = true;
    }
  }
  if (!(n >= 2 || virt) || !ok) return;
  frame_f32(g, t1, c, f.R);
  long long dE = 0, Ea = 0;
  bool oke = n < 512;
  for (int j = 0; j < n; ++j) {
    float w[3] = {rec[j].vx, rec[j].vy, rec[j].vz};
    const float term = rotate_relative(f, w);
    rec[j].vx = w[0];
    rec[j].vy = w[1];
    rec[j].vz = w[2];
    oke &= fx_add<kFixDE>(dE, __fmul_rn(m[j], term)) & fx_add<kFixV2>(Ea, __fmul_rn(m[j], sq3(w)));
  }
  const float df = cell_df_mass<THERMO>(g, n, dE, Ea, oke, t1, c);
  for (int j = 0; j < n; ++j) {
    rec[j].vx = __fadd_rn(f.u[0], fmaf(df, rec[j].vx, rec[j].vx));
    rec[j].vy = __fadd_rn(f.u[1], fmaf(df, rec[j].vy, rec[j].vy));
    rec[j].vz = __fadd_rn(f.u[2], fmaf(df, rec[j].vz, rec[j].vz));
  }
}

// A warp per group of cells, a lane per cell: each cell's records and masses are gathered
// through perm, streamed and written in cell order to the other buffer set, collided there
// with their masses, and given the next step's keys and counts (as collide_group_direct).
template <int WALLS, int FORCE, int THERMO, int MOMENTS>
__global__ void __launch_bounds__(128) k_collide_mass_mixed(MixBatch mb, MixBufs b, MixScratch s, Ctl* __restrict__ ctl,
                                                            MixMass ms) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int64_t t1 = ctl->t + 1;
  const int cur = ctl->cur, nxt = cur ^ 1;
  const MixRec* __restrict__ src = b.rec[cur];
  MixRec* __restrict__ dst = b.rec[nxt];
  const float* __restrict__ msrc = ms.m[cur];
  float* __restrict__ mdst = ms.m[nxt];
  for (int64_t gi = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; gi < mb.ngroups; gi += warps) {
    const MixGroup d = mb.groups[gi];
    const Geom& g = mb.boxes[d.box];
    const BoxShift* shp = mb.shifts + d.box;
    const float sf[3] = {shp->sf_next[0], shp->sf_next[1], shp->sf_next[2]};
    const int cbase = static_cast<int>(g.cbase);
    for (int64_t c = d.c0 + lane; c < d.c0 + d.ncells; c += 32) {
      const int o = s.offset[c];
      const int n = s.offset[c + 1] - o;
      const int32_t* pm = s.perm + o;
      for (int j = 0; j < n; ++j) {
        MixRec r = load_rec(src + pm[j]);
        stream_record<WALLS, FORCE>(g, r);
        dst[o + j] = r;
        mdst[o + j] = msrc[pm[j]];
      }
      mixed_collide_cell_mass<WALLS, THERMO, MOMENTS>(g, dst + o, mdst + o, n, c - cbase, t1, shp->s[2],
                                                      MOMENTS ? s.moments + 5 * (int64_t)cbase : nullptr);
      for (int j = 0; j < n; ++j) {
        const int k = cbase + next_key<WALLS, FORCE>(g, dst[o + j], sf);
        s.key[nxt][o + j] = k;
        atomicAdd(&s.count[nxt][k], 1);
      }
    }
  }
}

template <int WALLS, int FORCE, int THERMO, int MOMENTS>
void launch_mass_t(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, MixMass ms, cudaStream_t st) {
  int64_t grid = (static_cast<int64_t>(mb.ngroups) + 3) / 4;
  if (grid == 0) return;
  if (grid > 152 * 16) grid = 152 * 16;
  k_collide_mass_mixed<WALLS, FORCE, THERMO, MOMENTS><<<static_cast<unsigned>(grid), 128, 0, st>>>(mb, b, s, ctl, ms);
}

template <int WALLS, int FORCE>
void launch_mass_wf(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, MixMass ms, bool moments, cudaStream_t st) {
  switch (2 * mb.thermostat + (moments ? 1 : 0)) {
    case 0: return launch_mass_t<WALLS, FORCE, 0, 0>(mb, b, s, ctl, ms, st);
    case 1: return launch_mass_t<WALLS, FORCE, 0, 1>(mb, b, s, ctl, ms, st);
    case 2: return launch_mass_t<WALLS, FORCE, 1, 0>(mb, b, s, ctl, ms, st);
    case 3: return launch_mass_t<WALLS, FORCE, 1, 1>(mb, b, s, ctl, ms, st);
    case 4: return launch_mass_t<WALLS, FORCE, 2, 0>(mb, b, s, ctl, ms, st);
    default: return launch_mass_t<WALLS, FORCE, 2, 1>(mb, b, s, ctl, ms, st);
  }
}

void launch_collide_mass(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, MixMass ms, bool moments,
                         cudaStream_t st) {
  if (mb.walls)
    launch_mass_wf<1, 1>(mb, b, s, ctl, ms, moments, st);
  else if (mb.force)
    launch_mass_wf<0, 1>(mb, b, s, ctl, ms, moments, st);
  else
    launch_mass_wf<0, 0>(mb, b, s, ctl, ms, moments, st);
}

template <int FORCE, int THERMO, int MOMENTS>
void launch_direct_t(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, cudaStream_t st) {
  int64_t grid = (static_cast<int64_t>(mb.ngroups) + 3) / 4;
  if (grid == 0) return;
  if (grid > 152 * 16) grid = 152 * 16;
  k_collide_direct_mixed<FORCE, THERMO, MOMENTS><<<static_cast<unsigned>(grid), 128, 0, st>>>(mb, b, s, ctl);
}

void launch_collide_direct(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, bool moments, cudaStream_t st) {
  switch ((mb.force ? 6 : 0) + 2 * mb.thermostat + (moments ? 1 : 0)) {
    case 0: return launch_direct_t<0, 0, 0>(mb, b, s, ctl, st);
    case 1: return launch_direct_t<0, 0, 1>(mb, b, s, ctl, st);
    case 2: return launch_direct_t<0, 1, 0>(mb, b, s, ctl, st);
    case 3: return launch_direct_t<0, 1, 1>(mb, b, s, ctl, st);
    case 4: return launch_direct_t<0, 2, 0>(mb, b, s, ctl, st);
    case 5: return launch_direct_t<0, 2, 1>(mb, b, s, ctl, st);
    case 6: return launch_direct_t<1, 0, 0>(mb, b, s, ctl, st);
    case 7: return launch_direct_t<1, 0, 1>(mb, b, s, ctl, st);
    case 8: return launch_direct_t<1, 1, 0>(mb, b, s, ctl, st);
    case 9: return launch_direct_t<1, 1, 1>(mb, b, s, ctl, st);
    case 10: return launch_direct_t<1, 2, 0>(mb, b, s, ctl, st);
    default: return launch_direct_t<1, 2, 1>(mb, b, s, ctl, st);
  }
}

template <int WARPS>
cudaError_t launch_collide_w(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, bool moments, cudaStream_t st,
                             bool prepare, int sel_override = -1) {
  // 0-11: (walls | force | neither) x (fixed-target thermostat or none) x moments;
  // 12-17: (walls | force | neither) x moments with the Maxwell-Boltzmann-scaling thermostat
  const int kind = mb.walls ? 2 : (mb.force ? 1 : 0);
  const int sel = sel_override >= 0 ? sel_override
                  : mb.thermostat == 2 ? 12 + 2 * kind + (moments ? 1 : 0)
                                       : 4 * kind | (mb.thermostat ? 2 : 0) | (moments ? 1 : 0);
  switch (sel) {
    case 0: return launch_collide_t<WARPS, 0, 0, 0, 0>(mb, b, s, ctl, st, prepare);
    case 1: return launch_collide_t<WARPS, 0, 0, 0, 1>(mb, b, s, ctl, st, prepare);
    case 2: return launch_collide_t<WARPS, 0, 0, 1, 0>(mb, b, s, ctl, st, prepare);
    case 3: return launch_collide_t<WARPS, 0, 0, 1, 1>(mb, b, s, ctl, st, prepare);
    case 4: return launch_collide_t<WARPS, 0, 1, 0, 0>(mb, b, s, ctl, st, prepare);
    case 5: return launch_collide_t<WARPS, 0, 1, 0, 1>(mb, b, s, ctl, st, prepare);
    case 6: return launch_collide_t<WARPS, 0, 1, 1, 0>(mb, b, s, ctl, st, prepare);
    case 7: return launch_collide_t<WARPS, 0, 1, 1, 1>(mb, b, s, ctl, st, prepare);
    case 8: return launch_collide_t<WARPS, 1, 1, 0, 0>(mb, b, s, ctl, st, prepare);
    case 9: return launch_collide_t<WARPS, 1, 1, 0, 1>(mb, b, s, ctl, st, prepare);
    case 10: return launch_collide_t<WARPS, 1, 1, 1, 0>(mb, b, s, ctl, st, prepare);
    case 11: return launch_collide_t<WARPS, 1, 1, 1, 1>(mb, b, s, ctl, st, prepare);
    case 12: return launch_collide_t<WARPS, 0, 0, 2, 0>(mb, b, s, ctl, st, prepare);
    case 13: return launch_collide_t<WARPS, 0, 0, 2, 1>(mb, b, s, ctl, st, prepare);
    case 14: return launch_collide_t<WARPS, 0, 1, 2, 0>(mb, b, s, ctl, st, prepare);
    case 15: return launch_collide_t<WARPS, 0, 1, 2, 1>(mb, b, s, ctl, st, prepare);
    case 16: return launch_collide_t<WARPS, 1, 1, 2, 0>(mb, b, s, ctl, st, prepare);
    default: return launch_collide_t<WARPS, 1, 1, 2, 1>(mb, b, s, ctl, st, prepare);
  }
}

}  // namespace

template <int WARPS, int WALLS, int FORCE, int THERMO, int MOMENTS>
cudaError_t launch_step_t(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, const StepAux& aux, cudaStream_t st,
                          bool prepare) {
  auto kern = k_step_mixed<WARPS, WALLS, FORCE, THERMO, MOMENTS>;
  const int smem = WARPS * static_cast<int>(sizeof(MixWarpStage<3 + MOMENTS>));
  static int resident = 0;
  if (prepare) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) resident = per_sm * sms;
    return e;
  }
  if (resident <= 0) return cudaErrorInvalidConfiguration;
  // every block resident (a cooperative launch fails instead of starting if they cannot be)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(resident));
  cfg.blockDim = dim3(WARPS * 32);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, mb, b, s, ctl, aux);
}

template <int WARPS>
cudaError_t launch_step_w(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, const StepAux& aux, bool moments,
                          cudaStream_t st, bool prepare, int sel_override = -1) {
  const int kind = mb.walls ? 2 : (mb.force ? 1 : 0);
  const int sel = sel_override >= 0 ? sel_override
                  : mb.thermostat == 2 ? 12 + 2 * kind + (moments ? 1 : 0)
                                       : 4 * kind | (mb.thermostat ? 2 : 0) | (moments ? 1 : 0);
  switch (sel) {
    case 0: return launch_step_t<WARPS, 0, 0, 0, 0>(mb, b, s, ctl, aux, st, prepare);
    case 1: return launch_step_t<WARPS, 0, 0, 0, 1>(mb, b, s, ctl, aux, st, prepare);
    case 2: return launch_step_t<WARPS, 0, 0, 1, 0>(mb, b, s, ctl, aux, st, prepare);
    case 3: return launch_step_t<WARPS, 0, 0, 1, 1>(mb, b, s, ctl, aux, st, prepare);
    case 4: return launch_step_t<WARPS, 0, 1, 0, 0>(mb, b, s, ctl, aux, st, prepare);
    case 5: return launch_step_t<WARPS, 0, 1, 0, 1>(mb, b, s, ctl, aux, st, prepare);
    case 6: return launch_step_t<WARPS, 0, 1, 1, 0>(mb, b, s, ctl, aux, st, prepare);
    case 7: return launch_step_t<WARPS, 0, 1, 1, 1>(mb, b, s, ctl, aux, st, prepare);
    case 8: return launch_step_t<WARPS, 1, 1, 0, 0>(mb, b, s, ctl, aux, st, prepare);
    case 9: return launch_step_t<WARPS, 1, 1, 0, 1>(mb, b, s, ctl, aux, st, prepare);
    case 10: return launch_step_t<WARPS, 1, 1, 1, 0>(mb, b, s, ctl, aux, st, prepare);
    case 11: return launch_step_t<WARPS, 1, 1, 1, 1>(mb, b, s, ctl, aux, st, prepare);
    case 12: return launch_step_t<WARPS, 0, 0, 2, 0>(mb, b, s, ctl, aux, st, prepare);
    case 13: return launch_step_t<WARPS, 0, 0, 2, 1>(mb, b, s, ctl, aux, st, prepare);
    case 14: return launch_step_t<WARPS, 0, 1, 2, 0>(mb, b, s, ctl, aux, st, prepare);
    case 15: return launch_step_t<WARPS, 0, 1, 2, 1>(mb, b, s, ctl, aux, st, prepare);
    case 16: return launch_step_t<WARPS, 1, 1, 2, 0>(mb, b, s, ctl, aux, st, prepare);
    default: return launch_step_t<WARPS, 1, 1, 2, 1>(mb, b, s, ctl, aux, st, prepare);
  }
}

cudaError_t prepare_collide_mixed() {
  static std::mutex mu;
  static uint64_t done = 0;  // devices prepared (bit per ordinal < 64)
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
  if (done & bit) return cudaSuccess;
  MixBatch mb{};
  MixBufs b{};
  MixScratch s{};
  const StepAux aux{};
  for (int sel = 0; sel < 18 && e == cudaSuccess; ++sel) {
    e = launch_collide_w<2>(mb, b, s, nullptr, false, nullptr, true, sel);
    if (e == cudaSuccess) e = launch_collide_w<4>(mb, b, s, nullptr, false, nullptr, true, sel);
    if (e == cudaSuccess) e = launch_step_w<2>(mb, b, s, nullptr, aux, false, nullptr, true, sel);
    if (e == cudaSuccess) e = launch_step_w<4>(mb, b, s, nullptr, aux, false, nullptr, true, sel);
  }
  if (e == cudaSuccess) done |= bit;
  return e;
}

void launch_collide_stream_mixed(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, bool moments, cudaStream_t st,
                                 MixMass ms) {
  if (ms.m[0])
    launch_collide_mass(mb, b, s, ctl, ms, moments, st);
  else if (mb.angular)
    launch_collide_direct(mb, b, s, ctl, moments, st);
  else if (mb.warps == 2)
    (void)launch_collide_w<2>(mb, b, s, ctl, moments, st, false);
  else
    (void)launch_collide_w<4>(mb, b, s, ctl, moments, st, false);
}

int64_t step_scan_tiles(int64_t ncell) {
  constexpr int64_t kMinTile = 2 * 32 * kStepScanItems;  // two-warp blocks have the smallest tiles
  return (ncell + kMinTile - 1) / kMinTile;
}

cudaError_t launch_step_mixed(const MixBatch& mb, MixBufs b, MixScratch s, Ctl* ctl, bool moments,
                              const MixGroupSpec* spec, MixGroup* groups, unsigned* bar, int stall, cudaStream_t st) {
  const StepAux aux{spec, groups, bar, stall};
  return mb.warps == 2 ? launch_step_w<2>(mb, b, s, ctl, aux, moments, st, false)
                       : launch_step_w<4>(mb, b, s, ctl, aux, moments, st, false);
}

void launch_end_step_mixed(const MixBatch& mb, Ctl* ctl, cudaStream_t st) { k_end_step_mixed<<<1, 256, 0, st>>>(mb, ctl); }

void launch_scatter_cursor(int64_t n, const int32_t* key, const int32_t* offset, int32_t* cursor, int32_t* perm,
                           cudaStream_t st) {
  k_scatter_cursor<<<grid_for(n, 8), kThreads, 0, st>>>(n, key, offset, cursor, perm);
}

void launch_group_bounds(const MixBatch& mb, const MixGroupSpec* spec, const int32_t* offset, MixGroup* groups,
                         cudaStream_t st) {
  if (mb.ngroups > 0)
    k_group_bounds<<<grid_for(mb.ngroups), kThreads, 0, st>>>(mb.ngroups, mb.boxes, spec, offset, groups);
}

void launch_get_state_mixed(const MixBatch& mb, MixBufs b, int cur, double* r, double* v, cudaStream_t st) {
  k_get_state_mixed<<<grid_for(mb.n), kThreads, 0, st>>>(mb, b.rec[cur], r, v);
}

// The two halves of the single-box check, for a state whose positions arrive before its
// velocities: the lowest failing index over both lands in *bad (atomicMin), as with the whole.
__global__ void __launch_bounds__(kThreads) k_check_positions_box(int64_t n, Geom g, const double* __restrict__ r,
                                                                  unsigned long long* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) ok = ok && r[3 * i + d] >= 0.0 && r[3 * i + d] < g.B[d];
    if (!ok) atomicMin(bad, static_cast<unsigned long long>(i));
  }
}

__global__ void __launch_bounds__(kThreads) k_check_velocities(int64_t n, const double* __restrict__ v,
                                                               unsigned long long* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(isfinite(v[3 * i]) && isfinite(v[3 * i + 1]) && isfinite(v[3 * i + 2])))
      atomicMin(bad, static_cast<unsigned long long>(i));
}

void launch_check_positions(const Geom& g, int64_t n, const double* r, unsigned long long* bad, cudaStream_t st) {
  k_check_positions_box<<<grid_for(n), kThreads, 0, st>>>(n, g, r, bad);
}

void launch_check_velocities(int64_t n, const double* v, unsigned long long* bad, cudaStream_t st) {
  k_check_velocities<<<grid_for(n), kThreads, 0, st>>>(n, v, bad);
}

void launch_check_state(const MixBatch* mb, const Geom& g, int64_t n, const double* r, const double* v,
                        unsigned long long* bad, cudaStream_t st) {
  if (mb)
    k_check_state_batch<<<grid_for(n), kThreads, 0, st>>>(*mb, r, v, bad);
  else
    k_check_state_box<<<grid_for(n), kThreads, 0, st>>>(n, g, r, v, bad);
}

void launch_set_state_mixed(const MixBatch& mb, MixBufs b, const double* r, const double* v, cudaStream_t st) {
  k_set_state_mixed<<<grid_for(mb.n), kThreads, 0, st>>>(mb, b, r, v);
}

}  // namespace mpcd
