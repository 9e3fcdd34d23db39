// cellmath.cuh -- per-cell arithmetic of the collision step shared by every kernel path, so
// that the dense and the generic collide kernels give bit-identical results.
//
//  * Exact cell sums: each FP64 velocity component is added to a 128-bit two's-complement
//    fixed-point accumulator with 2^-80 resolution.  Integer addition is associative, so the
//    sum does not depend on the order the particles arrive in, and converting the total
//    back to FP64 rounds once.  The work runs on the integer pipe, which on GB300 is ~30x
//    wider than the FP64 pipe.
//  * Rotation frame: for a cell with centre-of-mass velocity u and random axis n, the
//    collision v' = u + R(n, alpha)(v - u) (paper Sec. 2, parts (ii)-(iii)) is applied as
//    v' = R v + b with b = u - R u, i.e. nine FMAs per particle.
//  * Cell coordinates: floor() and the periodic-wrap comparisons are done on the IEEE bit
//    patterns with integer instructions, and for a power-of-two cell size r - s too, in
//    fixed point, except within a few 2^-32 cells of a face, where the FP64 subtraction
//    decides; r + v dt stays in FP64.
#pragma once
#include <cstdint>
#include <cstring>

#include "device_common.cuh"
#include "mpcd_internal.h"

namespace mpcd {

// ------------------------------------------------------------ exact accumulator ----
struct Fx128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ void fx_zero(Fx128& a) {
  a.lo = 0ull;
  a.hi = 0ull;
}

// a += x * 2^80 (exact for |x| >= 2^-27, truncated below 2^-80).  Returns false, leaving a
// unchanged, when |x| >= 2^16: beyond that range a sum of up to 2^31 values could overflow.
// The 64-bit pattern of a double, assembled from its two 32-bit words.  Written this way,
// the floor and wrap tests of the streaming kernel issue no FP64-pipe instructions: ncu's
// pipe counters on GB300 fell from 12.3 to 6.3 per particle (the 3 DFMA + 3 DSUB).
__device__ __forceinline__ unsigned long long dbits(double x) {
  return (static_cast<unsigned long long>(static_cast<unsigned>(__double2hiint(x))) << 32) |
         static_cast<unsigned>(__double2loint(x));
}

// The same on the host too (the fixed-point cell floor below is checked there).
__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return dbits(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

__device__ __forceinline__ bool fx_add(Fx128& a, double x) {
  const unsigned long long bits = dbits(x);
  const int e = static_cast<int>((bits >> 52) & 0x7FF);
  if (e == 0) return true;          // zero or subnormal: below the 2^-80 grid
  if (e > 1038) return false;       // |x| >= 2^16, or inf / NaN
  const unsigned long long m = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int s = e - 995;            // x * 2^80 = m * 2^s, s <= 43
  unsigned long long lo, hi;
  if (s > 0) {
    lo = m << s;
    hi = m >> (64 - s);
  } else if (s > -64) {
    lo = m >> (-s);
    hi = 0ull;
  } else {
    return true;
  }
  if (bits >> 63) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(lo), "l"(hi));
  return true;
}

// The accumulated value rounded once to FP64 (round to nearest even).
__device__ __forceinline__ double fx_value(const Fx128& a) {
  unsigned long long lo = a.lo, hi = a.hi;
  const bool neg = static_cast<long long>(hi) < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  if ((hi | lo) == 0ull) return 0.0;
  unsigned long long top;
  int k;
  if (hi) {
    const int lz = __clzll(static_cast<long long>(hi));
    top = lz ? ((hi << lz) | (lo >> (64 - lz))) : hi;
    const unsigned long long rest = lz ? (lo << lz) : lo;
    top |= (rest != 0ull) ? 1ull : 0ull;  // sticky bit: keeps the single rounding correct
    k = 64 - lz;
  } else {
    const int lz = __clzll(static_cast<long long>(lo));
    top = lo << lz;
    k = -lz;
  }
  // top * 2^(k - 80) with top rounded to 53 bits (nearest, ties to even), assembled from its
  // fields: the same bits as converting top and scaling by 2^(k - 80), without the two
  // instructions on GB300's narrow FP64 pipe
  unsigned long long m = top >> 11;
  const unsigned rem = static_cast<unsigned>(top & 0x7FFull);
  if (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ++m;
  unsigned long long e = static_cast<unsigned long long>(1006 + k);  // top in [2^63, 2^64)
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  const unsigned long long bits = (e << 52) | (m & 0x000FFFFFFFFFFFFFull) | (neg ? 0x8000000000000000ull : 0ull);
  return __longlong_as_double(static_cast<long long>(bits));
}

// 1/n for the common occupancies (constant-folded, correctly rounded); others divide.
#define MPCD_INV8(k) 1.0 / (k), 1.0 / (k + 1), 1.0 / (k + 2), 1.0 / (k + 3), 1.0 / (k + 4), 1.0 / (k + 5), \
                     1.0 / (k + 6), 1.0 / (k + 7)
static __constant__ double c_inv_n[65] = {0.0,           MPCD_INV8(1),  MPCD_INV8(9),  MPCD_INV8(17), MPCD_INV8(25),
                                   MPCD_INV8(33), MPCD_INV8(41), MPCD_INV8(49), MPCD_INV8(57)};
#undef MPCD_INV8

static __device__ __noinline__ double inv_count_slow(int n) { return 1.0 / static_cast<double>(n); }
__device__ __forceinline__ double inv_count(int n) { return n <= 64 ? c_inv_n[n] : inv_count_slow(n); }

// ---------------------------------------------------------------- rotation frame ----
// R(n, alpha) v = cos(a) v + sin(a) (n x v) + (1 - cos(a)) (n . v) n; b = u - R u.
__device__ __forceinline__ void make_frame(const Geom& g, int64_t t1, int64_t cell, double u0, double u1, double u2,
                                           double R[9], double bvec[3]) {
  double n[3];
  random_axis(g.seed, t1, cell, n);
  const double c = g.cos_a, s = g.sin_a, w = 1.0 - g.cos_a;
  const double wx = w * n[0], wy = w * n[1], wz = w * n[2];
  const double sx = s * n[0], sy = s * n[1], sz = s * n[2];
  R[0] = fma(wx, n[0], c);
  R[1] = fma(wx, n[1], -sz);
  R[2] = fma(wx, n[2], sy);
  R[3] = fma(wy, n[0], sz);
  R[4] = fma(wy, n[1], c);
  R[5] = fma(wy, n[2], -sx);
  R[6] = fma(wz, n[0], -sy);
  R[7] = fma(wz, n[1], sx);
  R[8] = fma(wz, n[2], c);
  bvec[0] = u0 - fma(R[0], u0, fma(R[1], u1, R[2] * u2));
  bvec[1] = u1 - fma(R[3], u0, fma(R[4], u1, R[5] * u2));
  bvec[2] = u2 - fma(R[6], u0, fma(R[7], u1, R[8] * u2));
}

__device__ __forceinline__ void apply_frame(const double R[9], const double bvec[3], double& v0, double& v1,
                                            double& v2) {
  const double a0 = fma(R[0], v0, fma(R[1], v1, fma(R[2], v2, bvec[0])));
  const double a1 = fma(R[3], v0, fma(R[4], v1, fma(R[5], v2, bvec[1])));
  const double a2 = fma(R[6], v0, fma(R[7], v1, fma(R[8], v2, bvec[2])));
  v0 = a0;
  v1 = a1;
  v2 = a2;
}

// --------------------------------------------------- float-float rotation frame ----
// GB300 issues about 60 times fewer FP64 than FP32 instructions per clock, so the dense pair
// applies the frame v' = R v + b in float-float arithmetic (each value a pair of FP32 numbers
// hi + lo): an FP32 product's rounding error is exact through an FMA, and Knuth's two-sum
// gives a sum's error exactly, so the pair carries about 46 bits.  The split of a double and
// the assembly of the result use integer instructions, and one exact DADD per component
// joins the pair; the relative error of v' is below about 2^-44 (|v| + |b|) / max(|v'|, ...),
// far inside the 1e-12 bound the FP64 form is held to.

// x = hi + lo with hi the top 24 significand bits of x (truncated) and lo the remaining 29
// rounded to 24: |x - hi - lo| <= 2^-48 |x| for 2^-74 <= |x| < 2^127.  Smaller magnitudes
// give 0 (they lie far below the velocity scale); larger ones do not occur for finite states.
__device__ __forceinline__ void ff_split(double x, float& hi, float& lo) {
  const int h = __double2hiint(x);
  const unsigned l = static_cast<unsigned>(__double2loint(x));
  const int e = (h >> 20) & 0x7FF;
  if (e < 949 || e > 1150) {
    hi = e > 1150 ? __double2float_rn(x) : 0.0f;  // inf/NaN stay non-finite
    lo = 0.0f;
    return;
  }
  const unsigned sign = static_cast<unsigned>(h) & 0x80000000u;
  hi = __uint_as_float(sign | (static_cast<unsigned>(e - 896) << 23) | ((static_cast<unsigned>(h) & 0xFFFFFu) << 3) |
                       (l >> 29));
  // the remaining 29 bits, worth (l mod 2^29) 2^(e - 1075); 2^(e - 1075) is a normal float for e >= 949
  const float scale = __uint_as_float(static_cast<unsigned>(e - 948) << 23);
  const float rest = __fmul_rn(__uint2float_rn(l & 0x1FFFFFFFu), scale);
  lo = sign ? -rest : rest;
}

// A float as a double, from its bit fields (zero and subnormals give 0).
__device__ __forceinline__ double ff_widen(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  return __hiloint2double(static_cast<int>((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3)),
                          static_cast<int>(b << 29));
}

// acc += a * x in float-float (a and x pairs): the product of the high parts exactly as
// p + pe, the cross terms in FP32, p added to acc.hi by two-sum.  No contraction: every
// operation is an explicit intrinsic.
__device__ __forceinline__ void ff_madd(float ah, float al, float xh, float xl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, xh);
  const float pe = __fmaf_rn(ah, xh, -p);
  const float cross = __fmaf_rn(ah, xl, __fmul_rn(al, xh));
  const float s2 = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s2, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s2, bb)), __fsub_rn(p, bb));
  sh = s2;
  sl = __fadd_rn(sl, __fadd_rn(err, __fadd_rn(pe, cross)));
}

// (sh, sl) -> double: renormalise by two-sum, then join the two halves with one exact DADD.
__device__ __forceinline__ double ff_join(float sh, float sl) {
  const float s = __fadd_rn(sh, sl);
  const float bb = __fsub_rn(s, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(sl, bb));
  return __dadd_rn(ff_widen(s), ff_widen(e));
}

// A float-float value (hi + lo) and the two operations the frame needs, every FP32
// operation an explicit intrinsic (no contraction): the product keeps the exact error of the
// high parts' product (an FMA) and the cross terms; the sum adds the high parts by two-sum.
// Both renormalise (|lo| <= ulp(hi) / 2).
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ FF ff_of(double x) {
  FF r;
  ff_split(x, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  return ff_norm(p, __fadd_rn(pe, __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi))));
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return ff_norm(s, __fadd_rn(err, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

// Frame record of the float-float form (32 floats = 128 bytes per cell): row i of R and b
// as R hi (3), b hi, R lo (3), b lo at floats 8 i .. 8 i + 7 (two float4), so that a row can
// be loaded and applied on its own; the rotate flag (1 or 0) at float 24.
__host__ __device__ constexpr int ff_rhi(int i, int j) { return 8 * i + j; }
__host__ __device__ constexpr int ff_rlo(int i, int j) { return 8 * i + 4 + j; }
__host__ __device__ constexpr int ff_bhi(int i) { return 8 * i + 3; }
__host__ __device__ constexpr int ff_blo(int i) { return 8 * i + 7; }
constexpr int kFfFlag = 24;

// The frame of a cell with centre-of-mass velocity u directly in float-float form, written
// as the 128-byte record: the axis n comes from the FP64 draw (random_axis), then
// R = cos(a) 1 + sin(a) [n]x + (1 - cos(a)) n n^T and b = u - R u are built in float-float
// arithmetic, so the frame costs the FP64 pipe only the axis.
__device__ __forceinline__ void make_frame_ff(const Geom& g, int64_t t1, int64_t cell, double u0, double u1, double u2,
                                              float* rec) {
  double nd[3];
  random_axis(g.seed, t1, cell, nd);
  const FF n[3] = {ff_of(nd[0]), ff_of(nd[1]), ff_of(nd[2])};
  const FF c = ff_of(g.cos_a), s = ff_of(g.sin_a), w = ff_of(1.0 - g.cos_a);
  const FF wn[3] = {ff_mul(w, n[0]), ff_mul(w, n[1]), ff_mul(w, n[2])};
  const FF sn[3] = {ff_mul(s, n[0]), ff_mul(s, n[1]), ff_mul(s, n[2])};
  FF R[9];
  R[0] = ff_add(ff_mul(wn[0], n[0]), c);
  R[1] = ff_add(ff_mul(wn[0], n[1]), ff_neg(sn[2]));
  R[2] = ff_add(ff_mul(wn[0], n[2]), sn[1]);
  R[3] = ff_add(ff_mul(wn[1], n[0]), sn[2]);
  R[4] = ff_add(ff_mul(wn[1], n[1]), c);
  R[5] = ff_add(ff_mul(wn[1], n[2]), ff_neg(sn[0]));
  R[6] = ff_add(ff_mul(wn[2], n[0]), ff_neg(sn[1]));
  R[7] = ff_add(ff_mul(wn[2], n[1]), sn[0]);
  R[8] = ff_add(ff_mul(wn[2], n[2]), c);
  const FF u[3] = {ff_of(u0), ff_of(u1), ff_of(u2)};
  float w28[28];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float sh = u[i].hi, sl = u[i].lo;  // b_i = u_i - sum_j R_ij u_j
#pragma unroll
    for (int j = 0; j < 3; ++j) ff_madd(-R[3 * i + j].hi, -R[3 * i + j].lo, u[j].hi, u[j].lo, sh, sl);
    const FF b = ff_norm(sh, sl);
    w28[ff_bhi(i)] = b.hi;
    w28[ff_blo(i)] = b.lo;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    w28[ff_rhi(k / 3, k % 3)] = R[k].hi;
    w28[ff_rlo(k / 3, k % 3)] = R[k].lo;
  }
  w28[kFfFlag] = 1.0f;
  w28[25] = w28[26] = w28[27] = 0.0f;
  float4* o = reinterpret_cast<float4*>(rec);
#pragma unroll
  for (int k = 0; k < 7; ++k) o[k] = make_float4(w28[4 * k], w28[4 * k + 1], w28[4 * k + 2], w28[4 * k + 3]);
}

// v' = R v + b with the frame in float-float form (w: the record's first 28 floats).
__device__ __forceinline__ void ff_apply_frame(const float w[28], double& v0, double& v1, double& v2) {
  float vh[3], vl[3];
  ff_split(v0, vh[0], vl[0]);
  ff_split(v1, vh[1], vl[1]);
  ff_split(v2, vh[2], vl[2]);
  double out[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float sh = w[ff_bhi(i)], sl = w[ff_blo(i)];
#pragma unroll
    for (int j = 0; j < 3; ++j) ff_madd(w[ff_rhi(i, j)], w[ff_rlo(i, j)], vh[j], vl[j], sh, sl);
    out[i] = ff_join(sh, sl);
  }
  v0 = out[0];
  v1 = out[1];
  v2 = out[2];
}

// The same, loading each row of the record (two float4) just before it is applied, so that
// only one row is live at a time.
__device__ __forceinline__ void ff_apply_frame_rows(const float4* __restrict__ rec, double& v0, double& v1, double& v2) {
  float vh[3], vl[3];
  ff_split(v0, vh[0], vl[0]);
  ff_split(v1, vh[1], vl[1]);
  ff_split(v2, vh[2], vl[2]);
  double out[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float4 hi = rec[2 * i], lo = rec[2 * i + 1];  // R hi (3), b hi | R lo (3), b lo
    float sh = hi.w, sl = lo.w;
    ff_madd(hi.x, lo.x, vh[0], vl[0], sh, sl);
    ff_madd(hi.y, lo.y, vh[1], vl[1], sh, sl);
    ff_madd(hi.z, lo.z, vh[2], vl[2], sh, sl);
    out[i] = ff_join(sh, sl);
  }
  v0 = out[0];
  v1 = out[1];
  v2 = out[2];
}

// -------------------------------------------------------------- cell coordinates ----
// x / a in units of 2^-32 (truncated toward zero), a = 2^log2a, from the bit pattern of x,
// for |x / a| < 2^22; false for larger magnitudes, inf and NaN.
__host__ __device__ __forceinline__ bool fx32_trunc(double x, int log2a, long long& X) {
  const unsigned long long b = bits_of(x);
  const int e = static_cast<int>((b >> 52) & 0x7FFull) - 1023 - log2a;  // |x / a| in [2^e, 2^(e+1))
  if (e > 21) return false;
  const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int sh = 20 - e;  // |x / a| 2^32 = m 2^(e - 20); zero and subnormals shift out to 0
  const unsigned long long q = sh <= 0 ? (m << -sh) : (sh < 64 ? (m >> sh) : 0ull);
  X = (b >> 63) ? -static_cast<long long>(q) : static_cast<long long>(q);
  return true;
}

// floor(fl(x - s) / a) (a = 2^log2a, S = s / a as fx32_trunc gives it) without the FP64
// subtraction.  D = X - S is within 2 units of 2^-32 of (x - s) / a (each truncation less
// than one), and rounding x - s to FP64 moves it by at most 2^-53 |x - s| / a, under 2 more
// units for |x - s| < 2^22 a; so where D lies 8 or more units from a cell face its integer
// part is the floor of the rounded difference.  False otherwise (and for |x / a| >= 2^22):
// the caller subtracts in FP64.
__host__ __device__ __forceinline__ bool cell_floor_fx(double x, long long S, int log2a, int& c) {
  long long X;
  if (!fx32_trunc(x, log2a, X)) return false;
  const long long D = X - S;
  const unsigned frac = static_cast<unsigned>(static_cast<unsigned long long>(D) & 0xFFFFFFFFull);
  if (frac - 8u > 0xFFFFFFEFu) return false;  // frac < 8 or frac > 2^32 - 9
  c = static_cast<int>(D >> 32);
  return true;
}

// floor(q * 2^k) for |q * 2^k| < 2^30 from the bit pattern of q (integer pipe only; the
// power-of-two scale is an exponent shift, so no FP64 multiply is needed).  Larger
// magnitudes return +-2^30; callers clamp coordinates into range.
static __device__ __noinline__ int floor_bits_wide(double q, int k) {
  const long long b = __double_as_longlong(q);
  const int eb = static_cast<int>((b >> 52) & 0x7FF);
  if (eb == 0) return (b < 0 && (b << 1) != 0) ? -1 : 0;  // zero or subnormal
  const int e = eb - 1023 + k;
  if (e < 0) return (b < 0) ? -1 : 0;                      // 0 < |q 2^k| < 1
  if (e > 29) return (b < 0) ? -(1 << 30) : (1 << 30);
  const unsigned long long m = (static_cast<unsigned long long>(b) & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int sh = 52 - e;
  const int ip = static_cast<int>(m >> sh);
  if (b >= 0) return ip;
  return (m & ((1ull << sh) - 1ull)) ? -ip - 1 : -ip;
}

// The same value with 32-bit operations on the two words of q for |q 2^k| < 2^21, where
// the integer part lies in the high word (zero and subnormals fall under e < 0).
__device__ __forceinline__ int floor_bits(double q, int k = 0) {
  const int hi = __double2hiint(q);
  const unsigned lo = static_cast<unsigned>(__double2loint(q));
  const int e = ((hi >> 20) & 0x7FF) - 1023 + k;
  if (e < 0) return (hi < 0 && ((static_cast<unsigned>(hi) & 0x7FFFFFFFu) | lo) != 0u) ? -1 : 0;
  if (e > 20) return floor_bits_wide(q, k);
  const unsigned mh = (static_cast<unsigned>(hi) & 0xFFFFFu) | 0x100000u;  // bits 52..32 of the mantissa
  const int sh = 20 - e;
  const int ip = static_cast<int>(mh >> sh);
  if (hi >= 0) return ip;
  return ((mh & ((1u << sh) - 1u)) | lo) ? -ip - 1 : -ip;
}

// Out-of-range part of the periodic wrap; kept out of line so that the compiler does not
// evaluate its FP64 comparisons on the common in-range path.
static __device__ __noinline__ double wrap_slow(double x, double B) {
  if (x >= B)
    x = __dsub_rn(x, B);
  else if (x < 0.0)
    x = __dadd_rn(x, B);
  if (x >= B || x < 0.0) {  // moved more than one box length, or rounded onto B
    x = fmod(x, B);
    if (x < 0.0) x = __dadd_rn(x, B);
    if (x >= B) x = 0.0;
  }
  return x;
}

// Periodic wrap into [0, B): the in-range test runs on the bit patterns (for x >= +0 the
// IEEE order is the integer order; negative x has the sign bit set).
__device__ __forceinline__ double wrap_box(double x, double B, long long Bbits) {
  const long long b = static_cast<long long>(dbits(x));
  if (b < Bbits && (b >= 0 || (b << 1) == 0)) return x;  // 0 <= x < B (or -0.0)
  return wrap_slow(x, B);
}

// ------------------------------------------------------------------ grid shifts ----
// Shift of step t in cell units for the mixed form; with walls the z part lies in [0, 1).
__host__ __device__ __forceinline__ void shift_in_cells(const Geom& g, const double sd[3], float sf[3]) {
  for (int d = 0; d < 3; ++d) sf[d] = static_cast<float>(sd[d] * g.inv_a);
  if (g.walls && sf[2] >= 1.0f) sf[2] = 0.99999994f;
}

// Advance the control block's shifts so that they describe steps t + 1 and t + 2 (computed
// once per step here instead of in every block of the step's kernels).
__host__ __device__ __forceinline__ void set_shifts(const Geom& g, Ctl* c) {
  grid_shift(g.seed, c->t + 1, g.a, g.walls, c->shift);
  grid_shift(g.seed, c->t + 2, g.a, g.walls, c->shift_next);
  shift_in_cells(g, c->shift, c->sf);
  shift_in_cells(g, c->shift_next, c->sf_next);
}

}  // namespace mpcd
