// device_common.cuh -- device helpers shared by the libmpcd kernels: the counter-based
// Philox4x64-10 generator, exact uniform doubles, the random rotation axis and Box-Muller.
//
// Random numbers (axis, shift, initial state, wall particles, thermostat) all come from
// Philox4x64-10 (Salmon et al., SC'11) keyed by (seed, 0) with counter (a, b, tag, 0) -- the
// thermostat's rejection loop counts its attempts in the last word -- so that every draw
// is a pure function of (seed, step, cell) and independent of launch order (the paper's
// random axis per cell, Sec. 2; random grid shift, Sec. 2 and Listing 1's offset).
#pragma once
#include <cstdint>

namespace mpcd {

enum : uint64_t { kTagInit = 0, kTagShift = 1, kTagAxis = 2, kTagThermo = 3, kTagWall = 4 };

struct u64x4 {
  uint64_t x, y, z, w;
};

// Philox4x64-10: ten rounds of two 64x64->128 multiplications by fixed odd constants,
// mixing the high halves with the other two counter words and the round key; the key is
// advanced by two Weyl increments between rounds.
__host__ __device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                        uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#if defined(__CUDA_ARCH__)
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
#else
    const unsigned __int128 p0 = (unsigned __int128)M0 * c0, p1 = (unsigned __int128)M1 * c2;
    const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
#endif
    const uint64_t n0 = hi1 ^ c1 ^ k0;
    const uint64_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  return {c0, c1, c2, c3};
}

__host__ __device__ __forceinline__ u64x4 draw(uint64_t seed, uint64_t a, uint64_t b, uint64_t tag) {
  return philox4x64_10(a, b, tag, 0, seed, 0);
}

// The top 53 bits of w as k * 2^-53, uniform on [0, 1); exact in FP64.
__host__ __device__ __forceinline__ double unit53(uint64_t w) {
#ifdef __CUDA_ARCH__
  // the same value assembled from its fields (no 64-bit conversion on the narrow FP64 pipe):
  // m = w >> 11 < 2^53 is exact in FP64, and m 2^-53 = 1.f 2^(10 - clz(m))
  const uint64_t m = w >> 11;
  if (m == 0) return 0.0;
  const int lz = __clzll(static_cast<long long>(m));  // 11 .. 63
  const uint64_t mant = m << (lz - 11);                // leading one at bit 52
  return __longlong_as_double(static_cast<long long>((static_cast<uint64_t>(1033 - lz) << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
#else
  return static_cast<double>(w >> 11) * 0x1.0p-53;
#endif
}

// Grid shift of step t: uniform in [-a/2, a/2) per axis; with walls the z component is
// folded into [0, a) so the wall-bounded direction has exactly Lz + 1 cell layers.
__host__ __device__ __forceinline__ void grid_shift(uint64_t seed, int64_t t, double a, int walls, double s[3]) {
  const u64x4 w = draw(seed, static_cast<uint64_t>(t), 0, kTagShift);
  s[0] = (unit53(w.x) - 0.5) * a;
  s[1] = (unit53(w.y) - 0.5) * a;
  s[2] = (unit53(w.z) - 0.5) * a;
  if (walls && s[2] < 0.0) s[2] += a;
}

#if defined(__CUDACC__)
// Unit axis uniform on the sphere: z uniform on [-1, 1), azimuth uniform on [0, 2 pi).
__device__ __forceinline__ void random_axis(uint64_t seed, int64_t t, int64_t cell, double n[3]) {
  const u64x4 w = draw(seed, static_cast<uint64_t>(t), static_cast<uint64_t>(cell), kTagAxis);
  const double z = 2.0 * unit53(w.x) - 1.0;
  double sp, cp;
  sincospi(2.0 * unit53(w.y), &sp, &cp);
  const double rho = sqrt((1.0 - z) * (1.0 + z));
  n[0] = rho * cp;
  n[1] = rho * sp;
  n[2] = z;
}

// Two independent standard normals from two uniform words (Box-Muller).
__device__ __forceinline__ void gauss_pair(uint64_t w0, uint64_t w1, double& g0, double& g1) {
  const double u1 = 1.0 - unit53(w0);  // (0, 1]
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * unit53(w1), &s, &c);
  g0 = rad * c;
  g1 = rad * s;
}

// Gamma(shape, 1) variate of a cell for the Maxwell-Boltzmann-scaling thermostat, shape >= 1,
// by Marsaglia and Tsang's method (ACM TOMS 26(3), 2000): with d = shape - 1/3 and
// c = 1/sqrt(9 d), attempt k takes a standard normal x (Box-Muller, cosine branch, from words
// 0 and 1 of Philox counter (t, cell, THERMO, k)) and u in (0, 1] (word 2); with
// tt = 1 + c x > 0 and v = tt^3 it returns d v when u < 1 - 0.0331 x^4 or
// log u < x^2 / 2 + d (1 - v + log v).  Every product and sum is rounded on its own (no
// contraction), so the accept decisions are those of the same arithmetic on the host.  After
// 64 rejected attempts (probability below 1e-80) it returns d.
static __device__ __noinline__ double mbs_gamma(uint64_t seed, int64_t t, int64_t cell, double shape) {
  const double d = __dsub_rn(shape, 1.0 / 3.0);
  const double c = 1.0 / sqrt(__dmul_rn(9.0, d));
  for (uint64_t k = 0; k < 64; ++k) {
    const u64x4 w = philox4x64_10(static_cast<uint64_t>(t), static_cast<uint64_t>(cell), kTagThermo, k, seed, 0);
    const double rad = sqrt(__dmul_rn(-2.0, log(1.0 - unit53(w.x))));
    const double x = __dmul_rn(rad, cospi(2.0 * unit53(w.y)));
    const double tt = __dadd_rn(1.0, __dmul_rn(c, x));
    if (tt <= 0.0) continue;
    const double v = __dmul_rn(__dmul_rn(tt, tt), tt);
    const double u = 1.0 - unit53(w.z);
    const double x2 = __dmul_rn(x, x);
    if (u < __dsub_rn(1.0, __dmul_rn(0.0331, __dmul_rn(x2, x2)))) return __dmul_rn(d, v);
    if (log(u) < __dadd_rn(__dmul_rn(0.5, x2), __dmul_rn(d, __dadd_rn(__dsub_rn(1.0, v), log(v)))))
      return __dmul_rn(d, v);
  }
  return d;
}
#endif

}  // namespace mpcd
