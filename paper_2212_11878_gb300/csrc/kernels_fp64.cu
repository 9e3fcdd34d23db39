// kernels_fp64.cu -- the FP64 form of the SRD step (the paper's `double` state, Listing 1).
//
// Step = stream_bin -> scan -> scatter -> collide -> end_step:
//   stream_bin  per particle: ballistic move (+ body force, bounce-back walls), periodic
//               wrap, cell key on this step's shifted grid, arrival rank from one atomic
//               increment of the cell count (Sec. 2; Sec. 3.1 cell flagging).
//   scan        exclusive prefix sum of the counts (kernels_scan.cu).
//   scatter     perm[offset[key] + rank] = slot (linked-cell list as a counting sort).
//   collide     per cell: restore storage order inside the cell (stable sort), sum mass and
//               momentum (Listing 4), centre-of-mass velocity, random axis, rotate every
//               member's relative velocity by alpha (Sec. 2 (ii)-(iii)); on re-sort steps
//               write the members to the other buffer set in cell order (Listing 1 permute).
//   end_step    advances the device-side step counter.
//
// GB300 executes about 2 FP64 FMAs per clock per SM against ~128 FP32 and ~64 integer
// operations, so these kernels keep in FP64 only what decides the result's rounding:
// the streaming FMA and the r - s of the cell key (bit-exact keys), the nine FMAs of the
// rotation and the per-cell frame.  Wraps, floors and the cell sums run on the integer
// pipe (cellmath.cuh).
#include <climits>

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


// Cell keys of step t.  The dense pair double-buffers them by the parity of t: its fused
// rotate-and-stream kernel reads step t's keys (the frame of each slot's cell) while it writes
// step t + 1's at the re-sort destinations.  Everywhere else key2 == key.
__device__ __forceinline__ int32_t* keys_of(const Scratch& s, int64_t t) { return (t & 1) ? s.key2 : s.key; }

__device__ __forceinline__ double wrap_periodic(double x, double B) {
  return wrap_box(x, B, __double_as_longlong(B));
}

// floor(fl(x - s) / a) for a power-of-two a with the FP64 subtraction: out of line, for the
// rare coordinates the fixed-point test cannot decide.
static __device__ __noinline__ int cell_floor_fp64(double x, double s, int log2a) {
  return floor_bits(__dsub_rn(x, s), -log2a);
}

// Cell coordinate along one axis on the grid shifted by s.  POW2A (a a power of two): in
// 32.32 fixed point on the integer pipe (cell_floor_fx; S is loop-invariant), the FP64
// subtraction only within 8 / 2^32 cells of a face; either way the floor of the rounded
// FP64 difference.  Otherwise an FP64 division.
template <int POW2A>
__device__ __forceinline__ int cell_coord(double x, double s, const Geom& g, int d) {
  int c;
  if (POW2A) {
    long long S;
    if (!(fx32_trunc(s, g.log2a, S) && cell_floor_fx(x, S, g.log2a, c))) c = cell_floor_fp64(x, s, g.log2a);
  } else {
    c = floor_bits(__ddiv_rn(__dsub_rn(x, s), g.a));
  }
  if (g.walls && d == 2) {  // layers 0 .. Lz; rounding of (z - s)/a may reach Lz + 1
    c += 1;
    return c < 0 ? 0 : (c > g.L[2] ? g.L[2] : c);
  }
  if (c < 0) c += g.L[d];
  else if (c >= g.L[d]) c -= g.L[d];
  return c < 0 ? 0 : (c >= g.L[d] ? g.L[d] - 1 : c);  // only a state outside the box gets here
}

// Ballistic move over dt with bounce-back at z = 0 and z = H (velocity reversed at the
// crossing time, then the rest of the step).
__device__ __forceinline__ void stream_walls(const Geom& g, double r[3], double v[3]) {
  const double H = g.B[2];
  double left = g.dt;
  for (int bounce = 0; bounce < 64 && left > 0.0; ++bounce) {
    const double z1 = __dadd_rn(r[2], __dmul_rn(v[2], left));
    double tau = left, wall = -1.0;
    if (z1 < 0.0) {
      tau = __ddiv_rn(__dsub_rn(0.0, r[2]), v[2]);
      wall = 0.0;
    } else if (z1 >= H) {
      tau = __ddiv_rn(__dsub_rn(H, r[2]), v[2]);
      wall = H;
    }
    if (tau < 0.0) tau = 0.0;
    if (tau > left) tau = left;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const double hh = __dmul_rn(__dmul_rn(__dmul_rn(0.5, g.g[d]), tau), tau);
      r[d] = fma(v[d], tau, __dadd_rn(r[d], hh));
      v[d] = fma(g.g[d], tau, v[d]);
    }
    if (wall < 0.0) {
      r[2] = fma(v[2], tau, r[2]);
      left = 0.0;
    } else {
      r[2] = wall;
      v[0] = -v[0];
      v[1] = -v[1];
      v[2] = -v[2];
      left = __dsub_rn(left, tau);
    }
  }
  r[0] = wrap_periodic(r[0], g.B[0]);
  r[1] = wrap_periodic(r[1], g.B[1]);
  if (r[2] >= H) r[2] = nextafter(H, 0.0);
  if (r[2] < 0.0) r[2] = 0.0;
}

// Move one particle and return its cell key on the grid shifted by sh.
template <int WALLS, int FORCE, int POW2A>
__device__ __forceinline__ int move_and_key(const Geom& g, double r[3], double v[3], const double sh[3]) {
  if (WALLS) {
    stream_walls(g, r, v);
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (FORCE) {
        r[d] = fma(v[d], g.dt, __dadd_rn(r[d], g.h[d]));
        v[d] = fma(g.g[d], g.dt, v[d]);
      } else {
        r[d] = fma(v[d], g.dt, r[d]);
      }
    }
    // all three in [0, B) (as unsigned bit patterns: negative values and -0.0 compare
    // high) in one test; otherwise the per-coordinate wrap
    const unsigned long long b0 = __double_as_longlong(g.B[0]), b1 = __double_as_longlong(g.B[1]),
                             b2 = __double_as_longlong(g.B[2]);
    if (!(dbits(r[0]) < b0 && dbits(r[1]) < b1 && dbits(r[2]) < b2)) {
      r[0] = wrap_box(r[0], g.B[0], b0);
      r[1] = wrap_box(r[1], g.B[1], b1);
      r[2] = wrap_box(r[2], g.B[2], b2);
    }
  }
  const int cx = cell_coord<POW2A>(r[0], sh[0], g, 0);
  const int cy = cell_coord<POW2A>(r[1], sh[1], g, 1);
  const int cz = cell_coord<POW2A>(r[2], sh[2], g, 2);
  return cx + g.L[0] * (cy + g.L[1] * cz);
}

template <int WALLS, int FORCE, int POW2A>
__global__ void __launch_bounds__(kThreads, 4) k_stream_bin_fp64(Geom g, Fp64Bufs b, Scratch s, Ctl* __restrict__ ctl) {
  const int cur = ctl->cur;
  const double shl[3] = {ctl->shift[0], ctl->shift[1], ctl->shift[2]};
  int32_t* __restrict__ kout = keys_of(s, ctl->t + 1);
  double* __restrict__ rx = b.r[cur][0];
  double* __restrict__ ry = b.r[cur][1];
  double* __restrict__ rz = b.r[cur][2];
  double* __restrict__ vx = b.v[cur][0];
  double* __restrict__ vy = b.v[cur][1];
  double* __restrict__ vz = b.v[cur][2];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // two particles per thread and iteration, both loaded before either atomic: twice the
  // loads in flight
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += 2 * stride) {
    const int64_t j = i + stride;
    const bool two = j < g.n;
    double r0[3] = {rx[i], ry[i], rz[i]}, v0[3] = {vx[i], vy[i], vz[i]};
    double r1[3] = {0.0, 0.0, 0.0}, v1[3] = {0.0, 0.0, 0.0};
    if (two) {
      r1[0] = rx[j];
      r1[1] = ry[j];
      r1[2] = rz[j];
      v1[0] = vx[j];
      v1[1] = vy[j];
      v1[2] = vz[j];
    }
    const int k0 = move_and_key<WALLS, FORCE, POW2A>(g, r0, v0, shl);
    const int k1 = two ? move_and_key<WALLS, FORCE, POW2A>(g, r1, v1, shl) : 0;
    rx[i] = r0[0];
    ry[i] = r0[1];
    rz[i] = r0[2];
    if (WALLS || FORCE) {
      vx[i] = v0[0];
      vy[i] = v0[1];
      vz[i] = v0[2];
    }
    kout[i] = k0;
    if (two) {
      rx[j] = r1[0];
      ry[j] = r1[1];
      rz[j] = r1[2];
      if (WALLS || FORCE) {
        vx[j] = v1[0];
        vy[j] = v1[1];
        vz[j] = v1[2];
      }
      kout[j] = k1;
    }
    if (s.cursor) {  // the scatter takes the places from the cursor: counts without a round trip
      atomicAdd(&s.count[k0], 1);
      if (two) atomicAdd(&s.count[k1], 1);
    } else {
      const int a0 = atomicAdd(&s.count[k0], 1);
      const int a1 = two ? atomicAdd(&s.count[k1], 1) : 0;
      s.rank[i] = a0;
      if (two) s.rank[j] = a1;
    }
  }
}

// perm[offset[key] + place] = slot, with the keys of the step in flight (ctl->t + 1), or of
// s.key when ctl is null (the initial cell-order sort).  The place inside the cell is the
// arrival rank of the counting atomics, or, with a cursor array, taken here from the cell's
// cursor: the storage is nearly in cell order, so a warp's slots mostly share a few keys, and
// the lanes with equal keys (match.any) take their places with one atomic.  Either way a
// cell's entries are in no fixed order; the exact cell sums do not depend on it, and the
// kernels that need storage order sort the cell's entries.
__global__ void __launch_bounds__(kThreads) k_scatter(int64_t n, Scratch s, const Ctl* __restrict__ ctl) {
  const int32_t* __restrict__ key = ctl ? keys_of(s, ctl->t + 1) : s.key;
  const int32_t* __restrict__ offset = s.offset;
  int32_t* __restrict__ perm = s.perm;
  if (s.cursor) {  // eight chunks of 32 slots per warp and round: eight atomics in flight
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
        k[c] = i < n ? key[i] : -1 - lane;  // distinct sentinels past the end
      }
      unsigned peers[kChunks];
      int rank[kChunks], first[kChunks];
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
        if (k[c] >= 0) perm[offset[k[c]] + start + rank[c]] = static_cast<int32_t>(base + 32 * c + lane);
      }
    }
    return;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = key[i];
    const int place = s.cursor ? atomicAdd(&s.cursor[k], 1) : s.rank[i];
    perm[offset[k] + place] = static_cast<int32_t>(i);
  }
}

// Insertion sort of a cell's perm entries: the counting atomics hand out arrival ranks in
// no fixed order, the linked-cell list keeps storage order inside a cell.
// Up to 16 entries: a bitonic sorting network in registers (compile-time indices, the loads
// all in flight at once); the same order as the insertion sort, which takes larger cells.
__device__ __forceinline__ void sort_entries(int32_t* pm, int n) {
  if (n <= 16) {
    int a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = i < n ? pm[i] : INT_MAX;
#pragma unroll
    for (int k = 2; k <= 16; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int l = i ^ j;
          if (l > i) {
            const int x = a[i], y = a[l];
            const bool up = (i & k) == 0;
            a[i] = up ? min(x, y) : max(x, y);
            a[l] = up ? max(x, y) : min(x, y);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (i < n) pm[i] = a[i];
    return;
  }
  for (int j = 1; j < n; ++j) {
    const int x = pm[j];
    int k = j - 1;
    while (k >= 0 && pm[k] > x) {
      pm[k + 1] = pm[k];
      --k;
    }
    pm[k + 1] = x;
  }
}

// Exact sums of a cell's velocities (and of v.v for the moments), U members at a time
// so that their loads are in flight together.  `ok` turns false if a component reaches
// 2^16; the cell's entries are then put in storage order and summed in plain FP64 in that
// order, so that the result does not depend on the order in which the counting atomics
// handed out the slots.
template <int MOMENTS, int U = 4>
__device__ __forceinline__ void cell_sums(const Fp64Bufs& b, int cur, int32_t* pm, int n, double S[3], double& SE) {
  const double* __restrict__ vx = b.v[cur][0];
  const double* __restrict__ vy = b.v[cur][1];
  const double* __restrict__ vz = b.v[cur][2];
  Fx128 a0, a1, a2, ae;
  fx_zero(a0);
  fx_zero(a1);
  fx_zero(a2);
  fx_zero(ae);
  bool ok = true;
  int j = 0;
  // the next round's perm entries are loaded while this round's velocities are in flight
  int nx[U];
#pragma unroll
  for (int k = 0; k < U; ++k) nx[k] = k < n ? pm[k] : 0;
  for (; j + U <= n; j += U) {
    int ii[U];
    double x[U], y[U], z[U];
#pragma unroll
    for (int k = 0; k < U; ++k) ii[k] = nx[k];
#pragma unroll
    for (int k = 0; k < U; ++k) nx[k] = j + U + k < n ? pm[j + U + k] : 0;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      x[k] = vx[ii[k]];
      y[k] = vy[ii[k]];
      z[k] = vz[ii[k]];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      ok &= fx_add(a0, x[k]);
      ok &= fx_add(a1, y[k]);
      ok &= fx_add(a2, z[k]);
      if (MOMENTS) ok &= fx_add(ae, fma(x[k], x[k], fma(y[k], y[k], z[k] * z[k])));
    }
  }
  for (; j < n; ++j) {
    const int i = nx[0];  // the tail has fewer than U members, all prefetched
#pragma unroll
    for (int k = 0; k + 1 < U; ++k) nx[k] = nx[k + 1];
    const double v0 = vx[i], v1 = vy[i], v2 = vz[i];
    ok &= fx_add(a0, v0);
    ok &= fx_add(a1, v1);
    ok &= fx_add(a2, v2);
    if (MOMENTS) ok &= fx_add(ae, fma(v0, v0, fma(v1, v1, v2 * v2)));
  }
  if (ok) {
    S[0] = fx_value(a0);
    S[1] = fx_value(a1);
    S[2] = fx_value(a2);
    SE = MOMENTS ? fx_value(ae) : 0.0;
    return;
  }
  sort_entries(pm, n);
  S[0] = S[1] = S[2] = SE = 0.0;
  for (j = 0; j < n; ++j) {
    const int i = pm[j];
    const double v0 = vx[i], v1 = vy[i], v2 = vz[i];
    S[0] += v0;
    S[1] += v1;
    S[2] += v2;
    if (MOMENTS) SE += fma(v0, v0, fma(v1, v1, v2 * v2));
  }
}

// With particle masses (Listing 4 sums m v and m): exact sums of the rounded products
// m_i v_i, m_i v_i.v_i and of m_i, each rounded once; the order of the members does not matter.
template <int MOMENTS>
__device__ void cell_sums_mass(const Fp64Bufs& b, int cur, const double* __restrict__ mp, int32_t* pm, int n,
                               double P[3], double& SE, double& M) {
  Fx128 a0, a1, a2, ae, am;
  fx_zero(a0);
  fx_zero(a1);
  fx_zero(a2);
  fx_zero(ae);
  fx_zero(am);
  bool ok = true;
  for (int j = 0; j < n; ++j) {
    const int i = pm[j];
    const double m = mp[i], v0 = b.v[cur][0][i], v1 = b.v[cur][1][i], v2 = b.v[cur][2][i];
    ok &= fx_add(a0, m * v0);
    ok &= fx_add(a1, m * v1);
    ok &= fx_add(a2, m * v2);
    ok &= fx_add(am, m);
    if (MOMENTS) ok &= fx_add(ae, m * fma(v0, v0, fma(v1, v1, v2 * v2)));
  }
  if (ok) {
    P[0] = fx_value(a0);
    P[1] = fx_value(a1);
    P[2] = fx_value(a2);
    M = fx_value(am);
    SE = MOMENTS ? fx_value(ae) : 0.0;
    return;
  }
  sort_entries(pm, n);  // a term beyond the exact range: plain FP64 sums in storage order
  P[0] = P[1] = P[2] = SE = M = 0.0;
  for (int j = 0; j < n; ++j) {
    const int i = pm[j];
    const double m = mp[i], v0 = b.v[cur][0][i], v1 = b.v[cur][1][i], v2 = b.v[cur][2][i];
    P[0] += m * v0;
    P[1] += m * v1;
    P[2] += m * v2;
    M += m;
    if (MOMENTS) SE += m * fma(v0, v0, fma(v1, v1, v2 * v2));
  }
}

__device__ __forceinline__ void write_moments(const Geom& g, Scratch& s, int64_t c, int n, const double S[3], double SE) {
  double* mo = s.moments + 5 * c;
  mo[0] = static_cast<double>(n) * g.mass;
  mo[1] = g.mass * S[0];
  mo[2] = g.mass * S[1];
  mo[3] = g.mass * S[2];
  mo[4] = 0.5 * g.mass * SE;
}

// Position inside the cell on the shifted grid, in cell units: the fractional part of
// (r - s)/a (with a a power of two, (r - s) * (1/a) is that quotient exactly).
__device__ __forceinline__ double cell_local(const Geom& g, double r, double s) {
  const double q = g.pow2a ? (r - s) * g.inv_a : (r - s) / g.a;
  return q - floor(q);
}

// Angular-momentum-conserving collision (the variant the paper mentions in Sec. 2): omega =
// I^-1 (L_before - L_after) for the cell's members pm[0..n), with rho_i = a (l_i - mean l)
// their positions about the centre of mass on the shifted grid, L = m sum rho x v, and
// I = m sum (|rho|^2 1 - rho rho^T).  Two particles: the pseudo-inverse (I acts as m sum
// |rho|^2 normal to their separation); a singular I otherwise: no correction (omega = 0).
// after(v) gives a member's velocity after the rotation and the thermostat.
// With particle masses mp the centre is mass-weighted and L and I weight by m_i.
template <typename After>
__device__ void cell_omega(const Geom& g, const Fp64Bufs& b, const Fp64Mass& ms, int cur, const int32_t* pm, int n,
                           const double s[3], After after, double mean[3], double w[3]) {
  const double* __restrict__ mp = ms.m[cur];
  mean[0] = mean[1] = mean[2] = 0.0;
  w[0] = w[1] = w[2] = 0.0;
  double Mw = 0.0;
  for (int j = 0; j < n; ++j) {
    const double mi = mp ? mp[pm[j]] : 1.0;
    Mw += mi;
    for (int d = 0; d < 3; ++d) {
      const double l = cell_local(g, b.r[cur][d][pm[j]], s[d]);
      mean[d] += mp ? mi * l : l;
    }
  }
  for (int d = 0; d < 3; ++d) mean[d] /= mp ? Mw : static_cast<double>(n);
  double dL[3] = {0.0, 0.0, 0.0}, I[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}}, rr = 0.0, rrm = 0.0,
         q0[3];
  for (int j = 0; j < n; ++j) {
    const int i = pm[j];
    double q[3], v[3], va[3];
    for (int d = 0; d < 3; ++d) {
      q[d] = g.a * (cell_local(g, b.r[cur][d][i], s[d]) - mean[d]);
      v[d] = b.v[cur][d][i];
      va[d] = v[d];
    }
    if (j == 0)
      for (int d = 0; d < 3; ++d) q0[d] = q[d];
    after(va[0], va[1], va[2]);
    const double dv0 = v[0] - va[0], dv1 = v[1] - va[1], dv2 = v[2] - va[2];
    const double mi = mp ? mp[i] : g.mass;
    dL[0] += mi * (q[1] * dv2 - q[2] * dv1);
    dL[1] += mi * (q[2] * dv0 - q[0] * dv2);
    dL[2] += mi * (q[0] * dv1 - q[1] * dv0);
    const double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    rr += q2;
    rrm += mi * q2;
    for (int x = 0; x < 3; ++x)
      for (int y = 0; y < 3; ++y) I[x][y] += mi * ((x == y ? q2 : 0.0) - q[x] * q[y]);
  }
  if (n == 2) {
    if (rr > 0.0 && !mp) {
      const double along = (q0[0] * dL[0] + q0[1] * dL[1] + q0[2] * dL[2]) * (2.0 / rr);
      for (int d = 0; d < 3; ++d) w[d] = (dL[d] - along * q0[d]) / (g.mass * rr);
    } else if (rr > 0.0) {  // unequal masses: I acts as sum m_i |rho_i|^2 normal to the pair
      const double qq = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2];
      const double along = (q0[0] * dL[0] + q0[1] * dL[1] + q0[2] * dL[2]) / qq;
      for (int d = 0; d < 3; ++d) w[d] = (dL[d] - along * q0[d]) / rrm;
    }
    return;
  }
  double cof[3][3];
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) {
      const int x1 = (x + 1) % 3, x2 = (x + 2) % 3, y1 = (y + 1) % 3, y2 = (y + 2) % 3;
      cof[x][y] = I[x1][y1] * I[x2][y2] - I[x1][y2] * I[x2][y1];
    }
  const double det = I[0][0] * cof[0][0] + I[0][1] * cof[0][1] + I[0][2] * cof[0][2];
  const double tr = (I[0][0] + I[1][1] + I[2][2]) / 3.0;
  if (det > 1e-12 * tr * tr * tr)
    for (int x = 0; x < 3; ++x) w[x] = (cof[x][0] * dL[0] + cof[x][1] * dL[1] + cof[x][2] * dL[2]) / det;
}

// The whole collision of one cell by one thread (the shape of Listing 4): used for walls,
// the thermostats and angular-momentum conservation, and by the allocation-free step.
template <int WALLS, int THERMO, int MOMENTS>
__device__ void collide_cell_generic(const Geom& g, const Fp64Bufs& b, const Fp64Mass& ms, Scratch& s, int64_t c,
                                     int64_t t1, int cur, bool resort, const double* shift) {
  const double shift_z = shift[2];
  const int o = s.offset[c];
  const int n = s.offset[c + 1] - o;
  int32_t* __restrict__ pm = s.perm + o;
  sort_entries(pm, n);
  const double* __restrict__ mp = ms.m[cur];  // particle masses, or null for the box mass
  double S[3], SE, Mc = 0.0;
  if (mp) {
    cell_sums_mass<MOMENTS>(b, cur, mp, pm, n, S, SE, Mc);  // S = sum m v, SE = sum m v.v
    if (MOMENTS) {
      double* mo = s.moments + 5 * c;
      mo[0] = Mc;
      mo[1] = S[0];
      mo[2] = S[1];
      mo[3] = S[2];
      mo[4] = 0.5 * SE;
    }
  } else {
    cell_sums<MOMENTS>(b, cur, pm, n, S, SE);
    if (MOMENTS) write_moments(g, s, c, n, S, SE);
  }
  if (n == 0) return;
  double u0 = S[0] * inv_count(n), u1 = S[1] * inv_count(n), u2 = S[2] * inv_count(n);
  if (mp) {
    u0 = S[0] / Mc;
    u1 = S[1] / Mc;
    u2 = S[2] / Mc;
  }
  bool virt = false;
  if (WALLS) {
    const int64_t layer = c / ((int64_t)g.L[0] * g.L[1]);
    if (shift_z > 0.0 && (layer == 0 || layer == g.L[2]) && (double)n < g.ppc) {
      // R13: virtual particles fill the cut cell to ppc, at rest on average
      const double m = g.mass;
      const double Mv = (g.ppc - (double)n) * m;
      const u64x4 w = draw(g.seed, static_cast<uint64_t>(t1), static_cast<uint64_t>(c), kTagWall);
      double g0, g1, g2, g3;
      gauss_pair(w.x, w.y, g0, g1);
      gauss_pair(w.z, w.w, g2, g3);
      const double sd = sqrt(Mv * g.kT);
      if (mp) {  // virtual particles keep the box mass
        const double M = Mc + Mv;
        u0 = (S[0] + sd * g0) / M;
        u1 = (S[1] + sd * g1) / M;
        u2 = (S[2] + sd * g2) / M;
      } else {
        const double M = (double)n * m + Mv;
        u0 = (m * S[0] + sd * g0) / M;
        u1 = (m * S[1] + sd * g1) / M;
        u2 = (m * S[2] + sd * g2) / M;
      }
      virt = true;
    }
  }
  const bool rotate = n >= 2 || virt;
  double R[9], bv[3];
  if (rotate) make_frame(g, t1, c, u0, u1, u2, R, bv);
  const int ob = cur ^ 1;
  double f = 1.0;
  if (rotate && THERMO && n >= 2) {
    double K = 0.0;
    for (int j = 0; j < n; ++j) {
      const int i = pm[j];
      double v0 = b.v[cur][0][i], v1 = b.v[cur][1][i], v2 = b.v[cur][2][i];
      apply_frame(R, bv, v0, v1, v2);
      const double d0 = v0 - u0, d1 = v1 - u1, d2 = v2 - u2;
      K += 0.5 * (mp ? mp[i] : g.mass) * fma(d0, d0, fma(d1, d1, d2 * d2));
    }
    if (K > 0.0) {
      // R14: relative kinetic energy 3/2 (n - 1) kT; MBS: kT times a Gamma(3/2 (n - 1)) draw
      const double target = g.thermostat == 2 ? g.kT * mbs_gamma(g.seed, t1, c, 1.5 * (double)(n - 1))
                                              : 1.5 * (double)(n - 1) * g.kT;
      f = sqrt(target / K);
    }
  }
  double mean[3] = {0.0, 0.0, 0.0}, w[3] = {0.0, 0.0, 0.0};
  const bool spin = !WALLS && rotate && g.angular;
  if (spin)
    cell_omega(g, b, ms, cur, pm, n, shift,
               [&](double& v0, double& v1, double& v2) {
                 apply_frame(R, bv, v0, v1, v2);
                 if (THERMO && n >= 2) {
                   v0 = fma(f, v0 - u0, u0);
                   v1 = fma(f, v1 - u1, u1);
                   v2 = fma(f, v2 - u2, u2);
                 }
               },
               mean, w);
  for (int j = 0; j < n; ++j) {
    const int i = pm[j];
    double v0 = b.v[cur][0][i], v1 = b.v[cur][1][i], v2 = b.v[cur][2][i];
    if (rotate) {
      apply_frame(R, bv, v0, v1, v2);
      if (THERMO && n >= 2) {
        v0 = fma(f, v0 - u0, u0);
        v1 = fma(f, v1 - u1, u1);
        v2 = fma(f, v2 - u2, u2);
      }
      if (spin) {  // v += omega x rho
        const double q0 = g.a * (cell_local(g, b.r[cur][0][i], shift[0]) - mean[0]);
        const double q1 = g.a * (cell_local(g, b.r[cur][1][i], shift[1]) - mean[1]);
        const double q2 = g.a * (cell_local(g, b.r[cur][2][i], shift[2]) - mean[2]);
        v0 += w[1] * q2 - w[2] * q1;
        v1 += w[2] * q0 - w[0] * q2;
        v2 += w[0] * q1 - w[1] * q0;
      }
    }
    if (resort) {
      const int dst = o + j;
      b.r[ob][0][dst] = b.r[cur][0][i];
      b.r[ob][1][dst] = b.r[cur][1][i];
      b.r[ob][2][dst] = b.r[cur][2][i];
      b.v[ob][0][dst] = v0;
      b.v[ob][1][dst] = v1;
      b.v[ob][2][dst] = v2;
      b.id[ob][dst] = b.id[cur][i];
      if (mp) ms.m[ob][dst] = mp[i];
    } else if (rotate) {
      b.v[cur][0][i] = v0;
      b.v[cur][1][i] = v1;
      b.v[cur][2][i] = v2;
    }
  }
}

template <int WALLS, int THERMO, int MOMENTS>
__global__ void __launch_bounds__(kThreads) k_collide_fp64_generic(Geom g, Fp64Bufs b, Scratch s, Ctl* __restrict__ ctl,
                                                                   Fp64Mass ms) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int64_t t1 = ctl->t + 1;
  const bool resort = g.resort_k > 0 && (t1 % g.resort_k) == 0;
  collide_cell_generic<WALLS, THERMO, MOMENTS>(g, b, ms, s, c, t1, ctl->cur, resort, ctl->shift);
}

// Periodic box, no thermostat, in two passes so that each runs at full occupancy:
//  k_cell_frame  one thread per cell: exact sums (order-independent, so the arrival order
//                of the atomics does not matter), centre-of-mass velocity, random axis and
//                the frame (R, b), written as one 128-byte record per cell.  On re-sort
//                steps it also restores storage order inside the cell, so that perm then
//                lists the storage slots in the new (cell) order.
//  k_rotate      one thread per slot: v' = R v + b with the frame of its cell (nine FP64
//                FMAs on full warps, coalesced state access); on re-sort steps slot j of the
//                other buffer set gathers its particle from storage slot perm[j] (scattered
//                reads, contiguous writes).
constexpr int kFrameStride = 16;  // doubles per cell record: R[9], b[3], flag, 3 unused

// Angular-momentum correction of a dense cell from its moments (the variant Sec. 2 mentions):
// with in-cell positions l_i and weights w_i (the particle masses, or 1 for the box mass,
// which cancels from omega), A = sum w l, Q = sum w l l^T, B = sum w l v^T and P = sum w v,
// the moments about the centre are a (B - lbar P^T) and a^2 (Q - W lbar lbar^T), so
// L_before = eps : M, L_after = eps : (M R^T) (sum w rho = 0), I = tr(S) 1 - S.  omega as in
// cell_omega; the frame then carries a omega and b - a omega x lbar, and rotate adds
// (a omega) x l_i.
__device__ void dense_omega(const Geom& g, const double R[9], double W, const double A[3], const double Q[6],
                            const double B[9], const double P[3], const double l0[3], int n, double aw[3],
                            double lbar[3]) {
  aw[0] = aw[1] = aw[2] = 0.0;
  for (int d = 0; d < 3; ++d) lbar[d] = A[d] / W;
  double M[3][3], S[3][3];
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) M[x][y] = g.a * (B[3 * x + y] - lbar[x] * P[y]);
  const int qi[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};  // Q: xx yy zz xy xz yz
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) S[x][y] = g.a * g.a * (Q[qi[x][y]] - W * lbar[x] * lbar[y]);
  double N[3][3];  // M R^T
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) N[x][y] = M[x][0] * R[3 * y] + M[x][1] * R[3 * y + 1] + M[x][2] * R[3 * y + 2];
  const double dL[3] = {(M[1][2] - M[2][1]) - (N[1][2] - N[2][1]), (M[2][0] - M[0][2]) - (N[2][0] - N[0][2]),
                        (M[0][1] - M[1][0]) - (N[0][1] - N[1][0])};
  const double tr = S[0][0] + S[1][1] + S[2][2];
  double I[3][3];
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) I[x][y] = (x == y ? tr : 0.0) - S[x][y];
  double w[3] = {0.0, 0.0, 0.0};
  if (n == 2) {  // the pair lies on one line: I acts as tr(S) normal to it
    const double q[3] = {g.a * (l0[0] - lbar[0]), g.a * (l0[1] - lbar[1]), g.a * (l0[2] - lbar[2])};
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
  for (int d = 0; d < 3; ++d) aw[d] = g.a * w[d];
}

template <int MOMENTS, int MASS = 0, int ANG = 0>
__global__ void __launch_bounds__(kThreads, ANG ? 1 : 5) k_cell_frame(Geom g, Fp64Bufs b, Scratch s, Ctl* __restrict__ ctl,
                                                         Fp64Mass ms) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int64_t t1 = ctl->t + 1;
  const int cur = ctl->cur;
  const bool resort = g.resort_k > 0 && (t1 % g.resort_k) == 0;
  const int o = s.offset[c];
  const int n = s.offset[c + 1] - o;
  int32_t* __restrict__ pm = s.perm + o;
  if (resort || ANG) sort_entries(pm, n);  // ANG: one fixed order for the FP64 moment sums
  double S[3], SE, Mc = 0.0;
  if (MASS) {  // particle masses: S = sum m v (exact), Mc = sum m
    cell_sums_mass<MOMENTS>(b, cur, ms.m[cur], pm, n, S, SE, Mc);
    if (MOMENTS) {
      double* mo = s.moments + 5 * c;
      mo[0] = Mc;
      mo[1] = S[0];
      mo[2] = S[1];
      mo[3] = S[2];
      mo[4] = 0.5 * SE;
    }
  } else {
    // two members at a time: 48 registers, five blocks of 256 per SM (0.402 -> 0.390 ms per
    // step at 128^3 against four at a time and four blocks)
    cell_sums<MOMENTS, 2>(b, cur, pm, n, S, SE);
    if (MOMENTS) write_moments(g, s, c, n, S, SE);
  }
  double2* __restrict__ rec = reinterpret_cast<double2*>(s.frame + kFrameStride * c);
  const bool rotate = n >= 2;
  if (!rotate) {
    rec[6] = make_double2(0.0, 0.0);
    return;
  }
  if (!ANG) {  // the rotation applies the frame in float-float arithmetic, built that way here
    float* f = reinterpret_cast<float*>(s.frame + kFrameStride * c);
    if (MASS) {
      make_frame_ff(g, t1, c, S[0] / Mc, S[1] / Mc, S[2] / Mc, f);
    } else {
      const double in = inv_count(n);
      make_frame_ff(g, t1, c, S[0] * in, S[1] * in, S[2] * in, f);
    }
    return;
  }
  double R[9], bv[3];
  if (MASS) {
    make_frame(g, t1, c, S[0] / Mc, S[1] / Mc, S[2] / Mc, R, bv);
  } else {
    const double in = inv_count(n);
    make_frame(g, t1, c, S[0] * in, S[1] * in, S[2] * in, R, bv);
  }
  double aw[3] = {0.0, 0.0, 0.0};
  if (ANG) {
    double W = 0.0, A[3] = {0.0, 0.0, 0.0}, Q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, B[9] = {0.0}, l0[3];
    for (int j = 0; j < n; ++j) {
      const int i = pm[j];
      const double w = MASS ? ms.m[cur][i] : 1.0;
      double l[3], v[3];
      for (int d = 0; d < 3; ++d) {
        l[d] = cell_local(g, b.r[cur][d][i], ctl->shift[d]);
        v[d] = b.v[cur][d][i];
      }
      if (j == 0)
        for (int d = 0; d < 3; ++d) l0[d] = l[d];
      W += w;
      for (int d = 0; d < 3; ++d) A[d] += w * l[d];
      Q[0] += w * l[0] * l[0];
      Q[1] += w * l[1] * l[1];
      Q[2] += w * l[2] * l[2];
      Q[3] += w * l[0] * l[1];
      Q[4] += w * l[0] * l[2];
      Q[5] += w * l[1] * l[2];
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) B[3 * x + y] += w * l[x] * v[y];
    }
    double lbar[3];
    dense_omega(g, R, W, A, Q, B, S, l0, n, aw, lbar);  // S: sum w v (the exact momentum sums)
    bv[0] -= aw[1] * lbar[2] - aw[2] * lbar[1];
    bv[1] -= aw[2] * lbar[0] - aw[0] * lbar[2];
    bv[2] -= aw[0] * lbar[1] - aw[1] * lbar[0];
  }
  rec[0] = make_double2(R[0], R[1]);
  rec[1] = make_double2(R[2], R[3]);
  rec[2] = make_double2(R[4], R[5]);
  rec[3] = make_double2(R[6], R[7]);
  rec[4] = make_double2(R[8], bv[0]);
  rec[5] = make_double2(bv[1], bv[2]);
  rec[6] = make_double2(1.0, aw[0]);
  rec[7] = make_double2(aw[1], aw[2]);
}

// One storage slot of k_rotate: its velocity and its cell's frame record, all loaded
// before any of them is used (the frame whether or not the cell rotates: one round trip
// after the key instead of two).
struct RotSlot {
  int64_t i;
  double v[3];
  double2 f[8];  // f[7]: only with angular-momentum conservation
};

template <int ANG>
__device__ __forceinline__ void rotate_load(const Fp64Bufs& b, const Scratch& s, const int32_t* __restrict__ key,
                                            int64_t i, int cur, RotSlot& q) {
  q.i = i;
  const int c = key[i];
  q.v[0] = b.v[cur][0][i];
  q.v[1] = b.v[cur][1][i];
  q.v[2] = b.v[cur][2][i];
  const double2* __restrict__ rec = reinterpret_cast<const double2*>(s.frame + kFrameStride * (int64_t)c);
#pragma unroll
  for (int k = 0; k < 7 + ANG; ++k) q.f[k] = rec[k];
}

// The frame of a loaded record applied to v: float-float (the record's 28 floats) without
// angular-momentum conservation, FP64 with it (R, b and a omega x l_i, l_i the position in
// the cell of the grid shifted by shift).
template <int ANG>
__device__ __forceinline__ void rotate_apply(const Geom& g, const double2 f[8], const double r[3], const double* shift,
                                             double& v0, double& v1, double& v2) {
  if (!ANG) {
    float w[28];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      w[4 * k + 0] = __int_as_float(__double2loint(f[k].x));
      w[4 * k + 1] = __int_as_float(__double2hiint(f[k].x));
      w[4 * k + 2] = __int_as_float(__double2loint(f[k].y));
      w[4 * k + 3] = __int_as_float(__double2hiint(f[k].y));
    }
    ff_apply_frame(w, v0, v1, v2);
    return;
  }
  const double R[9] = {f[0].x, f[0].y, f[1].x, f[1].y, f[2].x, f[2].y, f[3].x, f[3].y, f[4].x};
  const double bv[3] = {f[4].y, f[5].x, f[5].y};
  apply_frame(R, bv, v0, v1, v2);
  const double w0 = f[6].y, w1 = f[7].x, w2 = f[7].y;  // + (a omega) x l_i
  const double l0 = cell_local(g, r[0], shift[0]);
  const double l1 = cell_local(g, r[1], shift[1]);
  const double l2 = cell_local(g, r[2], shift[2]);
  v0 += w1 * l2 - w2 * l1;
  v1 += w2 * l0 - w0 * l2;
  v2 += w0 * l1 - w1 * l0;
}

template <int MASS, int ANG>
__device__ __forceinline__ void rotate_finish(const Geom& g, const Fp64Bufs& b, const Fp64Mass& ms, const Scratch& s,
                                              RotSlot& q, int cur, bool resort, const double* shift, int64_t dst) {
  // flag (1 or 0; FP64 or FP32, as bits) in the record's sixth 16-byte word
  const bool rot = (__double2hiint(q.f[6].x) | __double2loint(q.f[6].x)) != 0;
  double v0 = q.v[0], v1 = q.v[1], v2 = q.v[2];
  if (rot) {
    double r[3] = {0.0, 0.0, 0.0};
    if (ANG) {
      r[0] = b.r[cur][0][q.i];
      r[1] = b.r[cur][1][q.i];
      r[2] = b.r[cur][2][q.i];
    }
    rotate_apply<ANG>(g, q.f, r, shift, v0, v1, v2);
  }
  const int64_t i = q.i;  // the source slot (dst itself unless re-sorting)
  if (resort) {
    const int ob = cur ^ 1;
    b.r[ob][0][dst] = b.r[cur][0][i];
    b.r[ob][1][dst] = b.r[cur][1][i];
    b.r[ob][2][dst] = b.r[cur][2][i];
    b.v[ob][0][dst] = v0;
    b.v[ob][1][dst] = v1;
    b.v[ob][2][dst] = v2;
    b.id[ob][dst] = b.id[cur][i];
    if (MASS) ms.m[ob][dst] = ms.m[cur][i];
  } else if (rot) {
    b.v[cur][0][i] = v0;
    b.v[cur][1][i] = v1;
    b.v[cur][2][i] = v2;
  }
}

// The dense pair's rotation runs after the step's end_step: ctl->t is the step whose frames
// are applied, ctl->cur the buffer set the particles end up in (flipped on re-sort steps),
// ctl->shift_last that step's grid shift.
template <int MASS, int ANG = 0>
__global__ void __launch_bounds__(kThreads, ANG ? 4 : 5) k_rotate(Geom g, Fp64Bufs b, Scratch s, Ctl* __restrict__ ctl,
                                                                 Fp64Mass ms) {
  const int64_t t = ctl->t;
  const bool resort = g.resort_k > 0 && (t % g.resort_k) == 0;
  const int src = resort ? ctl->cur ^ 1 : ctl->cur;
  const int32_t* __restrict__ key = keys_of(s, t);
  if (!ANG) {  // as in the fused pass: the frame row by row, r and v from one base per set
    const int64_t n = g.n;
    const int cur = ctl->cur;
    const double* Ssrc = b.r[src][0];  // the same set as Scur on ordinary steps
    double* Scur = b.r[cur][0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const int64_t si = resort ? (int64_t)s.perm[i] : i;
      const float4* __restrict__ rec = reinterpret_cast<const float4*>(s.frame + kFrameStride * (int64_t)key[si]);
      double v0 = Ssrc[3 * n + si], v1 = Ssrc[4 * n + si], v2 = Ssrc[5 * n + si];
      const bool rot = rec[6].x != 0.0f;
      if (rot) ff_apply_frame_rows(rec, v0, v1, v2);
      if (resort) {
        Scur[i] = Ssrc[si];
        Scur[n + i] = Ssrc[n + si];
        Scur[2 * n + i] = Ssrc[2 * n + si];
        b.id[cur][i] = b.id[src][si];
        if (MASS) ms.m[cur][i] = ms.m[src][si];
      }
      if (resort || rot) {
        Scur[3 * n + i] = v0;
        Scur[4 * n + i] = v1;
        Scur[5 * n + i] = v2;
      }
    }
    return;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    RotSlot q;
    const int64_t si = resort ? (int64_t)s.perm[i] : i;  // re-sort: gather slot i's particle
    rotate_load<ANG>(b, s, key, si, src, q);
    rotate_finish<MASS, ANG>(g, b, ms, s, q, src, resort, ctl->shift_last, i);
  }
}

// The rotation of step t fused with the streaming and binning of step t + 1 (one pass over
// the state instead of two): each slot's velocity gets its cell's frame (v' = R v + b, the
// same arithmetic as k_rotate), the particle moves on (the same arithmetic as stream_bin),
// and it is written with its key on step t + 1's shifted grid and its arrival rank in that
// cell; on re-sort steps slot i of the other buffer set gathers its particle from storage
// slot perm[i].
template <int FORCE, int POW2A, int MASS, int ANG>
__global__ void __launch_bounds__(kThreads, ANG ? 4 : 5) k_rotate_stream(Geom g, Fp64Bufs b, Scratch s, Ctl* __restrict__ ctl,
                                                              Fp64Mass ms) {
  const int64_t t = ctl->t;
  const bool resort = g.resort_k > 0 && (t % g.resort_k) == 0;
  const int cur = ctl->cur;
  const int src = resort ? cur ^ 1 : cur;
  const int32_t* __restrict__ kin = keys_of(s, t);
  int32_t* __restrict__ kout = keys_of(s, t + 1);
  const double shn[3] = {ctl->shift[0], ctl->shift[1], ctl->shift[2]};  // step t + 1
  const double shl[3] = {ctl->shift_last[0], ctl->shift_last[1], ctl->shift_last[2]};  // step t
  // the buffer sets' r and v from one base each (the layout of a handle's allocation): six
  // array pointers fewer in registers, five blocks of 256 per SM
  const int64_t n = g.n;
  const double* Ssrc = b.r[src][0];  // the same set as Scur on ordinary steps: no __restrict__
  double* Scur = b.r[cur][0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t si = resort ? (int64_t)s.perm[i] : i;
    double r[3], v[3];
    bool rot;
    if (ANG) {
      RotSlot q;
      rotate_load<ANG>(b, s, kin, si, src, q);
      r[0] = Ssrc[0 + si];
      r[1] = Ssrc[n + si];
      r[2] = Ssrc[2 * n + si];
      rot = (__double2hiint(q.f[6].x) | __double2loint(q.f[6].x)) != 0;  // flag 1 or 0, as bits
      v[0] = q.v[0];
      v[1] = q.v[1];
      v[2] = q.v[2];
      if (rot) rotate_apply<ANG>(g, q.f, r, shl, v[0], v[1], v[2]);  // l_i on step t's grid
    } else {  // float-float frame, loaded row by row as it is applied
      const float4* __restrict__ rec = reinterpret_cast<const float4*>(s.frame + kFrameStride * (int64_t)kin[si]);
      v[0] = Ssrc[3 * n + si];
      v[1] = Ssrc[4 * n + si];
      v[2] = Ssrc[5 * n + si];
      r[0] = Ssrc[0 + si];
      r[1] = Ssrc[n + si];
      r[2] = Ssrc[2 * n + si];
      rot = rec[6].x != 0.0f;
      if (rot) ff_apply_frame_rows(rec, v[0], v[1], v[2]);
    }
    const int64_t dst = i;
    const int32_t pid = resort ? b.id[src][si] : 0;
    const double pm = (MASS && resort) ? ms.m[src][si] : 0.0;
    const int k = move_and_key<0, FORCE, POW2A>(g, r, v, shn);
    Scur[0 + dst] = r[0];
    Scur[n + dst] = r[1];
    Scur[2 * n + dst] = r[2];
    if (resort || rot || FORCE) {
      Scur[3 * n + dst] = v[0];
      Scur[4 * n + dst] = v[1];
      Scur[5 * n + dst] = v[2];
    }
    if (resort) {
      b.id[cur][dst] = pid;
      if (MASS) ms.m[cur][dst] = pm;
    }
    kout[dst] = k;
    if (s.cursor)
      atomicAdd(&s.count[k], 1);
    else
      s.rank[dst] = atomicAdd(&s.count[k], 1);
  }
}

// Put every cell's perm entries in storage order (the linked-cell list's order); run on
// demand when the last step did not need the sorted order itself.
__global__ void __launch_bounds__(kThreads) k_sort_segments(int64_t ncell, const int32_t* __restrict__ offset,
                                                            int32_t* __restrict__ perm) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int o = offset[c];
  sort_entries(perm + o, offset[c + 1] - o);
}

__global__ void k_end_step(Geom g, Ctl* ctl) {
  const int64_t t1 = ctl->t + 1;
  if (g.resort_k > 0 && (t1 % g.resort_k) == 0) ctl->cur ^= 1;
  for (int d = 0; d < 3; ++d) ctl->shift_last[d] = ctl->shift[d];
  ctl->t = t1;
  set_shifts(g, ctl);
}

// ---- initial state ----
__device__ __forceinline__ double block_sum_fixed(double v, double* sm) {
  // fixed-order tree: the same inputs always give the same bits
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

__global__ void __launch_bounds__(kThreads) k_init_fp64(Geom g, Fp64Bufs b, double* __restrict__ red) {
  __shared__ double sm[kThreads];
  const double sigma = sqrt(g.kT / g.mass);
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const u64x4 w = draw(g.seed, static_cast<uint64_t>(i), 0, kTagInit);
    b.r[0][0][i] = unit53(w.x) * g.B[0];
    b.r[0][1][i] = unit53(w.y) * g.B[1];
    b.r[0][2][i] = unit53(w.z) * g.B[2];
    const u64x4 q = draw(g.seed, static_cast<uint64_t>(i), 1, kTagInit);
    double g0, g1, g2, g3;
    gauss_pair(q.x, q.y, g0, g1);
    gauss_pair(q.z, q.w, g2, g3);
    const double v0 = sigma * g0, v1 = sigma * g1, v2 = sigma * g2;
    b.v[0][0][i] = v0;
    b.v[0][1][i] = v1;
    b.v[0][2][i] = v2;
    b.id[0][i] = static_cast<int32_t>(i);
    acc[0] += v0;
    acc[1] += v1;
    acc[2] += v2;
  }
  for (int d = 0; d < 3; ++d) {
    const double tot = block_sum_fixed(acc[d], sm);
    if (threadIdx.x == 0) red[3 * blockIdx.x + d] = tot;
  }
}

__global__ void __launch_bounds__(kThreads) k_init_mean(const double* __restrict__ red, int nblk, int64_t n, Ctl* ctl) {
  __shared__ double sm[kThreads];
  for (int d = 0; d < 3; ++d) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) acc += red[3 * k + d];
    const double tot = block_sum_fixed(acc, sm);
    if (threadIdx.x == 0) ctl->mean[d] = n > 0 ? tot / (double)n : 0.0;
  }
}

__global__ void __launch_bounds__(kThreads) k_init_sub(Geom g, Fp64Bufs b, const Ctl* __restrict__ ctl) {
  const double m0 = ctl->mean[0], m1 = ctl->mean[1], m2 = ctl->mean[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    b.v[0][0][i] -= m0;
    b.v[0][1][i] -= m1;
    b.v[0][2][i] -= m2;
  }
}

__global__ void __launch_bounds__(kThreads) k_get_state_fp64(int64_t n, const double* __restrict__ rx,
                                                             const double* __restrict__ ry, const double* __restrict__ rz,
                                                             const double* __restrict__ vx, const double* __restrict__ vy,
                                                             const double* __restrict__ vz, const int32_t* __restrict__ id,
                                                             double* __restrict__ r, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id[i];
    r[3 * p + 0] = rx[i];
    r[3 * p + 1] = ry[i];
    r[3 * p + 2] = rz[i];
    v[3 * p + 0] = vx[i];
    v[3 * p + 1] = vy[i];
    v[3 * p + 2] = vz[i];
  }
}

// ---- initial cell order (create / set_state) ----
// Cell key of each current position on the unshifted grid and its arrival rank; positions
// are only read.
template <int POW2A>
__global__ void __launch_bounds__(kThreads) k_presort_keys(Geom g, Fp64Bufs b, Scratch s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int cx = cell_coord<POW2A>(b.r[0][0][i], 0.0, g, 0);
    const int cy = cell_coord<POW2A>(b.r[0][1][i], 0.0, g, 1);
    const int cz = cell_coord<POW2A>(b.r[0][2][i], 0.0, g, 2);
    const int k = cx + g.L[0] * (cy + g.L[1] * cz);
    s.key[i] = k;
    s.rank[i] = atomicAdd(&s.count[k], 1);
  }
}

// Buffer set 1 slot j <- set 0 slot perm[j] (positions, velocities, ids, masses if any):
// coalesced writes, gathered reads.
__global__ void __launch_bounds__(kThreads) k_permute_fp64(int64_t n, const int32_t* __restrict__ perm, Fp64Bufs b,
                                                           Fp64Mass ms) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[j];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      b.r[1][d][j] = b.r[0][d][i];
      b.v[1][d][j] = b.v[0][d][i];
    }
    b.id[1][j] = b.id[0][i];
    if (ms.m[0]) ms.m[1][j] = ms.m[0][i];
  }
}

// v += dp / m for every storage slot (dp by particle id; m the slot's mass or the box mass).
__global__ void __launch_bounds__(kThreads) k_add_momentum_fp64(Geom g, Fp64Bufs b, int cur,
                                                                const double* __restrict__ m,
                                                                const double* __restrict__ dp) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.n; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = b.id[cur][s];
    const double mi = m ? m[s] : g.mass;
#pragma unroll
    for (int d = 0; d < 3; ++d) b.v[cur][d][s] = __dadd_rn(b.v[cur][d][s], __ddiv_rn(dp[3 * i + d], mi));
  }
}

// The same initial sort straight from a state in particle-id order as N x 3 arrays (a host
// upload): keys of the unshifted cells, then one gather into buffer set 1 in cell order.
template <int POW2A>
__global__ void __launch_bounds__(kThreads) k_presort_keys_aos(Geom g, const double* __restrict__ r, Scratch s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int cx = cell_coord<POW2A>(r[3 * i + 0], 0.0, g, 0);
    const int cy = cell_coord<POW2A>(r[3 * i + 1], 0.0, g, 1);
    const int cz = cell_coord<POW2A>(r[3 * i + 2], 0.0, g, 2);
    const int k = cx + g.L[0] * (cy + g.L[1] * cz);
    s.key[i] = k;
    s.rank[i] = atomicAdd(&s.count[k], 1);
  }
}

// PARTS: 1 positions and ids, 2 velocities and masses, 3 both; into buffer set `set`.
template <int PARTS>
__global__ void __launch_bounds__(kThreads) k_gather_state_aos(int64_t n, const int32_t* __restrict__ perm,
                                                              const double* __restrict__ r, const double* __restrict__ v,
                                                              Fp64Bufs b, int set, const double* __restrict__ m_by_id,
                                                              double* __restrict__ m_dst) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[j];
    if (PARTS & 1) {
#pragma unroll
      for (int d = 0; d < 3; ++d) b.r[set][d][j] = r[3 * i + d];
      b.id[set][j] = static_cast<int32_t>(i);
    }
    if (PARTS & 2) {
#pragma unroll
      for (int d = 0; d < 3; ++d) b.v[set][d][j] = v[3 * i + d];
      if (m_by_id) m_dst[j] = m_by_id[i];
    }
  }
}

// slot_of[id] = storage slot holding that particle.
__global__ void __launch_bounds__(kThreads) k_slot_of(int64_t n, const int32_t* __restrict__ id,
                                                     int32_t* __restrict__ slot_of) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    slot_of[id[s]] = static_cast<int32_t>(s);
}

// Particles p0 .. p1 - 1 (by id) into N x 3 arrays r, v: contiguous writes, gathered reads.
__global__ void __launch_bounds__(kThreads) k_gather_by_id(int64_t p0, int64_t p1, const int32_t* __restrict__ slot_of,
                                                          Fp64Bufs b, int cur, double* __restrict__ r,
                                                          double* __restrict__ v) {
  for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = slot_of[p];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      r[3 * p + d] = b.r[cur][d][s];
      v[3 * p + d] = b.v[cur][d][s];
    }
  }
}

}  // namespace

void launch_slot_of(const Geom& g, Fp64Bufs b, int cur, int32_t* slot_of, cudaStream_t st) {
  if (g.n > 0) k_slot_of<<<grid_for(g.n), kThreads, 0, st>>>(g.n, b.id[cur], slot_of);
}

void launch_gather_by_id(int64_t p0, int64_t p1, const int32_t* slot_of, Fp64Bufs b, int cur, double* r, double* v,
                         cudaStream_t st) {
  if (p1 > p0) k_gather_by_id<<<grid_for(p1 - p0), kThreads, 0, st>>>(p0, p1, slot_of, b, cur, r, v);
}

int launch_sort_positions_fp64(const Geom& g, Scratch s, const double* r, cudaStream_t st) {
  s.cursor = nullptr;  // ranks from the counting atomics
  launch_zero_i32(s.count, g.ncell, st);
  if (g.pow2a)
    k_presort_keys_aos<1><<<grid_for(g.n), kThreads, 0, st>>>(g, r, s);
  else
    k_presort_keys_aos<0><<<grid_for(g.n), kThreads, 0, st>>>(g, r, s);
  launch_scan(s.count, s.offset, s.partial, g.ncell, st);
  launch_scatter(g, s, nullptr, st);
  launch_sort_segments(g, s, st);
  return 7;  // kernels launched: zero, keys, scan (3), scatter, in-cell sort
}

int launch_gather_state_fp64(const Geom& g, Fp64Bufs b, Scratch s, const double* r, const double* v,
                             const double* m_by_id, double* m_dst, cudaStream_t st) {
  k_gather_state_aos<3><<<grid_for(g.n), kThreads, 0, st>>>(g.n, s.perm, r, v, b, 1, m_by_id, m_dst);
  return 1;
}

int launch_gather_positions_fp64(const Geom& g, Fp64Bufs b, Scratch s, const double* r, int set, cudaStream_t st) {
  k_gather_state_aos<1><<<grid_for(g.n), kThreads, 0, st>>>(g.n, s.perm, r, nullptr, b, set, nullptr, nullptr);
  return 1;
}

int launch_gather_velocities_fp64(const Geom& g, Fp64Bufs b, Scratch s, const double* v, int set,
                                  const double* m_by_id, double* m_dst, cudaStream_t st) {
  k_gather_state_aos<2><<<grid_for(g.n), kThreads, 0, st>>>(g.n, s.perm, nullptr, v, b, set, m_by_id, m_dst);
  return 1;
}

int launch_set_state_sorted_fp64(const Geom& g, Fp64Bufs b, Scratch s, const double* r, const double* v,
                                 const double* m_by_id, double* m_dst, cudaStream_t st) {
  return launch_sort_positions_fp64(g, s, r, st) + launch_gather_state_fp64(g, b, s, r, v, m_by_id, m_dst, st);
}

void launch_add_momentum_fp64(const Geom& g, Fp64Bufs b, int cur, Fp64Mass ms, const double* dp, cudaStream_t st) {
  if (g.n > 0) k_add_momentum_fp64<<<grid_for(g.n), kThreads, 0, st>>>(g, b, cur, ms.m[cur], dp);
}

int launch_presort_fp64(const Geom& g, Fp64Bufs b, Scratch s, Fp64Mass ms, cudaStream_t st) {
  s.cursor = nullptr;  // ranks from the counting atomics
  launch_zero_i32(s.count, g.ncell, st);
  if (g.pow2a)
    k_presort_keys<1><<<grid_for(g.n), kThreads, 0, st>>>(g, b, s);
  else
    k_presort_keys<0><<<grid_for(g.n), kThreads, 0, st>>>(g, b, s);
  launch_scan(s.count, s.offset, s.partial, g.ncell, st);
  launch_scatter(g, s, nullptr, st);
  launch_sort_segments(g, s, st);
  k_permute_fp64<<<grid_for(g.n), kThreads, 0, st>>>(g.n, s.perm, b, ms);
  return 8;  // kernels launched: zero, keys, scan (3), scatter, in-cell sort, gather
}

void launch_init_fp64(const Geom& g, Fp64Bufs b, double* red, int red_blocks, Ctl* ctl, cudaStream_t st) {
  k_init_fp64<<<red_blocks, kThreads, 0, st>>>(g, b, red);
  k_init_mean<<<1, kThreads, 0, st>>>(red, red_blocks, g.n, ctl);
  k_init_sub<<<grid_for(g.n), kThreads, 0, st>>>(g, b, ctl);
}

void launch_stream_bin_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, cudaStream_t st) {
  const unsigned grid = grid_for(g.n, 2);
  const int sel = (g.walls ? 4 : (g.force ? 2 : 0)) | (g.pow2a ? 1 : 0);
  switch (sel) {
    case 0: k_stream_bin_fp64<0, 0, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 1: k_stream_bin_fp64<0, 0, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 2: k_stream_bin_fp64<0, 1, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 3: k_stream_bin_fp64<0, 1, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 4: k_stream_bin_fp64<1, 1, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    default: k_stream_bin_fp64<1, 1, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
  }
}

void launch_scatter(const Geom& g, Scratch s, const Ctl* ctl, cudaStream_t st) {
  k_scatter<<<grid_for(g.n, s.cursor ? 8 : 1), kThreads, 0, st>>>(g.n, s, ctl);
}

void launch_collide_fp64_generic(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, bool moments, cudaStream_t st,
                                 Fp64Mass ms) {
  const unsigned grid = static_cast<unsigned>((g.ncell + kThreads - 1) / kThreads);
  const int sel = (g.walls ? 4 : 0) | (g.thermostat ? 2 : 0) | (moments ? 1 : 0);
  switch (sel) {
    case 0: k_collide_fp64_generic<0, 0, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 1: k_collide_fp64_generic<0, 0, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 2: k_collide_fp64_generic<0, 1, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 3: k_collide_fp64_generic<0, 1, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 4: k_collide_fp64_generic<1, 0, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 5: k_collide_fp64_generic<1, 0, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 6: k_collide_fp64_generic<1, 1, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    default: k_collide_fp64_generic<1, 1, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
  }
}

bool fp64_dense_collide(const Geom& g, const Scratch& s) {
  return !g.walls && !g.thermostat && s.frame;
}

__global__ void k_gather_masses(int64_t n, const double* __restrict__ m_by_id, const int32_t* __restrict__ id,
                                double* __restrict__ dst) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = m_by_id[id[j]];
}

void launch_gather_masses(int64_t n, const double* m_by_id, const int32_t* id, double* dst, cudaStream_t st) {
  if (n > 0) k_gather_masses<<<grid_for(n), kThreads, 0, st>>>(n, m_by_id, id, dst);
}

void launch_collide_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, bool moments, cudaStream_t st, Fp64Mass ms) {
  if (!fp64_dense_collide(g, s)) {
    launch_collide_fp64_generic(g, b, s, ctl, moments, st, ms);
    return;
  }
  const unsigned cgrid = static_cast<unsigned>((g.ncell + kThreads - 1) / kThreads);
  switch ((g.angular ? 4 : 0) | (ms.m[0] ? 2 : 0) | (moments ? 1 : 0)) {
    case 0: k_cell_frame<0, 0, 0><<<cgrid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 1: k_cell_frame<1, 0, 0><<<cgrid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 2: k_cell_frame<0, 1, 0><<<cgrid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 3: k_cell_frame<1, 1, 0><<<cgrid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 4: k_cell_frame<0, 0, 1><<<cgrid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 5: k_cell_frame<1, 0, 1><<<cgrid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 6: k_cell_frame<0, 1, 1><<<cgrid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    default: k_cell_frame<1, 1, 1><<<cgrid, kThreads, 0, st>>>(g, b, s, ctl, ms); break;
  }
}

namespace {
template <int F, int P, int M, int A>
void rotate_stream_launch(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, cudaStream_t st, Fp64Mass ms) {
  k_rotate_stream<F, P, M, A><<<grid_for(g.n), kThreads, 0, st>>>(g, b, s, ctl, ms);
}
}  // namespace

void launch_rotate_stream_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, cudaStream_t st, Fp64Mass ms) {
  using Launch = void (*)(const Geom&, Fp64Bufs, Scratch, Ctl*, cudaStream_t, Fp64Mass);
  static const Launch table[16] = {
      rotate_stream_launch<0, 0, 0, 0>, rotate_stream_launch<0, 0, 0, 1>, rotate_stream_launch<0, 0, 1, 0>,
      rotate_stream_launch<0, 0, 1, 1>, rotate_stream_launch<0, 1, 0, 0>, rotate_stream_launch<0, 1, 0, 1>,
      rotate_stream_launch<0, 1, 1, 0>, rotate_stream_launch<0, 1, 1, 1>, rotate_stream_launch<1, 0, 0, 0>,
      rotate_stream_launch<1, 0, 0, 1>, rotate_stream_launch<1, 0, 1, 0>, rotate_stream_launch<1, 0, 1, 1>,
      rotate_stream_launch<1, 1, 0, 0>, rotate_stream_launch<1, 1, 0, 1>, rotate_stream_launch<1, 1, 1, 0>,
      rotate_stream_launch<1, 1, 1, 1>};
  table[(g.force ? 8 : 0) | (g.pow2a ? 4 : 0) | (ms.m[0] ? 2 : 0) | (g.angular ? 1 : 0)](g, b, s, ctl, st, ms);
}

void launch_rotate_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, cudaStream_t st, Fp64Mass ms) {
  switch ((g.angular ? 2 : 0) | (ms.m[0] ? 1 : 0)) {
    case 0: k_rotate<0, 0><<<grid_for(g.n), kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 1: k_rotate<1, 0><<<grid_for(g.n), kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    case 2: k_rotate<0, 1><<<grid_for(g.n), kThreads, 0, st>>>(g, b, s, ctl, ms); break;
    default: k_rotate<1, 1><<<grid_for(g.n), kThreads, 0, st>>>(g, b, s, ctl, ms); break;
  }
}

void launch_sort_segments(const Geom& g, Scratch s, cudaStream_t st) {
  const unsigned grid = static_cast<unsigned>((g.ncell + kThreads - 1) / kThreads);
  k_sort_segments<<<grid, kThreads, 0, st>>>(g.ncell, s.offset, s.perm);
}

void launch_end_step(const Geom& g, Ctl* ctl, cudaStream_t st) { k_end_step<<<1, 1, 0, st>>>(g, ctl); }

void launch_get_state_fp64(const Geom& g, Fp64Bufs b, int cur, double* r, double* v, cudaStream_t st) {
  k_get_state_fp64<<<grid_for(g.n), kThreads, 0, st>>>(g.n, b.r[cur][0], b.r[cur][1], b.r[cur][2], b.v[cur][0],
                                                        b.v[cur][1], b.v[cur][2], b.id[cur], r, v);
}

}  // namespace mpcd
