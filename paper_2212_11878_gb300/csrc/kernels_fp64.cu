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
#include "device_common.cuh"
#include "mpcd_internal.h"

namespace mpcd {

namespace {
constexpr int kThreads = 256;

__device__ __forceinline__ double wrap_periodic(double x, double B) {
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

// Cell coordinate along one axis on the grid shifted by s.
__device__ __forceinline__ int cell_coord(double x, double s, const Geom& g, int d) {
  const double diff = __dsub_rn(x, s);
  const double q = g.pow2a ? __dmul_rn(diff, g.inv_a) : __ddiv_rn(diff, g.a);
  int c = static_cast<int>(floor(q));
  if (g.walls && d == 2) {  // layers 0 .. Lz; rounding of (z - s)/a may reach Lz + 1
    c += 1;
    return c < 0 ? 0 : (c > g.L[2] ? g.L[2] : c);
  }
  if (c < 0) c += g.L[d];
  else if (c >= g.L[d]) c -= g.L[d];
  return c;
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

template <int WALLS, int FORCE>
__global__ void __launch_bounds__(kThreads) k_stream_bin_fp64(Geom g, Fp64Bufs b, Scratch s, Ctl* __restrict__ ctl) {
  __shared__ double sh[3];
  __shared__ int scur;
  if (threadIdx.x == 0) {
    double sv[3];
    grid_shift(g.seed, ctl->t + 1, g.a, g.walls, sv);
    sh[0] = sv[0];
    sh[1] = sv[1];
    sh[2] = sv[2];
    scur = ctl->cur;
    if (blockIdx.x == 0) {
      ctl->shift[0] = sv[0];
      ctl->shift[1] = sv[1];
      ctl->shift[2] = sv[2];
    }
  }
  __syncthreads();
  const int cur = scur;
  double* __restrict__ rx = b.r[cur][0];
  double* __restrict__ ry = b.r[cur][1];
  double* __restrict__ rz = b.r[cur][2];
  double* __restrict__ vx = b.v[cur][0];
  double* __restrict__ vy = b.v[cur][1];
  double* __restrict__ vz = b.v[cur][2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    double r[3] = {rx[i], ry[i], rz[i]};
    double v[3] = {vx[i], vy[i], vz[i]};
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
        r[d] = wrap_periodic(r[d], g.B[d]);
      }
    }
    rx[i] = r[0];
    ry[i] = r[1];
    rz[i] = r[2];
    if (WALLS || FORCE) {
      vx[i] = v[0];
      vy[i] = v[1];
      vz[i] = v[2];
    }
    const int cx = cell_coord(r[0], sh[0], g, 0);
    const int cy = cell_coord(r[1], sh[1], g, 1);
    const int cz = cell_coord(r[2], sh[2], g, 2);
    const int key = cx + g.L[0] * (cy + g.L[1] * cz);
    s.key[i] = key;
    s.rank[i] = atomicAdd(&s.count[key], 1);
  }
}

__global__ void __launch_bounds__(kThreads) k_scatter(int64_t n, const int32_t* __restrict__ key,
                                                      const int32_t* __restrict__ rank, const int32_t* __restrict__ offset,
                                                      int32_t* __restrict__ perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    perm[offset[key[i]] + rank[i]] = static_cast<int32_t>(i);
}

// One thread per collision cell (the shape of Listing 4).
template <int WALLS, int THERMO, int MOMENTS>
__global__ void __launch_bounds__(kThreads) k_collide_fp64(Geom g, Fp64Bufs b, Scratch s, Ctl* __restrict__ ctl) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int64_t t1 = ctl->t + 1;
  const int cur = ctl->cur;
  const bool resort = g.resort_k > 0 && (t1 % g.resort_k) == 0;
  const int o = s.offset[c];
  const int n = s.offset[c + 1] - o;
  int32_t* __restrict__ pm = s.perm + o;

  // the counting atomics hand out arrival ranks in no fixed order: restore storage order
  for (int j = 1; j < n; ++j) {
    const int x = pm[j];
    int k = j - 1;
    while (k >= 0 && pm[k] > x) {
      pm[k + 1] = pm[k];
      --k;
    }
    pm[k + 1] = x;
  }

  const double m = g.mass;
  double M = 0.0, P0 = 0.0, P1 = 0.0, P2 = 0.0, E = 0.0;
  for (int j = 0; j < n; ++j) {
    const int i = pm[j];
    const double v0 = b.v[cur][0][i], v1 = b.v[cur][1][i], v2 = b.v[cur][2][i];
    P0 += m * v0;
    P1 += m * v1;
    P2 += m * v2;
    M += m;
    if (MOMENTS) E += 0.5 * m * (v0 * v0 + v1 * v1 + v2 * v2);
  }
  if (MOMENTS) {
    double* mo = s.moments + 5 * c;
    mo[0] = M;
    mo[1] = P0;
    mo[2] = P1;
    mo[3] = P2;
    mo[4] = E;
  }
  if (n == 0) return;

  bool virt = false;
  if (WALLS) {
    const double sz = ctl->shift[2];
    const int64_t layer = c / ((int64_t)g.L[0] * g.L[1]);
    if (sz > 0.0 && (layer == 0 || layer == g.L[2]) && (double)n < g.ppc) {
      const double Mv = (g.ppc - (double)n) * m;
      const u64x4 w = draw(g.seed, static_cast<uint64_t>(t1), static_cast<uint64_t>(c), kTagWall);
      double g0, g1, g2, g3;
      gauss_pair(w.x, w.y, g0, g1);
      gauss_pair(w.z, w.w, g2, g3);
      const double sd = sqrt(Mv * g.kT);
      P0 += sd * g0;
      P1 += sd * g1;
      P2 += sd * g2;
      M += Mv;
      virt = true;
    }
  }

  const int ob = cur ^ 1;
  if (n >= 2 || virt) {
    const double u0 = P0 / M, u1 = P1 / M, u2 = P2 / M;
    double ax[3];
    random_axis(g.seed, t1, c, ax);
    const double ca = g.cos_a, sa = g.sin_a;
    for (int j = 0; j < n; ++j) {
      const int i = pm[j];
      const double d0 = b.v[cur][0][i] - u0, d1 = b.v[cur][1][i] - u1, d2 = b.v[cur][2][i] - u2;
      const double par = ax[0] * d0 + ax[1] * d1 + ax[2] * d2;
      const double c0 = ax[1] * d2 - ax[2] * d1;
      const double c1 = ax[2] * d0 - ax[0] * d2;
      const double c2 = ax[0] * d1 - ax[1] * d0;
      const double w0 = par * ax[0] + ca * (d0 - par * ax[0]) + sa * c0;
      const double w1 = par * ax[1] + ca * (d1 - par * ax[1]) + sa * c1;
      const double w2 = par * ax[2] + ca * (d2 - par * ax[2]) + sa * c2;
      b.v[cur][0][i] = u0 + w0;
      b.v[cur][1][i] = u1 + w1;
      b.v[cur][2][i] = u2 + w2;
    }
    if (THERMO && n >= 2) {
      double K = 0.0;
      for (int j = 0; j < n; ++j) {
        const int i = pm[j];
        const double d0 = b.v[cur][0][i] - u0, d1 = b.v[cur][1][i] - u1, d2 = b.v[cur][2][i] - u2;
        K += 0.5 * m * (d0 * d0 + d1 * d1 + d2 * d2);
      }
      if (K > 0.0) {
        const double f = sqrt(1.5 * (double)(n - 1) * g.kT / K);
        for (int j = 0; j < n; ++j) {
          const int i = pm[j];
          b.v[cur][0][i] = u0 + f * (b.v[cur][0][i] - u0);
          b.v[cur][1][i] = u1 + f * (b.v[cur][1][i] - u1);
          b.v[cur][2][i] = u2 + f * (b.v[cur][2][i] - u2);
        }
      }
    }
  }
  if (resort) {
    for (int j = 0; j < n; ++j) {
      const int i = pm[j];
      const int dst = o + j;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        b.r[ob][d][dst] = b.r[cur][d][i];
        b.v[ob][d][dst] = b.v[cur][d][i];
      }
      b.id[ob][dst] = b.id[cur][i];
    }
  }
}

__global__ void k_end_step(Ctl* ctl, int32_t resort_k) {
  const int64_t t1 = ctl->t + 1;
  if (resort_k > 0 && (t1 % resort_k) == 0) ctl->cur ^= 1;
  ctl->t = t1;
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

__global__ void __launch_bounds__(kThreads) k_set_state_fp64(int64_t n, const double* __restrict__ r,
                                                             const double* __restrict__ v, Fp64Bufs b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      b.r[0][d][i] = r[3 * i + d];
      b.v[0][d][i] = v[3 * i + d];
    }
    b.id[0][i] = static_cast<int32_t>(i);
  }
}

unsigned grid_for(int64_t n, int per_thread = 1) {
  int64_t blocks = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 64) blocks = 152 * 64;
  return static_cast<unsigned>(blocks);
}
}  // namespace

void launch_init_fp64(const Geom& g, Fp64Bufs b, double* red, int red_blocks, Ctl* ctl, cudaStream_t st) {
  k_init_fp64<<<red_blocks, kThreads, 0, st>>>(g, b, red);
  k_init_mean<<<1, kThreads, 0, st>>>(red, red_blocks, g.n, ctl);
  k_init_sub<<<grid_for(g.n), kThreads, 0, st>>>(g, b, ctl);
}

void launch_stream_bin_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, cudaStream_t st) {
  const unsigned grid = grid_for(g.n);
  if (g.walls)
    k_stream_bin_fp64<1, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl);
  else if (g.force)
    k_stream_bin_fp64<0, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl);
  else
    k_stream_bin_fp64<0, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl);
}

void launch_scatter(const Geom& g, Scratch s, cudaStream_t st) {
  k_scatter<<<grid_for(g.n), kThreads, 0, st>>>(g.n, s.key, s.rank, s.offset, s.perm);
}

void launch_collide_fp64(const Geom& g, Fp64Bufs b, Scratch s, Ctl* ctl, bool moments, cudaStream_t st) {
  const unsigned grid = static_cast<unsigned>((g.ncell + kThreads - 1) / kThreads);
  const int sel = (g.walls ? 4 : 0) | (g.thermostat ? 2 : 0) | (moments ? 1 : 0);
  switch (sel) {
    case 0: k_collide_fp64<0, 0, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 1: k_collide_fp64<0, 0, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 2: k_collide_fp64<0, 1, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 3: k_collide_fp64<0, 1, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 4: k_collide_fp64<1, 0, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 5: k_collide_fp64<1, 0, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    case 6: k_collide_fp64<1, 1, 0><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
    default: k_collide_fp64<1, 1, 1><<<grid, kThreads, 0, st>>>(g, b, s, ctl); break;
  }
}

void launch_end_step(const Geom& g, Ctl* ctl, cudaStream_t st) { k_end_step<<<1, 1, 0, st>>>(ctl, g.resort_k); }

void launch_get_state_fp64(const Geom& g, Fp64Bufs b, int cur, double* r, double* v, cudaStream_t st) {
  k_get_state_fp64<<<grid_for(g.n), kThreads, 0, st>>>(g.n, b.r[cur][0], b.r[cur][1], b.r[cur][2], b.v[cur][0],
                                                        b.v[cur][1], b.v[cur][2], b.id[cur], r, v);
}

void launch_set_state_fp64(const Geom& g, Fp64Bufs b, const double* r, const double* v, cudaStream_t st) {
  k_set_state_fp64<<<grid_for(g.n), kThreads, 0, st>>>(g.n, r, v, b);
}

}  // namespace mpcd
