// kernels_scan.cu -- exclusive prefix sum of the per-cell counts (the offsets of the
// linked-cell list, paper Sec. 3.1 / Listing 4's binOffset).
//
// Reduce-then-scan in three launches: per-tile sums, one block scanning the tile sums, and a
// per-tile scan that adds its tile's prefix.  No block ever waits on another block, so the
// scan cannot hang however the blocks are scheduled.  Counts are read twice (8 bytes per
// cell); with about ten particles per cell that is under one byte per particle.
#include "mpcd_internal.h"

namespace mpcd {

namespace {
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kPartialThreads = 1024;

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the block total in *total.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int warp_tot[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int incl = warp_incl_scan(v);
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < NT / 32) ? warp_tot[lane] : 0;
    w = warp_incl_scan(w);
    if (lane < NT / 32) warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int warp_prefix = wid ? warp_tot[wid - 1] : 0;
  *total = warp_tot[NT / 32 - 1];
  __syncthreads();
  return warp_prefix + incl - v;
}

__global__ void __launch_bounds__(kThreads) k_zero_i32(int32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int32_t* __restrict__ count, int32_t* __restrict__ partial,
                                                          int64_t n) {
  const int64_t base = (int64_t)blockIdx.x * kTile;
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    if (i < n) sum += count[i];
  }
  int total;
  block_excl_scan<kThreads>(sum, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// One block: exclusive scan of the tile sums in place; writes the grand total to offset[n].
__global__ void __launch_bounds__(kPartialThreads) k_scan_partials(int32_t* __restrict__ partial, int tiles,
                                                                   int32_t* __restrict__ offset, int64_t n) {
  int carry = 0;
  for (int base = 0; base < tiles; base += kPartialThreads) {
    const int i = base + threadIdx.x;
    const int v = (i < tiles) ? partial[i] : 0;
    int total;
    const int ex = block_excl_scan<kPartialThreads>(v, &total);
    if (i < tiles) partial[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) offset[n] = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_final(const int32_t* __restrict__ count, int32_t* __restrict__ offset,
                                                         const int32_t* __restrict__ partial, int64_t n) {
  __shared__ int tile[kTile];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  // coalesced load, then each thread owns kItems consecutive entries
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    tile[k * kThreads + threadIdx.x] = (i < n) ? count[i] : 0;
  }
  __syncthreads();
  int vals[kItems];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    vals[k] = tile[threadIdx.x * kItems + k];
    sum += vals[k];
  }
  int total;
  int run = block_excl_scan<kThreads>(sum, &total) + partial[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    tile[threadIdx.x * kItems + k] = run;
    run += vals[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    if (i < n) offset[i] = tile[k * kThreads + threadIdx.x];
  }
}
}  // namespace

int scan_tiles(int64_t count) { return static_cast<int>((count + kTile - 1) / kTile); }

__global__ void __launch_bounds__(kThreads) k_zero_i32_pair(int32_t* p, int32_t* q, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = 0;
    q[i] = 0;
  }
}

void launch_zero_i32_pair(int32_t* p, int32_t* q, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  int64_t blocks = (n + kThreads * 4 - 1) / (kThreads * 4);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_zero_i32_pair<<<static_cast<unsigned>(blocks), kThreads, 0, st>>>(p, q, n);
}

void launch_zero_i32(int32_t* p, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  int64_t blocks = (n + kThreads * 4 - 1) / (kThreads * 4);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_zero_i32<<<static_cast<unsigned>(blocks), kThreads, 0, st>>>(p, n);
}

void launch_scan(const int32_t* count, int32_t* offset, int32_t* partial, int64_t n, cudaStream_t st) {
  const int tiles = scan_tiles(n);
  if (tiles > 0) k_scan_reduce<<<tiles, kThreads, 0, st>>>(count, partial, n);
  k_scan_partials<<<1, kPartialThreads, 0, st>>>(partial, tiles, offset, n);
  if (tiles > 0) k_scan_final<<<tiles, kThreads, 0, st>>>(count, offset, partial, n);
}

}  // namespace mpcd
