// probe.cu -- measurement of this GPU's FP64 FMA issue rate, the ceiling of the FP64 form's
// kernels (GB300 issues far fewer FP64 than FP32 instructions per clock).  Not part of the
// method: bench reports the FP64 kernels' instruction rates against it.
#include <cuda_runtime.h>

#include <string>

#include "mpcd.h"

namespace {
constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;    // independent FMA chains per thread (hides the FMA latency)
constexpr int kProbeIters = 4096;  // FMAs per chain

__global__ void __launch_bounds__(kProbeThreads) k_dfma_chains(double b, double c, double* sink) {
  double acc[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) acc[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc[k] = fma(acc[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += acc[k];
  if (s == -1.0) *sink = s;  // never true for these inputs; keeps the chains live
}
}  // namespace

extern "C" int mpcd_measure_fp64_rate(double* instr_per_s) {
  if (!instr_per_s) return MPCD_ERR_ARG;
  *instr_per_s = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MPCD_ERR_CUDA;
  double* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MPCD_OK;
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MPCD_ERR_CUDA;
  } else {
    const int blocks = sms * 8;
    const double per_launch = (double)blocks * kProbeThreads * kProbeChains * kProbeIters;  // DFMAs, one per lane
    double best = 0.0;
    for (int rep = 0; rep < 4 && rc == MPCD_OK; ++rep) {
      cudaEventRecord(e0, st);
      k_dfma_chains<<<blocks, kProbeThreads, 0, st>>>(0.999999, 1e-7, sink);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = MPCD_ERR_CUDA;
        break;
      }
      const double rate = per_launch / (ms * 1e-3);
      if (rep > 0 && rate > best) best = rate;  // the first launch is a warm-up
    }
    *instr_per_s = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  cudaGetLastError();
  return rc;
}
