// FP64 throughput probe: the denominator of the trajectory kernel's roofline.
// Every thread runs 8 independent FMA chains; the grid covers every SM with
// `blocks_per_sm` CTAs of 256 threads, and each thread writes one result.
#include <cuda_runtime.h>

#include "../../include/tnrc.h"

namespace {

__global__ void fp64_fma_chains(double* out, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = fma(acc[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" tnrc_status tnrc_measure_fp64_peak(void* scratch, size_t scratch_bytes, double* gflops) {
  if (!scratch || !gflops) return TNRC_E_INVALID;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TNRC_E_CUDA;
  const int threads = 256, blocks = 4 * n_sm, iters = 16384;   // ~30 ms per launch
  if (scratch_bytes < (size_t)blocks * threads * sizeof(double)) return TNRC_E_INVALID;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TNRC_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TNRC_E_CUDA;
  }
  double best = 0.0;
  bool ok = true;
  for (int rep = 0; rep < 5 && ok; ++rep) {   // best of four after a warm-up launch
    ok = cudaEventRecord(e0, 0) == cudaSuccess;
    fp64_fma_chains<<<blocks, threads>>>(static_cast<double*>(scratch), iters, 0.999999, 1e-7);
    ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, 0) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
      const double g = 2.0 * 8 * iters * (double)blocks * threads / (ms * 1e6);
      if (rep > 0 && g > best) best = g;  // the first launch is a warm-up
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return TNRC_E_CUDA;
  *gflops = best;
  return TNRC_OK;
}
