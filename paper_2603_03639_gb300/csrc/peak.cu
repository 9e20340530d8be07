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

// FP64 tensor-core (DMMA) throughput: every warp runs 4 independent chains of
// m8n8k4 FP64 matrix multiply-accumulates (512 flops each).  A probe only:
// the trajectory kernel's contractions stay on the FMA pipe because this
// rate is not above the FMA rate on GB300.
__global__ void fp64_dmma_chains(double* out, int iters) {
  const int lane = threadIdx.x & 31;
  const double a = 1e-3 * (lane + 1), b = 0.999 - 1e-4 * lane;
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i][0] = c[i][1] = 0.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best rate (GFLOP/s) of four timed launches after a warm-up launch on the
// legacy default stream; launch(i) enqueues one launch, flops its work.
template <class Launch>
tnrc_status time_best(Launch launch, double flops, double* gflops) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TNRC_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TNRC_E_CUDA;
  }
  double best = 0.0;
  bool ok = true;
  for (int rep = 0; rep < 5 && ok; ++rep) {
    ok = cudaEventRecord(e0, 0) == cudaSuccess;
    launch();
    ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, 0) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
      const double g = flops / (ms * 1e6);
      if (rep > 0 && g > best) best = g;  // the first launch is a warm-up
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return TNRC_E_CUDA;
  *gflops = best;
  return TNRC_OK;
}

}  // namespace

extern "C" tnrc_status tnrc_measure_dmma_peak(void* scratch, size_t scratch_bytes, double* gflops) {
  if (!scratch || !gflops) return TNRC_E_INVALID;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TNRC_E_CUDA;
  const int threads = 256, blocks = 4 * n_sm, iters = 4096;
  if (scratch_bytes < (size_t)blocks * threads * sizeof(double)) return TNRC_E_INVALID;
  (void)cudaGetLastError();  // report only the launches below
  double* out = static_cast<double*>(scratch);
  return time_best([&]() { fp64_dmma_chains<<<blocks, threads>>>(out, iters); },
                   512.0 * 4 * iters * (double)blocks * (threads / 32), gflops);
}

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
