// pdhg_fp64_fma_rate: the device's FP64 fused multiply-add throughput.
//
// No counterpart in the paper. The FP64 form of the iteration issues one FP64
// FMA per stored matrix entry plus a few FP64 operations per row and column,
// and B300 executes FP64 at a small fraction of its FP32 rate, so besides HBM
// bandwidth the FP64 pipe is the second bound of the FP64 step kernels. This
// measures that bound on the device at hand: every thread of a full-occupancy
// grid runs 8 independent FMA chains (so the pipe, not the FMA latency, limits
// the rate) for a fixed count, timed with CUDA events.
#include <cuda_runtime.h>

#include "../../include/pdhg.h"

namespace {

constexpr int RATE_TPB = 256;
constexpr int RATE_CHAINS = 8;
constexpr int RATE_UNROLL = 4;

__global__ void __launch_bounds__(RATE_TPB) k_dfma_rate(double* __restrict__ sink, long long iters, double m,
                                                       double c) {
  double a[RATE_CHAINS];
#pragma unroll
  for (int q = 0; q < RATE_CHAINS; ++q) a[q] = 1.0 + 1e-3 * (double)(threadIdx.x + q);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < RATE_UNROLL; ++u) {
#pragma unroll
      for (int q = 0; q < RATE_CHAINS; ++q) a[q] = fma(a[q], m, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < RATE_CHAINS; ++q) s += a[q];
  // never true for the arguments the host passes; keeps the chains live
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

void pdhg_set_global_error(const char* msg);

extern "C" {

PDHG_API pdhg_status pdhg_fp64_fma_rate(void* cuda_stream, double* fma_per_s, double* ms) {
  if (!fma_per_s) {
    pdhg_set_global_error("fma_per_s is NULL");
    return PDHG_ERR_INVALID;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_rate, RATE_TPB, 0);
  if (e != cudaSuccess) {
    pdhg_set_global_error(cudaGetErrorString(e));
    return PDHG_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  // m = 1 - 2^-30, c = 2^-30: every chain stays near 1 (a fixed point at 1)
  const double m = 1.0 - 1.0 / 1073741824.0, c = 1.0 / 1073741824.0;
  const long long iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float t = 0.0f;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_dfma_rate<<<blocks, RATE_TPB, 0, s>>>(nullptr, iters / 8, m, c);  // warm-up
    e = cudaEventRecord(e0, s);
  }
  if (e == cudaSuccess) {
    k_dfma_rate<<<blocks, RATE_TPB, 0, s>>>(nullptr, iters, m, c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    pdhg_set_global_error(cudaGetErrorString(e));
    return PDHG_ERR_CUDA;
  }
  const double fmas = (double)blocks * RATE_TPB * (double)iters * RATE_UNROLL * RATE_CHAINS;
  *fma_per_s = fmas / ((double)t * 1e-3);
  if (ms) *ms = (double)t;
  return PDHG_OK;
}

}  // extern "C"
