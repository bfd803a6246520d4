// FMA-throughput probe (a measurement aid for reporting ALU-bound kernels against the
// device they run on; not part of the reconstruction).  Every thread runs 8 independent
// FMA chains for a fixed number of steps; the grid fills every SM several times over.
#include <math.h>

#include "bsct_internal.h"

namespace {
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T* __restrict__ out, int steps, T a, T c) {
  T v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = T(threadIdx.x) * T(1e-3) + T(k);
  for (int s = 0; s < steps; ++s) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, c);
  }
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) acc += v[k];
  out[(long)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <typename T> int fma_peak(double* flops, cudaStream_t st) {
  int dev = 0, sms = 0;
  BSCT_CUDA_TRY(cudaGetDevice(&dev));
  BSCT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 16, threads = 256;
  const int steps = sizeof(T) == 4 ? 4096 : 256;
  T* out = nullptr;
  BSCT_CUDA_TRY(cudaMalloc(&out, (size_t)blocks * threads * sizeof(T)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = BSCT_OK;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && rc == BSCT_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, st);
    k_fma_chain<T><<<blocks, threads, 0, st>>>(out, steps, T(0.999), T(1e-3));
    bsct::count_launch();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = BSCT_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  if (rc == BSCT_OK && cudaGetLastError() != cudaSuccess) rc = BSCT_ERR_CUDA;
  *flops = rc == BSCT_OK ? 2.0 * 8.0 * steps * (double)blocks * threads / (best * 1e-3) : 0.0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}
}  // namespace

extern "C" int bsct_fma_peak(int precision, double* flops_per_s, void* stream) {
  if (!flops_per_s || (precision != BSCT_F32 && precision != BSCT_F64)) {
    bsct_set_last_message("invalid argument");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return precision == BSCT_F32 ? fma_peak<float>(flops_per_s, st) : fma_peak<double>(flops_per_s, st);
}
