// Detection of non-finite input values.
//
// The synchronous solvers see a non-finite right-hand side or initial guess in their own
// inner products (<b, b>, <r, r>) and return BSCT_ERR_NONFINITE.  The asynchronous entry
// points (Gram apply, back projection, forward projection) cannot return what their
// kernels find, so those kernels set a per-device status word instead; the caller reads
// (and clears) it with bsct_input_status at a synchronisation point of its choosing.
// bsct_check_finite checks one caller buffer synchronously.
#include "bsct_internal.h"

namespace {

constexpr int ST_MAX_DEV = 64;
constexpr int ST_THREADS = 256;

// word 0: sticky flag of the asynchronous entry points; word 1: result of the last
// bsct_check_finite call; word 2: set by a kernel whose bounded wait gave up
static __device__ __align__(16) unsigned int g_status_words[4];

unsigned int* g_words[ST_MAX_DEV] = {};

unsigned int* words_ptr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= ST_MAX_DEV) return nullptr;
  if (!g_words[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_words) != cudaSuccess) return nullptr;
    g_words[dev] = (unsigned int*)p;
  }
  return g_words[dev];
}

template <typename T>
__global__ void __launch_bounds__(ST_THREADS) k_check_finite(const T* __restrict__ p, long n, unsigned int* flag) {
  bool bad = false;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    bad |= !isfinite(p[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

}  // namespace

namespace bsct {

unsigned int* input_status_ptr() { return words_ptr(); }
unsigned int* timeout_status_ptr() {
  unsigned int* w = words_ptr();
  return w ? w + 2 : nullptr;
}

template <typename T> int check_finite_async(const T* p, long n, cudaStream_t st, int word) {
  unsigned int* w = words_ptr();
  if (!w) { bsct_set_last_message("status word lookup failed"); return BSCT_ERR_CUDA; }
  if (n <= 0) return BSCT_OK;
  long blocks = (n + ST_THREADS - 1) / ST_THREADS;
  if (blocks > 4096) blocks = 4096;
  k_check_finite<T><<<(unsigned)blocks, ST_THREADS, 0, st>>>(p, n, w + word);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}
template int check_finite_async<float>(const float*, long, cudaStream_t, int);
template int check_finite_async<double>(const double*, long, cudaStream_t, int);

}  // namespace bsct

extern "C" int bsct_input_status(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* w = words_ptr();
  if (!w) { bsct_set_last_message("status word lookup failed"); return BSCT_ERR_CUDA; }
  unsigned int h[3] = {0, 0, 0};
  BSCT_CUDA_TRY(cudaMemcpyAsync(h, w, sizeof(h), cudaMemcpyDeviceToHost, st));
  BSCT_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(unsigned int), st));
  BSCT_CUDA_TRY(cudaMemsetAsync(w + 2, 0, sizeof(unsigned int), st));
  BSCT_CUDA_TRY(cudaStreamSynchronize(st));
  if (h[2]) {
    bsct_set_last_message("a kernel gave up a bounded wait (its result is incomplete)");
    return BSCT_ERR_TIMEOUT;
  }
  if (h[0]) {
    bsct_set_last_message("a non-finite input value reached a Gram apply, back projection or forward projection");
    return BSCT_ERR_NONFINITE;
  }
  return BSCT_OK;
}

extern "C" int bsct_check_finite(const void* d_buf, int64_t n, int precision, void* stream) {
  if ((!d_buf && n > 0) || n < 0 || (precision != BSCT_F32 && precision != BSCT_F64)) {
    bsct_set_last_message("invalid argument");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* w = words_ptr();
  if (!w) { bsct_set_last_message("status word lookup failed"); return BSCT_ERR_CUDA; }
  BSCT_CUDA_TRY(cudaMemsetAsync(w + 1, 0, sizeof(unsigned int), st));
  const int rc = precision == BSCT_F32 ? bsct::check_finite_async<float>((const float*)d_buf, (long)n, st, 1)
                                       : bsct::check_finite_async<double>((const double*)d_buf, (long)n, st, 1);
  if (rc != BSCT_OK) return rc;
  unsigned int h = 0;
  BSCT_CUDA_TRY(cudaMemcpyAsync(&h, w + 1, sizeof(h), cudaMemcpyDeviceToHost, st));
  BSCT_CUDA_TRY(cudaStreamSynchronize(st));
  if (h) {
    bsct_set_last_message("buffer holds a non-finite value");
    return BSCT_ERR_NONFINITE;
  }
  return BSCT_OK;
}
