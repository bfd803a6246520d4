// Gram apply that allocates no device memory (bsct_gram_apply_noalloc).
//
// Some callers cannot allocate device memory: a plug-in running inside a host
// application that owns the whole device memory pool, or code on a latency-critical
// path where cudaMalloc / cudaFree would synchronise the device or fail under memory
// pressure.  For them this file keeps every buffer the FP32 Gram apply needs in
// file-scope device arrays of fixed size (resident on each GPU that loads the library,
// until the process exits):
//   g_na_scratch   - the N x N complex half-spectrum scratch of the three FFT passes,
//   g_na_spectrum  - the packed, scaled spectrum the column pass reads,
//   g_na_tw        - FFT twiddle tables of the call's N.
// The size limit is BSCT_NOALLOC_MAX_N = 512 (2 MiB of scratch).  The kernels are the
// ones bsct_gram_apply launches; only the buffers differ.  Every call writes the
// twiddle tables and the packed spectrum it reads before the three FFT passes (eight
// small kernels beside the three passes), so no call depends on what an earlier call
// left in the arrays, whatever N it had.
#include "bsct_internal.h"

namespace {

constexpr int NA_MAX_N = BSCT_NOALLOC_MAX_N;
constexpr int NA_MAX_DEV = 64;

static __device__ __align__(256) bsct::cpx<float> g_na_scratch[(size_t)NA_MAX_N * NA_MAX_N];
static __device__ __align__(256) float g_na_spectrum[(size_t)(NA_MAX_N + 1) * 2 * NA_MAX_N];
static __device__ __align__(256) bsct::cpx<float> g_na_tw[8 * NA_MAX_N];

struct NaDevice {
  bool ready = false;
  bsct::cpx<float>* scratch = nullptr;
  float* spectrum = nullptr;
  bsct::cpx<float>* tw = nullptr;
};
NaDevice g_na_dev[NA_MAX_DEV];

// [2N][N+1] plain FP64 spectrum -> [N+1][2N] FP32 layout of the column pass:
// row v (1..N-1) = spectrum[:, v], row 0 = (S0 + SN)/2, row N = (S0 - SN)/2, all / (2N)^2
__global__ void k_na_pack(const double* __restrict__ spec, int N, float* __restrict__ out) {
  const int L = 2 * N;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)(N + 1) * L) return;
  const int v = (int)(i / L), u = (int)(i % L);
  const double sc = 1.0 / ((double)L * (double)L);
  const double s0 = spec[(long)u * (N + 1)], sN = spec[(long)u * (N + 1) + N];
  double g;
  if (v == 0) g = 0.5 * (s0 + sN);
  else if (v == N) g = 0.5 * (s0 - sN);
  else g = spec[(long)u * (N + 1) + v];
  out[i] = (float)(g * sc);
}

}  // namespace

extern "C" int bsct_gram_apply_noalloc(int32_t N, const double* d_spectrum, const float* d_x, float* d_y,
                                       void* stream) {
  using namespace bsct;
  if (!d_spectrum || !d_x || !d_y) {
    bsct_set_last_message("NULL device pointer");
    return BSCT_ERR_INVALID_ARG;
  }
  if ((const void*)d_x == (const void*)d_y) {
    bsct_set_last_message("x and y may not alias");
    return BSCT_ERR_INVALID_ARG;
  }
  FftOps<float> ops;
  if (N > NA_MAX_N || !fft_ops_for<float>(N, &ops)) {
    bsct_set_last_message("bsct_gram_apply_noalloc: N must be a supported size <= BSCT_NOALLOC_MAX_N (512)");
    return BSCT_ERR_UNSUPPORTED_SIZE;
  }
  int dev = 0;
  BSCT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEV) {
    bsct_set_last_message("device index out of range");
    return BSCT_ERR_INVALID_ARG;
  }
  NaDevice& d = g_na_dev[dev];
  cudaStream_t st = (cudaStream_t)stream;
  if (!d.ready) {
    // host code must not use the array names as addresses: ask the runtime for the
    // device addresses of this GPU's copies (the current device is `dev`)
    BSCT_CUDA_TRY(cudaGetSymbolAddress((void**)&d.scratch, g_na_scratch));
    BSCT_CUDA_TRY(cudaGetSymbolAddress((void**)&d.spectrum, g_na_spectrum));
    BSCT_CUDA_TRY(cudaGetSymbolAddress((void**)&d.tw, g_na_tw));
    d.ready = true;
  }
  // tables of this N, rebuilt on every call (8N entries: cheap beside the FFT passes)
  const int rc = build_fft_tables<float>(d.tw, N, st);
  if (rc != BSCT_OK) return rc;
  const long n = (long)(N + 1) * 2 * N;
  k_na_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_spectrum, N, d.spectrum);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return ops.apply(d_x, d_y, d.scratch, d.spectrum, d.tw, st);
}
