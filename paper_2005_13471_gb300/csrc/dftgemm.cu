// Gram apply with the 2N x 2N DFTs computed as split-BF16 DFT-GEMMs on the tensor cores
// (precision variant of the FFT apply; FP32 accumulation, error against the FP64
// oracle reported by the tests and the benchmark).
//
// A length-L DFT (L = 2N = P Q) along the leading index of a planar complex tensor
// T[re/im][L][R] is done in two GEMM stages (Cooley-Tukey with n = Q n1 + n2,
// k = k1 + P k2):
//   stage 1: D1[ri][k1][n2][rest] = sum_n1 W_P^(n1 k1) T[ri][Q n1 + n2][rest]
//   twiddle: D1 *= W_L^(n2 k1), reordered to [n2][k1][rest]
//   stage 2: D2[ri][k2][k1][rest] = sum_n2 W_Q^(n2 k2) D1'[ri][n2][k1][rest]  = out[k][rest]
// Each stage is one real GEMM: the complex DFT matrix as the 2P x 2P real matrix
// [[Re W, -Im W], [Im W, Re W]], and both operands split into BF16 high and low parts
// so that A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (K = 6P: the data's high part appears
// twice in the operand).  The 2-D convolution chains four such DFTs:
//   pad x -> DFT over rows index -> transpose -> DFT over columns -> x spectrum ->
//   inverse DFT over columns -> transpose -> inverse DFT over rows -> crop.
#include <cuda_bf16.h>

#include "bsct_internal.h"

namespace bsct {

int gemm_bf16(bool ta, bool tb, int M, int N, int K, float alpha, const void* A, long lda, long sA, const void* B,
              long ldb, long sB, float beta, float* C, long ldc, long sC, int batch, cudaStream_t st);

namespace {

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// A3[(ro, k)][(s, ri, n)] for a P-point DFT (sign -1 forward, +1 inverse)
__global__ void k_dft_matrix(__nv_bfloat16* A3, int P, int inverse) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int M = 2 * P, K = 6 * P;
  if (i >= M * K) return;
  const int m = i / K, kk = i % K;
  const int ro = m / P, k = m % P;
  const int s = kk / (2 * P), ri = (kk / P) % 2, n = kk % P;
  double sn, cs;
  sincospi((inverse ? 2.0 : -2.0) * (double)((long)n * k % P) / (double)P, &sn, &cs);
  // [[Re, -Im], [Im, Re]]
  double a;
  if (ro == 0) a = (ri == 0) ? cs : -sn;
  else a = (ri == 0) ? sn : cs;
  const float af = (float)a;
  __nv_bfloat16 hi, lo;
  split_bf16(af, hi, lo);
  A3[i] = (s == 2) ? lo : hi;  // operand order [B_hi; B_lo; B_hi] pairs with [A_hi, A_hi, A_lo]
}

// first operand of the row-index DFT: zero-padded real image x (N x N) as T[ri][L][L];
// grid (rows L, planes 2), threads over the columns of a row
__global__ void k_split_pad(const float* __restrict__ x, int N, __nv_bfloat16* __restrict__ B) {
  const int L = 2 * N;
  const long plane = (long)L * L;
  const int r = blockIdx.x, ri = blockIdx.y;
  for (int c = threadIdx.x; c < L; c += blockDim.x) {
    const long i = (long)ri * plane + (long)r * L + c;
    const float v = (ri == 0 && r < N && c < N) ? x[(long)r * N + c] : 0.f;
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    B[i] = hi;
    B[2 * plane + i] = lo;
    B[4 * plane + i] = hi;
  }
}

// D1[ri][k1][n2][rest] * W_L^(+-n2 k1) -> split operand [s][ri][n2][k1][rest]; grid (Q, P):
// one (k1, n2) row of R values per block
__global__ void k_twiddle_split(const float* __restrict__ D, int P, int Q, long R, const float2* __restrict__ tw,
                                int inverse, __nv_bfloat16* __restrict__ B) {
  const long L = (long)P * Q;
  const long plane = L * R;
  const int n2 = blockIdx.x, k1 = blockIdx.y;
  const float2 w = tw[((long)n2 * k1) % L];
  const float wi = inverse ? -w.y : w.y;
  const float* dre = D + ((long)k1 * Q + n2) * R;
  const long o0 = ((long)n2 * P + k1) * R;
  for (long rest = threadIdx.x; rest < R; rest += blockDim.x) {
    const float re = dre[rest], im = dre[plane + rest];
    const float yr = re * w.x - im * wi, yi = re * wi + im * w.x;
    const long o = o0 + rest;
    __nv_bfloat16 hr, lr, hi_, li;
    split_bf16(yr, hr, lr);
    split_bf16(yi, hi_, li);
    B[o] = hr; B[plane + o] = hi_;
    B[2 * plane + o] = lr; B[3 * plane + o] = li;
    B[4 * plane + o] = hr; B[5 * plane + o] = hi_;
  }
}

// D[ri][a][b] (L x L) -> split operand of the transposed tensor [s][ri][b][a]; optionally
// multiplied by the real spectrum first (Gt layout of the FFT path, scaled by 1/L^2):
// element (a, b) = (v, u) column frequency v, row frequency u.  32 x 32 tiles through
// shared memory (grid (L/32, L/32), block 32 x 8): reads and writes both coalesced.
__global__ void k_transpose_split(const float* __restrict__ D, int N, const float* __restrict__ Gt,
                                  __nv_bfloat16* __restrict__ B) {
  const int L = 2 * N;
  const long plane = (long)L * L;
  __shared__ float tre[32][33], tim[32][33];
  const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int a = a0 + dy, b = b0 + threadIdx.x;
    const long src = (long)a * L + b;
    float re = D[src], im = D[plane + src];
    if (Gt) {
      const int v = a, u = b;
      float g;
      if (v == 0) g = Gt[u] + Gt[(long)N * L + u];
      else if (v == N) g = Gt[u] - Gt[(long)N * L + u];
      else if (v < N) g = Gt[(long)v * L + u];
      else g = Gt[(long)(L - v) * L + (u == 0 ? 0 : L - u)];
      re *= g;
      im *= g;
    }
    tre[dy][threadIdx.x] = re;
    tim[dy][threadIdx.x] = im;
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int b = b0 + dy, a = a0 + threadIdx.x;
    const long i = (long)b * L + a;
    __nv_bfloat16 hr, lr, hi_, li;
    split_bf16(tre[threadIdx.x][dy], hr, lr);
    split_bf16(tim[threadIdx.x][dy], hi_, li);
    B[i] = hr; B[plane + i] = hi_;
    B[2 * plane + i] = lr; B[3 * plane + i] = li;
    B[4 * plane + i] = hr; B[5 * plane + i] = hi_;
  }
}

// y[r][c] = Re D[c][r] for r, c < N (the last DFT ran over the column index, leading)
__global__ void k_crop_t(const float* __restrict__ D, int N, float* __restrict__ y) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)N * N) return;
  const int r = (int)(i / N), c = (int)(i % N);
  y[i] = D[(long)c * (2 * N) + r];
}

}  // namespace

bool dftgemm_factor(int L, int* P, int* Q) {
  for (int p = 64; p >= 4; p -= 4)
    if (L % p == 0 && (L / p) % 4 == 0 && L / p <= 64) {
      *P = p;
      *Q = L / p;
      return true;
    }
  return false;
}

size_t dftgemm_scratch_bytes(int N) {
  int P, Q;
  if (!dftgemm_factor(2 * N, &P, &Q)) return 0;
  const size_t plane = (size_t)4 * N * N;
  const size_t mats = (size_t)2 * (2 * P * 6 * P + 2 * Q * 6 * Q) * 2;
  return 6 * plane * 2 /*B bf16*/ + 2 * (2 * plane * 4) /*two D fp32*/ + mats + 4096;
}

// one length-L DFT along the leading index of T[ri][L][R] held as split operand B (in),
// result in Dout[ri][L][R]; Dtmp is FP32 scratch, B is reused for the twiddled operand
static int dft_leading(int L, int P, int Q, long R, const __nv_bfloat16* Ap, const __nv_bfloat16* Aq, __nv_bfloat16* B,
                       float* Dtmp, float* Dout, const float2* tw, int inverse, cudaStream_t st) {
  // stage 1: M = 2P, K = 6P, N = Q R
  int rc = gemm_bf16(false, false, 2 * P, (int)(Q * R), 6 * P, 1.f, Ap, 6 * P, 0, B, Q * R, 0, 0.f, Dtmp, Q * R, 0, 1, st);
  if (rc != BSCT_OK) return rc;
  k_twiddle_split<<<dim3((unsigned)Q, (unsigned)P), 256, 0, st>>>(Dtmp, P, Q, R, tw, inverse, B);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  // stage 2: M = 2Q, K = 6Q, N = P R
  return gemm_bf16(false, false, 2 * Q, (int)(P * R), 6 * Q, 1.f, Aq, 6 * Q, 0, B, P * R, 0, 0.f, Dout, P * R, 0, 1, st);
}

// y = G x (FP32 in/out) with split-BF16 DFT-GEMMs.  work: dftgemm_scratch_bytes(N) bytes.
int dftgemm_apply(int N, const float* x, float* y, const float* Gt, const float2* tw_untangle, void* work,
                  cudaStream_t st) {
  const int L = 2 * N;
  int P, Q;
  if (!dftgemm_factor(L, &P, &Q)) return BSCT_ERR_UNSUPPORTED_SIZE;
  const long plane = (long)L * L;
  char* w = (char*)work;
  auto take = [&](size_t bytes) {
    char* p = w;
    w += (bytes + 255) & ~(size_t)255;
    return p;
  };
  __nv_bfloat16* B = (__nv_bfloat16*)take(6 * plane * 2);
  float* D1 = (float*)take(2 * plane * 4);
  float* D2 = (float*)take(2 * plane * 4);
  __nv_bfloat16* Apf = (__nv_bfloat16*)take((size_t)2 * P * 6 * P * 2);
  __nv_bfloat16* Api = (__nv_bfloat16*)take((size_t)2 * P * 6 * P * 2);
  __nv_bfloat16* Aqf = (__nv_bfloat16*)take((size_t)2 * Q * 6 * Q * 2);
  __nv_bfloat16* Aqi = (__nv_bfloat16*)take((size_t)2 * Q * 6 * Q * 2);
  k_dft_matrix<<<(12 * P * P + 255) / 256, 256, 0, st>>>(Apf, P, 0);
  k_dft_matrix<<<(12 * P * P + 255) / 256, 256, 0, st>>>(Api, P, 1);
  k_dft_matrix<<<(12 * Q * Q + 255) / 256, 256, 0, st>>>(Aqf, Q, 0);
  k_dft_matrix<<<(12 * Q * Q + 255) / 256, 256, 0, st>>>(Aqi, Q, 1);
  const dim3 gt((unsigned)(L / 32), (unsigned)(L / 32)), bt(32, 8);
  k_split_pad<<<dim3((unsigned)L, 2), 256, 0, st>>>(x, N, B);
  count_launch(5);
  BSCT_CUDA_TRY(cudaGetLastError());
  int rc;
  // forward over the row index r (leading), then over the column index
  if ((rc = dft_leading(L, P, Q, L, Apf, Aqf, B, D1, D2, tw_untangle, 0, st)) != BSCT_OK) return rc;
  k_transpose_split<<<gt, bt, 0, st>>>(D2, N, nullptr, B);
  count_launch();
  if ((rc = dft_leading(L, P, Q, L, Apf, Aqf, B, D1, D2, tw_untangle, 0, st)) != BSCT_OK) return rc;
  // D2[ri][v][u]: multiply by the spectrum, transpose to [u][v] -> inverse over u first
  k_transpose_split<<<gt, bt, 0, st>>>(D2, N, Gt, B);
  count_launch();
  if ((rc = dft_leading(L, P, Q, L, Api, Aqi, B, D1, D2, tw_untangle, 1, st)) != BSCT_OK) return rc;
  // D2[ri][r][v] -> [v][r] -> inverse over v
  k_transpose_split<<<gt, bt, 0, st>>>(D2, N, nullptr, B);
  count_launch();
  if ((rc = dft_leading(L, P, Q, L, Api, Aqi, B, D1, D2, tw_untangle, 1, st)) != BSCT_OK) return rc;
  // D2[ri][c][r]: crop the transposed result
  k_crop_t<<<(unsigned)(((long)N * N + 255) / 256), 256, 0, st>>>(D2, N, y);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

}  // namespace bsct
