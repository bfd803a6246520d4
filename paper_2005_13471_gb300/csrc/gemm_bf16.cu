// BF16 x BF16 -> FP32 tensor-core GEMM used by the split-BF16 DFT-GEMM Gram apply and
// by the learned warm start's convolutions:
//
//   C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b]       (b = blockIdx.z batch index)
//   op(A) is M x K: A stored row-major M x K (lda), or K x M when TA (A^T stored)
//   op(B) is K x N: B stored row-major K x N (ldb), or N x K when TB
//
// 128 x 128 x 32 CTA tiles, 8 warps of 64 x 32, mma.sync m16n8k16 (FP32 accumulate),
// operands double-buffered in shared memory by cp.async (zero fill outside the
// matrix), fragments by ldmatrix (.trans for the K-contiguous / N-contiguous cases).
// Requirements (checked by the host wrapper): K, lda, ldb multiples of 8 elements,
// 16-byte aligned base pointers.
#include <cuda_bf16.h>

#include "bsct_internal.h"

namespace bsct {

constexpr int GB_M = 128, GB_N = 128, GB_K = 32, GB_PAD = 8;

__device__ __forceinline__ void cp16z(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N_> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N_) : "memory"); }

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(s));
}
__device__ __forceinline__ void mma16816(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// shared tile shapes: A as [M][K+PAD] (row) or [K][M+PAD] (TA); B as [K][N+PAD] (row) or [N][K+PAD] (TB)
template <bool TA> struct ATile {
  static constexpr int R = TA ? GB_K : GB_M, C = (TA ? GB_M : GB_K) + GB_PAD;
};
template <bool TB> struct BTile {
  static constexpr int R = TB ? GB_N : GB_K, C = (TB ? GB_K : GB_N) + GB_PAD;
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_bf16(int M, int N, int K, float alpha, const __nv_bfloat16* __restrict__ A,
                                                   long lda, long sA, const __nv_bfloat16* __restrict__ B, long ldb,
                                                   long sB, float beta, float* __restrict__ C, long ldc, long sC) {
  typedef ATile<TA> AT;
  typedef BTile<TB> BT;
  __shared__ __align__(16) __nv_bfloat16 As[2][AT::R][AT::C];
  __shared__ __align__(16) __nv_bfloat16 Bs[2][BT::R][BT::C];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, warp tile 64 x 32
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  A += blockIdx.z * sA;
  B += blockIdx.z * sB;
  C += blockIdx.z * sC;

  auto load = [&](int stage, int k0) {
    // 512 16-byte pieces per operand tile, 2 per thread
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int q = tid + i * 256;
      if (!TA) {  // [128 m][32 k]: 4 pieces per row
        const int r = q >> 2, c = (q & 3) * 8;
        const int gm = m0 + r, gk = k0 + c;
        const bool ok = gm < M && gk < K;
        cp16z(&As[stage][r][c], ok ? A + (long)gm * lda + gk : A, ok);
      } else {  // [32 k][128 m]: 16 pieces per row
        const int r = q >> 4, c = (q & 15) * 8;
        const int gk = k0 + r, gm = m0 + c;
        const bool ok = gk < K && gm < M;
        cp16z(&As[stage][r][c], ok ? A + (long)gk * lda + gm : A, ok);
      }
      if (!TB) {  // [32 k][128 n]
        const int r = q >> 4, c = (q & 15) * 8;
        const int gk = k0 + r, gn = n0 + c;
        const bool ok = gk < K && gn < N;
        cp16z(&Bs[stage][r][c], ok ? B + (long)gk * ldb + gn : B, ok);
      } else {  // [128 n][32 k]
        const int r = q >> 2, c = (q & 3) * 8;
        const int gn = n0 + r, gk = k0 + c;
        const bool ok = gn < N && gk < K;
        cp16z(&Bs[stage][r][c], ok ? B + (long)gn * ldb + gk : B, ok);
      }
    }
    cp_commit();
  };

  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  const int nk = (K + GB_K - 1) / GB_K;
  load(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    if (kt + 1 < nk) {
      load(st ^ 1, (kt + 1) * GB_K);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; kk += 16) {
      unsigned af[4][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int mrow = wm * 64 + i * 16;
        if (!TA) {
          ldsm_x4(af[i][0], af[i][1], af[i][2], af[i][3], &As[st][mrow + (lane & 15)][kk + (lane >> 4) * 8]);
        } else {
          // stored [k][m]: matrices (m 0-7,k 0-7), (m 8-15,k 0-7), (m 0-7,k 8-15), (m 8-15,k 8-15)
          const int kr = kk + (lane & 7) + ((lane >> 4) << 3);
          const int mc = mrow + ((lane >> 3) & 1) * 8;
          ldsm_x4_t(af[i][0], af[i][1], af[i][2], af[i][3], &As[st][kr][mc]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        const int ncol = wn * 32 + j * 8;
        unsigned r0, r1, r2, r3;
        if (!TB) {
          // stored [k][n]: .trans gives (k 0-7 | k 8-15) for n tiles j, j+1
          const int kr = kk + (lane & 7) + (((lane >> 3) & 1) << 3);
          const int nc = ncol + (lane >> 4) * 8;
          ldsm_x4_t(r0, r1, r2, r3, &Bs[st][kr][nc]);
        } else {
          // stored [n][k]
          const int nr = ncol + (lane & 7) + ((lane >> 4) << 3);
          const int kc = kk + ((lane >> 3) & 1) * 8;
          ldsm_x4(r0, r1, r2, r3, &Bs[st][nr][kc]);
        }
        bf[j][0] = r0; bf[j][1] = r1; bf[j + 1][0] = r2; bf[j + 1][1] = r3;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
  // epilogue: fragment (i, j): rows g, g+8 of the 16 x 8 tile, cols 2t, 2t+1
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 64 + i * 16 + g + h * 8;
        if (m >= M) continue;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int n = n0 + wn * 32 + j * 8 + t4 * 2 + e;
          if (n >= N) continue;
          float v = alpha * acc[i][j][h * 2 + e];
          if (beta != 0.f) v += beta * C[(long)m * ldc + n];
          C[(long)m * ldc + n] = v;
        }
      }
}

int g_gemm_path = 0;

int gemm_bf16(bool ta, bool tb, int M, int N, int K, float alpha, const void* A, long lda, long sA, const void* B,
              long ldb, long sB, float beta, float* C, long ldc, long sC, int batch, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return BSCT_OK;
  if ((K % 8) || (lda % 8) || (ldb % 8) || (sA % 8) || (sB % 8) || (((uintptr_t)A) & 15) || (((uintptr_t)B) & 15) ||
      (ta && (M % 8)) || (!tb && (N % 8))) {
    bsct_set_last_message("gemm_bf16: K, leading dimensions, batch strides (and M if trans_a, N unless trans_b) "
                          "must be multiples of 8");
    return BSCT_ERR_INVALID_ARG;
  }
  if (g_gemm_path == 0) {
    const int rc = gemm_bf16_tc(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, st);
    if (rc != BSCT_ERR_UNSUPPORTED_SIZE) return rc;
  }
  dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M, batch);
  const __nv_bfloat16* a = (const __nv_bfloat16*)A;
  const __nv_bfloat16* b = (const __nv_bfloat16*)B;
  if (!ta && !tb) k_gemm_bf16<false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, a, lda, sA, b, ldb, sB, beta, C, ldc, sC);
  else if (ta && !tb) k_gemm_bf16<true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, a, lda, sA, b, ldb, sB, beta, C, ldc, sC);
  else if (!ta && tb) k_gemm_bf16<false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, a, lda, sA, b, ldb, sB, beta, C, ldc, sC);
  else k_gemm_bf16<true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, a, lda, sA, b, ldb, sB, beta, C, ldc, sC);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

}  // namespace bsct

extern "C" int bsct_gemm_bf16(int trans_a, int trans_b, int32_t M, int32_t N, int32_t K, float alpha, const void* d_A,
                              int64_t lda, int64_t stride_a, const void* d_B, int64_t ldb, int64_t stride_b, float beta,
                              float* d_C, int64_t ldc, int64_t stride_c, int32_t batch, void* stream) {
  if (!d_A || !d_B || !d_C) {
    bsct_set_last_message("NULL device pointer");
    return BSCT_ERR_INVALID_ARG;
  }
  return bsct::gemm_bf16(trans_a != 0, trans_b != 0, M, N, K, alpha, d_A, lda, stride_a, d_B, ldb, stride_b, beta, d_C,
                         ldc, stride_c, batch, (cudaStream_t)stream);
}

extern "C" int bsct_set_gemm_path(int path) {
  if (path != 0 && path != 1) {
    bsct_set_last_message("GEMM path must be 0 (tcgen05) or 1 (mma.sync)");
    return BSCT_ERR_INVALID_ARG;
  }
  bsct::g_gemm_path = path;
  return BSCT_OK;
}
