// BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores of sm_100+ (tcgen05):
//
//   C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b]   (same contract as k_gemm_bf16)
//
// One CTA of four warps computes a 128 x BN tile of C (BN = 128; 64 or 32 when the B operand
// is K-major and has at most that many columns, as for the CNN's narrow layers):
//   * warp 0, one lane: producer - the tensor-memory accelerator copies 128 x 64 (A) and
//     64 x BN (B) operand tiles into a ring of STAGES shared-memory stages
//     (cp.async.bulk.tensor, 128-byte swizzle, zero fill outside the matrices), each
//     stage tracked by a "full" mbarrier (transaction bytes) and an "empty" mbarrier;
//   * warp 1, one lane: issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction, FP32
//     accumulator in tensor memory); tcgen05.commit on a stage's "empty" barrier frees it
//     once the MMAs reading it have completed, and a last commit signals the epilogue;
//   * all four warps: epilogue - each warp reads its 32 tensor-memory lanes (rows) with
//     tcgen05.ld, scales and stores C.  When the roles of A and B were exchanged (C^T =
//     op(B)^T op(A)^T, chosen for M < 128 <= N), rows of the accumulator are columns of
//     C and the stores are transposed (consecutive threads then write consecutive n).
// Operands whose K index is contiguous in memory are "K-major" tiles (rows of 64 K values
// = 128 bytes); operands whose M / N index is contiguous are "MN-major" tiles (rows of 64
// M / N values, one row per K index, two 64-wide chunks for 128 rows), both in the
// canonical 128-byte-swizzled layouts of the tcgen05 shared-memory matrix descriptor.
// Every wait on an mbarrier has an iteration and clock bound: past it the CTA records a
// timeout in the library's device status, waits (bounded) for its own copies and MMAs,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "bsct_internal.h"

namespace bsct {

namespace tc {

constexpr int BM = 128, BK = 64, STAGES = 3, THREADS = 128;
constexpr int A_BYTES = BM * BK * 2;
// tile width BN (128, or 64 / 32 for narrow K-major B operands): bytes of a B tile and of a stage
template <int BN> __host__ __device__ constexpr int b_bytes() { return BN * BK * 2; }
template <int BN> __host__ __device__ constexpr int stage_bytes() { return A_BYTES + b_bytes<BN>(); }
// (the epilogue reuses the stage ring for its per-warp 32 x 33 transposition tiles)
template <int BN> __host__ __device__ constexpr int smem_bytes() {
  return STAGES * stage_bytes<BN>() + 1024 /* alignment */ + 256 /* barriers */;
}
static_assert(4 * 32 * 33 * 4 <= STAGES * stage_bytes<32>(), "epilogue tiles fit in the stage ring");
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false when it gave up (or another role already gave up: *abort)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  for (unsigned it = 0; it < (1u << 26); ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > WAIT_CYCLES) break;
  }
  *abort = 1;
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// shared-memory matrix descriptor, 128-byte swizzle (layout type 2), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// instruction descriptor of kind::f16: BF16 A and B, FP32 D, majors, N, M = 128
__host__ __device__ constexpr uint32_t instr_desc(int n, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// A_MN / B_MN: the operand tile is MN-major (M / N contiguous in memory); TRANS_C: the
// accumulator rows are columns of C (roles of A and B exchanged by the host)
template <bool A_MN, bool B_MN, bool TRANS_C, int BN>
__global__ void __launch_bounds__(THREADS, 2)
k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N, int K,
          float alpha, float beta, float* __restrict__ C, long ldc, long sC, int a_bcast, int b_bcast,
          unsigned int* status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  // 1024-byte aligned stage ring (the swizzle atoms), barriers and the TMEM address after it
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  static_assert(BN == 128 || (!B_MN && (BN == 64 || BN == 32)), "narrow tiles need a K-major B operand");
  constexpr int B_BYTES = b_bytes<BN>(), STAGE_BYTES = stage_bytes<BN>();
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(base + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN, bz = blockIdx.z;
  const int za = a_bcast ? 0 : bz, zb = b_bcast ? 0 : bz;  // batch coordinates (0: one matrix for all)
  const int nk = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    int issued = 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (kt / STAGES) & 1;
      if (kt >= STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1, abort)) break;
      const uint32_t sa = smem_u32(base + s * STAGE_BYTES), sb = sa + A_BYTES;
      mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
      if (A_MN) {  // two 64-wide M chunks of 64 K rows
        tma_load_3d(sa, &mapA, full0 + 8 * s, m0, kt * BK, za);
        tma_load_3d(sa + A_BYTES / 2, &mapA, full0 + 8 * s, m0 + 64, kt * BK, za);
      } else {
        tma_load_3d(sa, &mapA, full0 + 8 * s, kt * BK, m0, za);
      }
      if (B_MN) {
        tma_load_3d(sb, &mapB, full0 + 8 * s, n0, kt * BK, zb);
        tma_load_3d(sb + B_BYTES / 2, &mapB, full0 + 8 * s, n0 + 64, kt * BK, zb);
      } else {
        tma_load_3d(sb, &mapB, full0 + 8 * s, kt * BK, n0, zb);
      }
      ++issued;
    }
    // stages whose copies were issued but never waited for by the MMA loop (abort only)
    if (*abort) {
      for (int kt = issued - STAGES > 0 ? issued - STAGES : 0; kt < issued; ++kt) {
        volatile int no_abort = 0;
        mbar_wait(full0 + 8 * (kt % STAGES), (kt / STAGES) & 1, &no_abort);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t IDESC = instr_desc(BN, A_MN, B_MN);
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (kt / STAGES) & 1;
      if (!mbar_wait(full0 + 8 * s, ph, abort)) break;
      fence_after();
      const uint32_t sa = smem_u32(base + s * STAGE_BYTES), sb = sa + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        // K-major: +32 bytes per 16 K values inside the swizzled 128-byte rows (LBO unused,
        // SBO = 8 rows of 128 bytes); MN-major: +16 rows of 128 bytes, LBO = the second
        // 64-wide chunk, SBO = 8 rows of 128 bytes
        const uint64_t da = A_MN ? smem_desc(sa + kk * 2048, A_BYTES / 2, 1024) : smem_desc(sa + kk * 32, 16, 1024);
        const uint64_t db = B_MN ? smem_desc(sb + kk * 2048, B_BYTES / 2, 1024) : smem_desc(sb + kk * 32, 16, 1024);
        mma_f16(tmem, da, db, IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);  // also after an abort: the epilogue then knows every MMA has completed
  }
  __syncwarp();

  // epilogue (all four warps; warp w owns accumulator lanes 32 w .. 32 w + 31)
  const bool ok = mbar_wait(done, 0, abort) && !*abort;
  fence_after();
  if (ok) {
    const int row = warp * 32 + lane;  // accumulator row
    float* Cb = C + (long)bz * sC;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (!TRANS_C) {
        // transpose the warp's 32 x 32 chunk through shared memory (the free stage ring) so
        // that every store instruction writes one row segment of 32 consecutive floats
        float* t = reinterpret_cast<float*>(base) + warp * (32 * 33);
#pragma unroll
        for (int j = 0; j < 32; ++j) t[lane * 33 + j] = v[j];
        __syncwarp();
        const int n = n0 + c0 + lane;
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const int m = m0 + warp * 32 + r;
          if (m < M && n < N) {
            float* p = Cb + (long)m * ldc + n;
            const float o = alpha * t[r * 33 + lane];
            *p = beta != 0.f ? fmaf(beta, *p, o) : o;
          }
        }
        __syncwarp();
      } else {
        // accumulator (row = n, column = m): C[m][n]
        const int n = m0 + row;
        if (n < N) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int m = n0 + c0 + j;
            if (m < M) {
              float* p = Cb + (long)m * ldc + n;
              *p = beta != 0.f ? fmaf(alpha, v[j], beta * *p) : alpha * v[j];
            }
          }
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicOr(status, 1u);  // a bounded wait gave up
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// tensor map of one operand: `rows` x `cols` row-major with leading dimension ld (elements),
// batch stride sb (elements; 0 = the same matrix for every batch), box of 64 columns x
// box_rows rows, 128-byte swizzle, zero fill outside
static bool make_map(CUtensorMap* map, const void* ptr, long rows, long cols, long ld, long sb, int batch,
                     int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)(sb > 0 ? batch : 1)};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)(sb > 0 ? sb : ld * rows) * 2};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

// one instantiation: shared-memory opt-in once per device, then the launch
template <bool XMN, bool YMN, bool TC, int BN>
static int launch_tc(dim3 grid, const CUtensorMap& mx, const CUtensorMap& my, int M, int N, int K, float alpha,
                     float beta, float* C, long ldc, long sC, int x_bc, int y_bc, unsigned int* status,
                     cudaStream_t st) {
  using namespace tc;
  static bool attr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!attr[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<XMN, YMN, TC, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               smem_bytes<BN>());
    if (e != cudaSuccess) {
      bsct_set_last_cuda_error(e);
      return BSCT_ERR_CUDA;
    }
    attr[dev] = true;
  }
  k_gemm_tc<XMN, YMN, TC, BN><<<grid, THREADS, smem_bytes<BN>(), st>>>(mx, my, M, N, K, alpha, beta, C, ldc, sC, x_bc, y_bc,
                                                              status);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    bsct_set_last_cuda_error(e);
    bsct_set_last_message("tcgen05 GEMM launch failed");
    return BSCT_ERR_CUDA;
  }
  return BSCT_OK;
}

// The tcgen05 path of gemm_bf16 (same arguments and requirements).  Returns
// BSCT_ERR_UNSUPPORTED_SIZE when the operands cannot be described to the copy engine
// (the caller then uses the warp-level MMA path).
int gemm_bf16_tc(bool ta, bool tb, int M, int N, int K, float alpha, const void* A, long lda, long sA, const void* B,
                 long ldb, long sB, float beta, float* C, long ldc, long sC, int batch, cudaStream_t st) {
  using namespace tc;
  // exchange the roles of A and B when M is small and N large (M >= 128 keeps the MMA full)
  const bool swap = M < BM && N > M;
  // operand X (accumulator rows: M, or N when swapped) and Y (accumulator columns)
  const int MX = swap ? N : M, NY = swap ? M : N;
  // X tile K-major iff its K index is contiguous: A row-major (!ta) or, swapped, B stored N x K (tb)
  const bool x_mn = swap ? !tb : ta;
  const bool y_mn = swap ? ta : !tb;
  const void* X = swap ? B : A;
  const void* Y = swap ? A : B;
  const long ldx = swap ? ldb : lda, ldy = swap ? lda : ldb;
  const long sx = swap ? sB : sA, sy = swap ? sA : sB;
  if ((lda % 8) || (ldb % 8) || (sA % 8) || (sB % 8) || (((uintptr_t)A) & 15) || (((uintptr_t)B) & 15))
    return BSCT_ERR_UNSUPPORTED_SIZE;
  CUtensorMap mx, my;
  // K-major: rows = M or N, cols = K; MN-major: rows = K, cols = M or N
  // narrow K-major B operands (N = 32 or 64 columns, the CNN's small channel counts) use
  // a tile of that width so that the MMA and its tensor memory do no padding work
  const int BNsel = y_mn ? 128 : (NY <= 32 ? 32 : (NY <= 64 ? 64 : 128));
  const bool okx = x_mn ? make_map(&mx, X, K, MX, ldx, sx, batch, BK) : make_map(&mx, X, MX, K, ldx, sx, batch, BM);
  const bool oky = y_mn ? make_map(&my, Y, K, NY, ldy, sy, batch, BK) : make_map(&my, Y, NY, K, ldy, sy, batch, BNsel);
  if (!okx || !oky) return BSCT_ERR_UNSUPPORTED_SIZE;
  unsigned int* status = timeout_status_ptr();
  if (!status) return BSCT_ERR_CUDA;
  const int x_bc = (swap ? sB : sA) == 0 && batch > 1, y_bc = (swap ? sA : sB) == 0 && batch > 1;
  dim3 grid((NY + BNsel - 1) / BNsel, (MX + BM - 1) / BM, batch);
#define BSCT_TC(XM, YM, TCV, BNV) \
  return launch_tc<XM, YM, TCV, BNV>(grid, mx, my, M, N, K, alpha, beta, C, ldc, sC, x_bc, y_bc, status, st)
  if (y_mn) {
    if (!swap) { if (x_mn) BSCT_TC(true, true, false, 128); else BSCT_TC(false, true, false, 128); }
    if (x_mn) BSCT_TC(true, true, true, 128); else BSCT_TC(false, true, true, 128);
  }
  if (BNsel == 32) {
    if (!swap) { if (x_mn) BSCT_TC(true, false, false, 32); else BSCT_TC(false, false, false, 32); }
    if (x_mn) BSCT_TC(true, false, true, 32); else BSCT_TC(false, false, true, 32);
  }
  if (BNsel == 64) {
    if (!swap) { if (x_mn) BSCT_TC(true, false, false, 64); else BSCT_TC(false, false, false, 64); }
    if (x_mn) BSCT_TC(true, false, true, 64); else BSCT_TC(false, false, true, 64);
  }
  if (!swap) { if (x_mn) BSCT_TC(true, false, false, 128); else BSCT_TC(false, false, false, 128); }
  if (x_mn) BSCT_TC(true, false, true, 128); else BSCT_TC(false, false, true, 128);
#undef BSCT_TC
}

}  // namespace bsct
