// Internal (C++) interfaces between the libbsct translation units.
#pragma once
#include <atomic>
#include <cuda_runtime.h>

#include "bsct_common.cuh"

namespace bsct {

// Launch counter (exported through bsct_launch_count).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// Optional per-kernel timing of the Gram apply (CUDA events recorded on the launching
// stream between its kernels; off unless bsct_set_kernel_timing(1)).
struct KernelTimer {
  bool on = false;
  bool created = false;
  cudaEvent_t ev[4];
  int n_recorded = 0;
};
extern KernelTimer g_timer;
inline void timer_mark(cudaStream_t st, int i) {
  if (!g_timer.on) return;
  if (!g_timer.created) {
    for (int k = 0; k < 4; ++k) cudaEventCreate(&g_timer.ev[k]);
    g_timer.created = true;
  }
  cudaEventRecord(g_timer.ev[i], st);
  g_timer.n_recorded = i + 1;
}

// Programmatic dependent launch of the Gram-apply kernels: a kernel launched by
// launch_overlap() may be scheduled while the previous kernel of the stream is still
// running its last CTAs.  Each such kernel calls pdl_trigger() first (its own successor
// may then be scheduled once all of its CTAs have started) and pdl_wait() before its
// first global-memory access; pdl_wait returns once the previous grid has completed.
// The L1 invalidation between dependent grids can then precede the predecessor's
// stores, so these kernels read every datum another kernel wrote through L2 only
// (ld_cpx_cg, __ldcg, cp.async.cg); only constant tables go through L1.
// On by default; bsct_set_launch_overlap(0) launches them plainly.
extern bool g_overlap;
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KP, typename... A>
inline cudaError_t launch_overlap(void (*k)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = g_overlap ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KP>(args)...);
}

// CG scalars in device memory (FP64), 16 slots per CG state; the last two hold the
// arrival counters of the last-block reductions below (zero between launches).
// SC_RR holds <r, r> for CG and rho = <r, M^-1 r> for preconditioned CG, whose <r, r>
// (the convergence measure) goes to SC_RRP
enum { SC_RR = 0, SC_PQ = 1, SC_ALPHA = 2, SC_BETA = 3, SC_BB = 4, SC_TMP = 5, SC_RRP = 6, /* 7: graph iterations */
       SC_CNT_PQ = 14, SC_CNT_RR = 15 };
__device__ __forceinline__ unsigned long long* sc_counter(double* sc, int slot) {
  return reinterpret_cast<unsigned long long*>(sc + slot);
}

// Last-block reduction: thread 0 of every CTA has written its partial to part[blockIdx.x];
// the CTA that arrives last sums part[0 .. gridDim.x) in index order (so the result does
// not depend on which CTA that is), calls fin(sum) in thread 0 and resets the counter.
// ws: shared scratch of blockDim.x doubles.  Called by all threads of every CTA.
template <typename F>
__device__ __forceinline__ void last_block_sum(const double* part, unsigned long long* cnt, double* ws, F fin) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(cnt, 1ull) == (unsigned long long)gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(part + i);
  if (blockDim.x % 32 == 0) {  // shuffle tree (FP64 adds are slow: keep the chain short)
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = threadIdx.x < (int)(blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) {
        fin(t);
        *cnt = 0ull;
      }
    }
  } else {  // blocks of fewer than 32 threads
    ws[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)blockDim.x; ++i) t += ws[i];
      fin(t);
      *cnt = 0ull;
    }
  }
}

// FFT convolution kernels for one image size N (row FFT length N, column length 2N).
//   S:   N x N complex scratch (row-block interleaved half spectra)
//   Gt:  spectrum, [N+1][2N] real, scaled by 1/(2N)^2 (row 0 = (G0+GN)/2, row N = (G0-GN)/2)
//   tw:  8N twiddles (fft_table_elems): [0, 2N) exp(-2 pi i k / 2N) for the real/complex
//        untangling, then the stage tables of the row plan (forward order, reversed
//        order; N each) and of the column plan (2N each)
template <typename T> struct FftOps {
  int (*apply)(const T* x, T* y, cpx<T>* S, const T* Gt, const cpx<T>* tw, cudaStream_t st);
  // CG step q = G p with p = r + beta p done in the first pass (p overwritten,
  // beta = sc[SC_BETA]); the last pass writes per-CTA partial sums of <p, q> to
  // part[0 .. cg_partials) and its last CTA turns them into sc[SC_PQ] and
  // sc[SC_ALPHA] = sc[SC_RR] / <p, q>
  int (*apply_cg)(const T* r, T* p, T* q, double* sc, double* part, cpx<T>* S, const T* Gt, const cpx<T>* tw,
                  cudaStream_t st);
  int cg_partials;
  // preconditioner step z = M^-1 r, the apply with spectrum Mt: the last pass writes
  // per-CTA partial sums of rho = <r, z> to part[0 .. cg_partials) and its last CTA forms
  // sc[SC_BETA] = rho / sc[SC_RR] (0 when sc[SC_RR] <= 0) and sc[SC_RR] = rho
  int (*apply_pc)(const T* r, T* z, double* sc, double* part, cpx<T>* S, const T* Mt, const cpx<T>* tw,
                  cudaStream_t st);
  // launch shapes of the three passes (rows per CTA of the forward and inverse row pass,
  // CTAs per SM of the column pass): the row counts of the three candidates of each row
  // pass (0 where not valid for this size), and the current choice as candidate indices
  // (idx[2]: 0 = occupancy limit, 1 = one CTA per SM), read (set = 0) or set after
  // validation (set = 1), per device and precision
  void (*shape_cands)(int fwd[3], int inv[3]);
  int (*shape_index)(int idx[3], int set);
  // emb: 2N x 2N real circulant kernel; S2: 2N x N complex scratch; writes Gt (scaled)
  int (*spectrum)(const T* emb, cpx<T>* S2, T* Gt, const cpx<T>* tw, cudaStream_t st);
};
template <typename T, int N> FftOps<T> fft_ops();
template <typename T> bool fft_ops_for(int N, FftOps<T>* out);

inline long fft_table_elems(int N) { return 8L * N; }

// Non-finite input detection (status.cu): the device address of this device's status
// words (word 0: the sticky flag read by bsct_input_status), and a check of n values of
// p that sets status word `word` when one is not finite (asynchronous).
unsigned int* input_status_ptr();
unsigned int* timeout_status_ptr();  // word 2: a kernel's bounded wait gave up
template <typename T> int check_finite_async(const T* p, long n, cudaStream_t st, int word = 0);
// fill the 8N-entry twiddle array of size N (see FftOps)
template <typename T> int build_fft_tables(cpx<T>* d_tw, int N, cudaStream_t st);

// Back projection split into its per-geometry and per-sinogram parts (device memory
// owned by the caller of these functions).
struct BpPlan {
  int N = 0, na = 0, M = 0;
  double lambda = 1.0, zeta = 0.0;
  double* ang = nullptr;     // [na] half turns (device)
  double* p00 = nullptr;     // [na]
  double2* csl = nullptr;    // [na] (cos, sin) / lambda
  void* tab = nullptr;       // bp_table_bytes(na, precision)
  int* status = nullptr;
  float* part = nullptr;     // bp_partial_bytes(N, na, lambda, precision) of scratch (may be 0 bytes)
};
template <typename T> int bp_make_tables(const BpPlan& p, cudaStream_t st);
template <typename T> int bp_apply(const BpPlan& p, const T* sino, T* ct, T* b, cudaStream_t st);
size_t bp_table_bytes(int n_angles, int precision);
int bp_view_split(int N, int na, double lambda, int precision);
size_t bp_partial_bytes(int N, int na, double lambda, int precision);

// split-BF16 DFT-GEMM Gram apply (dftgemm.cu)
bool dftgemm_factor(int L, int* P, int* Q);
size_t dftgemm_scratch_bytes(int N);
int dftgemm_apply(int N, const float* x, float* y, const float* Gt, const float2* tw_untangle, void* work,
                  cudaStream_t st);
int gemm_bf16(bool ta, bool tb, int M, int N, int K, float alpha, const void* A, long lda, long sA, const void* B,
              long ldb, long sB, float beta, float* C, long ldc, long sC, int batch, cudaStream_t st);
// the tcgen05 path (gemm_tc.cu); BSCT_ERR_UNSUPPORTED_SIZE when the copy engine cannot
// describe the operands
int gemm_bf16_tc(bool ta, bool tb, int M, int N, int K, float alpha, const void* A, long lda, long sA, const void* B,
                 long ldb, long sB, float beta, float* C, long ldc, long sC, int batch, cudaStream_t st);
extern int g_gemm_path;  // 0: tcgen05 (default), 1: warp-level mma.sync

}  // namespace bsct

int bsct_check_geom(const bsct_geom* g);
// detector boxes of a geometry (checked): their number (0, 1 or 2) and widths
int bsct_blur_boxes(const bsct_geom* g, double w[2]);
int bsct_check_bp_geom(const bsct_geom* g);

namespace bsct {
// two detector boxes (multibox.cu): back projection and forward projection of a checked geometry
int mb_check_bp(const bsct_geom* g);
size_t mb_bp_workspace(const bsct_geom* g, int precision);
template <typename T> int mb_bp_run(const bsct_geom* g, const T* sino, T* b, char* work, cudaStream_t st);
size_t mb_fp_workspace(const bsct_geom* g, int precision);
template <typename T> int mb_fp_run(const bsct_geom* g, const T* c, T* sino, char* work, cudaStream_t st);
}  // namespace bsct

// Library-owned state of one geometry (see bsct_gram_build).
struct bsct_host_pipe;  // streams, events and device images of bsct_gram_apply_host
void bsct_host_pipe_free(bsct_host_pipe* p);
struct bsct_graph_solver;  // executable graph of bsct_solve_graph
void bsct_graph_solver_free(bsct_graph_solver* s);

struct bsct_gram {
  int N = 0, precision = 0, n_angles = 0;
  double zeta = 0.0, lambda = 1.0;
  double* taps = nullptr;    // (2N-1)^2 FP64 taps
  double* Gt64 = nullptr;    // scaled spectrum [N+1][2N], FP64
  float* Gt32 = nullptr;     // same, FP32 (precision F32 only)
  void* tw = nullptr;        // FFT twiddle tables (T), fft_table_elems(N) entries
  void* S = nullptr;         // apply scratch, N x N complex T
  void* r = nullptr;         // CG vectors (T, N*N each)
  void* p = nullptr;
  void* q = nullptr;
  double* scal = nullptr;    // CG scalars
  double* partials = nullptr;
  int n_partials = 0;
  bool owns_filter = true;   // false for batch slices sharing another handle's taps/spectrum/twiddles
  void* dg_work = nullptr;   // DFT-GEMM scratch, allocated on first DFT-GEMM apply
  void* z = nullptr;         // preconditioned residual (T, N*N), allocated on first use
  double* Mt64 = nullptr;    // circulant preconditioner spectrum [N+1][2N], packed like Gt64
  float* Mt32 = nullptr;     // same, FP32 (precision F32 only)
  double m_eps = -1.0;       // floor the preconditioner spectrum was built with
  bsct_host_pipe* pipe = nullptr;  // created on the first host-memory apply
  bsct_graph_solver* sgraph = nullptr;  // created on the first graph solve
  size_t dg_bytes = 0;
};
