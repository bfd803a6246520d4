// Conjugate gradients on the normal equations G x = b (Sec. 2) with the Gram filter
// applied by FFT convolution (Sec. 4).  Vectors in the handle's precision T; inner
// products reduced in FP64 and the step scalars alpha, beta kept in FP64 in device
// memory, so an iteration never waits for the host:
//
//   p = r + beta p; q = G p; <p, q>     (gram apply with the update fused into its
//                                         first pass and the inner product into its
//                                         last pass, whose last CTA forms
//                                         alpha = rr / pq)
//   x += alpha p;  r -= alpha q;  <r, r> (k_xr_update; its last CTA forms
//   beta = rr_new / rr;  rr = rr_new      beta and rr; beta = 0 before the first iteration)
// so one iteration is four kernels and the scalar reductions need no launches of their own.
// Steepest descent (the solver of the paper's reconstruction study, Sec. 6) is the same
// iteration with beta held at 0, i.e. the direction is always the residual.
#include "bsct_internal.h"

namespace bsct {

enum { OP_STORE_RR = 0, OP_STORE_BB = 1, OP_ALPHA = 2, OP_STORE_TMP = 4, OP_STORE_RRP = 5 };

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[RED_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < RED_THREADS / 32 ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_dot(const T* __restrict__ a, const T* __restrict__ b, long n,
                                                     double* __restrict__ part) {
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// ||a - b||^2
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_diff2(const T* __restrict__ a, const T* __restrict__ b, long n,
                                                       double* __restrict__ part) {
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double d = (double)a[i] - (double)b[i];
    acc += d * d;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(RED_THREADS) k_finish(const double* __restrict__ part, int np, double* __restrict__ sc,
                                                        int op) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    switch (op) {
      case OP_STORE_RR: sc[SC_RR] = acc; break;
      case OP_STORE_BB: sc[SC_BB] = acc; break;
      // an exactly zero residual (or <p, Gp> <= 0) stops the update instead of 0 / 0
      case OP_ALPHA: sc[SC_PQ] = acc; sc[SC_ALPHA] = acc > 0.0 ? sc[SC_RR] / acc : 0.0; break;
      case OP_STORE_TMP: sc[SC_TMP] = acc; break;
      case OP_STORE_RRP: sc[SC_RRP] = acc; break;
    }
  }
}

// x += alpha p; r -= alpha q; partial <r, r> (4 elements per thread step); the last CTA
// forms beta = <r, r>_new / <r, r> (0 for an exactly zero residual) and stores <r, r>_new
template <typename T> struct V4;
template <> struct V4<float> { typedef float4 t; };
template <> struct V4<double> { typedef double4 t; };

// What the last CTA does with <r, r>_new: CG forms beta = <r, r>_new / <r, r> and stores
// <r, r>_new; PCG stores it in sc[SC_RRP] only (beta comes from the preconditioner
// step); steepest descent stores it and keeps beta = 0 (the next direction is r)
enum { UPD_CG = 0, UPD_PCG = 1, UPD_SD = 2 };
template <typename T, int UPD = UPD_CG>
__global__ void __launch_bounds__(RED_THREADS) k_xr_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                           const T* __restrict__ q, double* __restrict__ sc, long n,
                                                           double* __restrict__ part) {
  typedef typename V4<T>::t v4;
  const T alpha = T(sc[SC_ALPHA]);
  double acc = 0.0;
  const long n4 = n / 4;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
    v4 xv = reinterpret_cast<v4*>(x)[i], rv = reinterpret_cast<v4*>(r)[i];
    const v4 pv = reinterpret_cast<const v4*>(p)[i], qv = reinterpret_cast<const v4*>(q)[i];
    xv.x = fma(alpha, pv.x, xv.x); xv.y = fma(alpha, pv.y, xv.y);
    xv.z = fma(alpha, pv.z, xv.z); xv.w = fma(alpha, pv.w, xv.w);
    rv.x = fma(-alpha, qv.x, rv.x); rv.y = fma(-alpha, qv.y, rv.y);
    rv.z = fma(-alpha, qv.z, rv.z); rv.w = fma(-alpha, qv.w, rv.w);
    reinterpret_cast<v4*>(x)[i] = xv;
    reinterpret_cast<v4*>(r)[i] = rv;
    const T s4 = rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
    acc += (double)s4;
  }
  for (long i = n4 * 4 + (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const T ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    acc += (double)ri * (double)ri;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  __shared__ double lb_ws[RED_THREADS];
  last_block_sum(part, sc_counter(sc, SC_CNT_RR), lb_ws, [&](double rr) {
    if constexpr (UPD == UPD_PCG) {
      sc[SC_RRP] = rr;
    } else if constexpr (UPD == UPD_SD) {
      sc[SC_BETA] = 0.0;
      sc[SC_RR] = rr;
    } else {
      sc[SC_BETA] = sc[SC_RR] > 0.0 ? rr / sc[SC_RR] : 0.0;
      sc[SC_RR] = rr;
    }
  });
}

template <typename T>
__global__ void k_p_update(T* __restrict__ p, const T* __restrict__ r, const double* __restrict__ sc, long n) {
  const T beta = T(sc[SC_BETA]);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], r[i]);
}

// r = b - q (q = G x0), p = r
template <typename T>
__global__ void k_init_r(const T* __restrict__ b, const T* __restrict__ q, T* __restrict__ r, T* __restrict__ p, long n,
                         int has_x0) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T v = has_x0 ? b[i] - q[i] : b[i];
    r[i] = v;
    p[i] = v;
  }
}

// Preconditioner spectrum from the Gram spectrum, in the same packed, scaled layout
// [N+1][2N]: rows 1 .. N-1 hold G^(u, v) / L^2, rows 0 and N hold (G^(u,0) +- G^(u,N)) / 2L^2.
// Each value becomes 1 / max(G^, eps G^(0,0)) (L = 2N); one thread per (u, v < N), the
// v = 0 thread also writes row N.
__global__ void k_precond_spectrum(const double* __restrict__ Gt, int N, double eps, double* __restrict__ Mt,
                                   float* __restrict__ Mt32) {
  const int L = 2 * N;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)L * N) return;
  const int v = (int)(i / L), u = (int)(i % L);
  const double sc = (double)L * (double)L;
  const double floor_ = eps * (Gt[0] + Gt[(long)N * L]) * sc;  // eps G^(0, 0)
  if (v == 0) {
    const double a = Gt[u], b = Gt[(long)N * L + u];
    const double h0 = 1.0 / fmax((a + b) * sc, floor_), hN = 1.0 / fmax((a - b) * sc, floor_);
    const double m0 = 0.5 * (h0 + hN) / sc, mN = 0.5 * (h0 - hN) / sc;
    Mt[u] = m0;
    Mt[(long)N * L + u] = mN;
    if (Mt32) { Mt32[u] = (float)m0; Mt32[(long)N * L + u] = (float)mN; }
  } else {
    const double m = 1.0 / fmax(Gt[i] * sc, floor_) / sc;
    Mt[i] = m;
    if (Mt32) Mt32[i] = (float)m;
  }
}

template <typename T> __global__ void k_zero(T* __restrict__ x, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] = T(0);
}

}  // namespace bsct

using namespace bsct;

static int nblk(const bsct_gram* g, long n) {
  long b = (n + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
  if (b < 1) b = 1;
  if (b > g->n_partials) b = g->n_partials;
  return (int)b;
}

static int apply_g(const bsct_gram* g, const void* x, void* y, cudaStream_t st) {
  return bsct_gram_apply(g, x, y, g->precision == BSCT_F32 ? BSCT_APPLY_FFT32 : BSCT_APPLY_F64, st);
}

template <typename T>
static int cg_begin_t(bsct_gram* g, const T* b, T* x, int x0_is_zero, cudaStream_t st) {
  const long n = (long)g->N * g->N;
  const int nb = nblk(g, n);
  T* r = (T*)g->r;
  T* p = (T*)g->p;
  T* q = (T*)g->q;
  if (x0_is_zero) {
    k_zero<T><<<nb, RED_THREADS, 0, st>>>(x, n);
    count_launch();
  } else {
    int rc = apply_g(g, x, q, st);
    if (rc != BSCT_OK) return rc;
  }
  k_init_r<T><<<nb, RED_THREADS, 0, st>>>(b, q, r, p, n, x0_is_zero ? 0 : 1);
  BSCT_CUDA_TRY(cudaMemsetAsync(g->scal + SC_BETA, 0, sizeof(double), st));  // first direction p = r
  BSCT_CUDA_TRY(cudaMemsetAsync(g->scal + SC_CNT_PQ, 0, 2 * sizeof(double), st));  // reduction counters
  k_dot<T><<<nb, RED_THREADS, 0, st>>>(r, r, n, g->partials);
  k_finish<<<1, RED_THREADS, 0, st>>>(g->partials, nb, g->scal, OP_STORE_RR);
  k_dot<T><<<nb, RED_THREADS, 0, st>>>(b, b, n, g->partials);
  k_finish<<<1, RED_THREADS, 0, st>>>(g->partials, nb, g->scal, OP_STORE_BB);
  count_launch(5);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

template <typename T, int UPD = UPD_CG>
static int cg_iter_t(bsct_gram* g, T* x, int n_iter, cudaStream_t st) {
  const long n = (long)g->N * g->N;
  const int nb = nblk(g, n);
  T* r = (T*)g->r;
  T* p = (T*)g->p;
  T* q = (T*)g->q;
  FftOps<T> o;
  if (!fft_ops_for<T>(g->N, &o)) return BSCT_ERR_UNSUPPORTED_SIZE;
  const T* Gt = (g->precision == BSCT_F32) ? (const T*)(const void*)g->Gt32 : (const T*)(const void*)g->Gt64;
  if (o.cg_partials > g->n_partials) return BSCT_ERR_UNSUPPORTED_SIZE;
  for (int it = 0; it < n_iter; ++it) {
    int rc = o.apply_cg(r, p, q, g->scal, g->partials, (cpx<T>*)g->S, Gt, (const cpx<T>*)g->tw, st);
    if (rc != BSCT_OK) return rc;
    k_xr_update<T, UPD><<<nb, RED_THREADS, 0, st>>>(x, r, p, q, g->scal, n, g->partials);
    count_launch(1);
  }
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

extern "C" int bsct_cg_begin(bsct_gram* g, const void* d_b, void* d_x, int x0_is_zero, void* stream) {
  if (!g || !d_b || !d_x) { bsct_set_last_message("NULL argument"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (g->precision == BSCT_F32) return cg_begin_t<float>(g, (const float*)d_b, (float*)d_x, x0_is_zero, st);
  return cg_begin_t<double>(g, (const double*)d_b, (double*)d_x, x0_is_zero, st);
}

extern "C" int bsct_cg_iterate(bsct_gram* g, void* d_x, int n_iter, void* stream) {
  if (!g || !d_x || n_iter < 0) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (g->precision == BSCT_F32) return cg_iter_t<float>(g, (float*)d_x, n_iter, st);
  return cg_iter_t<double>(g, (double*)d_x, n_iter, st);
}

extern "C" int bsct_cg_residual(const bsct_gram* g, double* rr, double* bb, void* stream) {
  if (!g) { bsct_set_last_message("NULL handle"); return BSCT_ERR_INVALID_ARG; }
  double h[16];
  cudaStream_t st = (cudaStream_t)stream;
  BSCT_CUDA_TRY(cudaMemcpyAsync(h, g->scal, sizeof(h), cudaMemcpyDeviceToHost, st));
  BSCT_CUDA_TRY(cudaStreamSynchronize(st));
  if (rr) *rr = h[SC_RR];
  if (bb) *bb = h[SC_BB];
  return BSCT_OK;
}

template <typename T>
static int true_residual_t(bsct_gram* g, const T* b, const T* x, double* out, cudaStream_t st) {
  const long n = (long)g->N * g->N;
  const int nb = nblk(g, n);
  int rc = apply_g(g, x, g->q, st);
  if (rc != BSCT_OK) return rc;
  k_diff2<T><<<nb, RED_THREADS, 0, st>>>(b, (const T*)g->q, n, g->partials);
  k_finish<<<1, RED_THREADS, 0, st>>>(g->partials, nb, g->scal, OP_STORE_TMP);
  count_launch(2);
  BSCT_CUDA_TRY(cudaGetLastError());
  double h[16];
  BSCT_CUDA_TRY(cudaMemcpyAsync(h, g->scal, sizeof(h), cudaMemcpyDeviceToHost, st));
  BSCT_CUDA_TRY(cudaStreamSynchronize(st));
  *out = (h[SC_BB] > 0.0) ? sqrt(h[SC_TMP] / h[SC_BB]) : 0.0;
  return BSCT_OK;
}

// A right-hand side or an initial guess holding a non-finite value shows in <b, b> or in
// the initial <r, r>: the synchronous solvers stop before their first iteration.
static int check_start(double rr, double bb) {
  if (!isfinite(bb)) {
    bsct_set_last_message("the right-hand side b holds a non-finite value");
    return BSCT_ERR_NONFINITE;
  }
  if (!isfinite(rr)) {
    bsct_set_last_message("the initial residual is not finite (x0 holds a non-finite value)");
    return BSCT_ERR_NONFINITE;
  }
  return BSCT_OK;
}

// CG (steepest = false) or steepest descent (steepest = true): the same begin, state and
// stopping rule; steepest descent is the CG iteration with beta held at 0
static int krylov_solve(bsct_gram* g, const void* d_b, void* d_x, int x0_is_zero, int max_iter, double rel_tol,
                        int check_every, bsct_cg_report* report, void* stream, bool steepest) {
  if (!g || !d_b || !d_x || max_iter < 0) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  if (check_every < 1) check_every = 1;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = bsct_cg_begin(g, d_b, d_x, x0_is_zero, stream);
  if (rc != BSCT_OK) return rc;
  double rr = 0.0, bb = 0.0;
  int it = 0, converged = 0;
  rc = bsct_cg_residual(g, &rr, &bb, stream);
  if (rc != BSCT_OK) return rc;
  if ((rc = check_start(rr, bb)) != BSCT_OK) return rc;
  if (rel_tol > 0.0 && (bb == 0.0 || sqrt(rr / bb) <= rel_tol)) converged = 1;
  while (!converged && it < max_iter) {
    const int k = (rel_tol > 0.0) ? (check_every < max_iter - it ? check_every : max_iter - it) : max_iter - it;
    if (steepest)
      rc = g->precision == BSCT_F32 ? cg_iter_t<float, UPD_SD>(g, (float*)d_x, k, st)
                                    : cg_iter_t<double, UPD_SD>(g, (double*)d_x, k, st);
    else
      rc = bsct_cg_iterate(g, d_x, k, stream);
    if (rc != BSCT_OK) return rc;
    it += k;
    if (rel_tol > 0.0) {
      rc = bsct_cg_residual(g, &rr, &bb, stream);
      if (rc != BSCT_OK) return rc;
      if (!isfinite(rr)) { bsct_set_last_message("CG residual is not finite"); return BSCT_ERR_NONFINITE; }
      if (sqrt(rr / bb) <= rel_tol) converged = 1;
    }
  }
  rc = bsct_cg_residual(g, &rr, &bb, stream);
  if (rc != BSCT_OK) return rc;
  if (!isfinite(rr)) { bsct_set_last_message("CG residual is not finite"); return BSCT_ERR_NONFINITE; }
  double tr = -1.0;
  if (rel_tol > 0.0) {
    rc = (g->precision == BSCT_F32) ? true_residual_t<float>(g, (const float*)d_b, (const float*)d_x, &tr, st)
                                    : true_residual_t<double>(g, (const double*)d_b, (const double*)d_x, &tr, st);
    if (rc != BSCT_OK) return rc;
  }
  if (report) {
    report->iterations = it;
    report->converged = converged;
    report->rel_residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    report->true_rel_residual = tr;
  }
  return (rel_tol > 0.0 && !converged) ? BSCT_WARN_NOT_CONVERGED : BSCT_OK;
}

extern "C" int bsct_cg_solve(bsct_gram* g, const void* d_b, void* d_x, int x0_is_zero, int max_iter, double rel_tol,
                             int check_every, bsct_cg_report* report, void* stream) {
  return krylov_solve(g, d_b, d_x, x0_is_zero, max_iter, rel_tol, check_every, report, stream, false);
}

extern "C" int bsct_sd_solve(bsct_gram* g, const void* d_b, void* d_x, int x0_is_zero, int max_iter, double rel_tol,
                             int check_every, bsct_cg_report* report, void* stream) {
  return krylov_solve(g, d_b, d_x, x0_is_zero, max_iter, rel_tol, check_every, report, stream, true);
}

// CG whose operator is the split-BF16 DFT-GEMM apply (unfused: p update, apply, <p, q>),
// followed by iterative refinement: the FP32 FFT apply recomputes the true residual
// b - G x and n_refine FP32 CG iterations continue from x.
extern "C" int bsct_cg_solve_mixed(bsct_gram* g, const void* d_b, void* d_x, int n_low, int n_refine,
                                   bsct_cg_report* report, void* stream) {
  if (!g || !d_b || !d_x || n_low < 0 || n_refine < 0) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  if (g->precision != BSCT_F32) { bsct_set_last_message("mixed CG needs an F32 handle"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const long n = (long)g->N * g->N;
  const int nb = nblk(g, n);
  float* x = (float*)d_x;
  float* r = (float*)g->r;
  float* p = (float*)g->p;
  float* q = (float*)g->q;
  int rc = bsct_cg_begin(g, d_b, d_x, 1, stream);
  if (rc != BSCT_OK) return rc;
  {
    double rr0 = 0.0, bb0 = 0.0;
    if ((rc = bsct_cg_residual(g, &rr0, &bb0, stream)) != BSCT_OK) return rc;
    if ((rc = check_start(rr0, bb0)) != BSCT_OK) return rc;
  }
  for (int it = 0; it < n_low; ++it) {
    k_p_update<float><<<nb, RED_THREADS, 0, st>>>(p, r, g->scal, n);
    count_launch();
    rc = bsct_gram_apply(g, p, q, BSCT_APPLY_DFTGEMM_BF16, stream);
    if (rc != BSCT_OK) return rc;
    k_dot<float><<<nb, RED_THREADS, 0, st>>>(p, q, n, g->partials);
    k_finish<<<1, RED_THREADS, 0, st>>>(g->partials, nb, g->scal, OP_ALPHA);
    k_xr_update<float><<<nb, RED_THREADS, 0, st>>>(x, r, p, q, g->scal, n, g->partials);
    count_launch(3);
  }
  BSCT_CUDA_TRY(cudaGetLastError());
  if (n_refine > 0) {
    rc = bsct_cg_begin(g, d_b, d_x, 0, stream);  // r = b - G x with the FP32 apply
    if (rc == BSCT_OK) rc = bsct_cg_iterate(g, d_x, n_refine, stream);
    if (rc != BSCT_OK) return rc;
  }
  double rr = 0.0, bb = 0.0, tr = -1.0;
  rc = bsct_cg_residual(g, &rr, &bb, stream);
  if (rc == BSCT_OK) rc = true_residual_t<float>(g, (const float*)d_b, (const float*)d_x, &tr, st);
  if (rc != BSCT_OK) return rc;
  if (!isfinite(rr) || !isfinite(tr)) { bsct_set_last_message("residual is not finite"); return BSCT_ERR_NONFINITE; }
  if (report) {
    report->iterations = n_low + n_refine;
    report->converged = 0;
    report->rel_residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    report->true_rel_residual = tr;
  }
  return BSCT_OK;
}

// ------------------------------------------------------------------------------------
// Preconditioned CG with the circulant preconditioner M^-1 = P C^-1 P^T: C is the
// 2N-periodic circulant whose N x N section is G (G is Toeplitz-block-Toeplitz, Sec. 4),
// P the zero-padding, and C's symbol floored at eps G^(0).  M^-1 r is the FFT apply with
// the reciprocal spectrum.  One iteration is seven kernels:
//   p = z + beta p; q = G p; alpha = rho / <p, q>       (apply_cg, z in place of r)
//   x += alpha p; r -= alpha q; <r, r> -> SC_RRP         (k_xr_update<UPD_PCG>)
//   z = M^-1 r; rho_new = <r, z>; beta = rho_new / rho   (apply_pc)
// ------------------------------------------------------------------------------------
static int precond_ready(bsct_gram* g, double eps, cudaStream_t st) {
  if (!(eps > 0.0 && eps <= 1.0)) { bsct_set_last_message("eps must lie in (0, 1]"); return BSCT_ERR_INVALID_ARG; }
  const int N = g->N, L = 2 * N;
  const bool f32 = g->precision == BSCT_F32;
  const size_t T = f32 ? sizeof(float) : sizeof(double);
  if (!g->Mt64) BSCT_CUDA_TRY(cudaMalloc(&g->Mt64, (size_t)(N + 1) * L * sizeof(double)));
  if (f32 && !g->Mt32) BSCT_CUDA_TRY(cudaMalloc(&g->Mt32, (size_t)(N + 1) * L * sizeof(float)));
  if (!g->z) BSCT_CUDA_TRY(cudaMalloc(&g->z, (size_t)N * N * T));
  if (g->m_eps != eps) {
    const long n = (long)L * N;
    k_precond_spectrum<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g->Gt64, N, eps, g->Mt64, f32 ? g->Mt32 : nullptr);
    count_launch();
    BSCT_CUDA_TRY(cudaGetLastError());
    g->m_eps = eps;
  }
  return BSCT_OK;
}

template <typename T> static const T* precond_spectrum(const bsct_gram* g) {
  return (g->precision == BSCT_F32) ? (const T*)(const void*)g->Mt32 : (const T*)(const void*)g->Mt64;
}

template <typename T>
static int precond_apply_t(bsct_gram* g, const T* x, T* y, cudaStream_t st) {
  FftOps<T> o;
  if (!fft_ops_for<T>(g->N, &o)) return BSCT_ERR_UNSUPPORTED_SIZE;
  return o.apply(x, y, (cpx<T>*)g->S, precond_spectrum<T>(g), (const cpx<T>*)g->tw, st);
}

template <typename T>
static int pcg_begin_t(bsct_gram* g, const T* b, T* x, int x0_is_zero, cudaStream_t st) {
  const long n = (long)g->N * g->N;
  const int nb = nblk(g, n);
  T* r = (T*)g->r;
  T* p = (T*)g->p;
  T* q = (T*)g->q;
  FftOps<T> o;
  if (!fft_ops_for<T>(g->N, &o)) return BSCT_ERR_UNSUPPORTED_SIZE;
  if (o.cg_partials > g->n_partials) return BSCT_ERR_UNSUPPORTED_SIZE;
  if (x0_is_zero) {
    k_zero<T><<<nb, RED_THREADS, 0, st>>>(x, n);
    count_launch();
  } else {
    int rc = apply_g(g, x, q, st);
    if (rc != BSCT_OK) return rc;
  }
  // r = b - G x0; p = r only keeps p finite for the first update p = z + 0 p
  k_init_r<T><<<nb, RED_THREADS, 0, st>>>(b, q, r, p, n, x0_is_zero ? 0 : 1);
  BSCT_CUDA_TRY(cudaMemsetAsync(g->scal, 0, 16 * sizeof(double), st));  // rho = beta = 0, counters
  k_dot<T><<<nb, RED_THREADS, 0, st>>>(r, r, n, g->partials);
  k_finish<<<1, RED_THREADS, 0, st>>>(g->partials, nb, g->scal, OP_STORE_RRP);
  k_dot<T><<<nb, RED_THREADS, 0, st>>>(b, b, n, g->partials);
  k_finish<<<1, RED_THREADS, 0, st>>>(g->partials, nb, g->scal, OP_STORE_BB);
  count_launch(5);
  // z = M^-1 r, rho = <r, z>; beta stays 0 because the stored rho is 0
  return o.apply_pc(r, (T*)g->z, g->scal, g->partials, (cpx<T>*)g->S, precond_spectrum<T>(g),
                    (const cpx<T>*)g->tw, st);
}

template <typename T>
static int pcg_iter_t(bsct_gram* g, T* x, int n_iter, cudaStream_t st) {
  const long n = (long)g->N * g->N;
  const int nb = nblk(g, n);
  T* r = (T*)g->r;
  T* p = (T*)g->p;
  T* q = (T*)g->q;
  T* z = (T*)g->z;
  FftOps<T> o;
  if (!fft_ops_for<T>(g->N, &o)) return BSCT_ERR_UNSUPPORTED_SIZE;
  const T* Gt = (g->precision == BSCT_F32) ? (const T*)(const void*)g->Gt32 : (const T*)(const void*)g->Gt64;
  const T* Mt = precond_spectrum<T>(g);
  for (int it = 0; it < n_iter; ++it) {
    int rc = o.apply_cg(z, p, q, g->scal, g->partials, (cpx<T>*)g->S, Gt, (const cpx<T>*)g->tw, st);
    if (rc != BSCT_OK) return rc;
    k_xr_update<T, UPD_PCG><<<nb, RED_THREADS, 0, st>>>(x, r, p, q, g->scal, n, g->partials);
    count_launch(1);
    rc = o.apply_pc(r, z, g->scal, g->partials, (cpx<T>*)g->S, Mt, (const cpx<T>*)g->tw, st);
    if (rc != BSCT_OK) return rc;
  }
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

static int read_scalars(const bsct_gram* g, double* h, cudaStream_t st) {
  BSCT_CUDA_TRY(cudaMemcpyAsync(h, g->scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  BSCT_CUDA_TRY(cudaStreamSynchronize(st));
  return BSCT_OK;
}

extern "C" int bsct_precond_apply(bsct_gram* g, double eps, const void* d_x, void* d_y, void* stream) {
  if (!g || !d_x || !d_y) { bsct_set_last_message("NULL argument"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = precond_ready(g, eps, st);
  if (rc != BSCT_OK) return rc;
  if (g->precision == BSCT_F32) return precond_apply_t<float>(g, (const float*)d_x, (float*)d_y, st);
  return precond_apply_t<double>(g, (const double*)d_x, (double*)d_y, st);
}

extern "C" int bsct_pcg_solve(bsct_gram* g, double eps, const void* d_b, void* d_x, int x0_is_zero, int max_iter,
                              double rel_tol, int check_every, bsct_cg_report* report, void* stream) {
  if (!g || !d_b || !d_x || max_iter < 0) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  if (check_every < 1) check_every = 1;
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = g->precision == BSCT_F32;
  int rc = precond_ready(g, eps, st);
  if (rc != BSCT_OK) return rc;
  rc = f32 ? pcg_begin_t<float>(g, (const float*)d_b, (float*)d_x, x0_is_zero, st)
           : pcg_begin_t<double>(g, (const double*)d_b, (double*)d_x, x0_is_zero, st);
  if (rc != BSCT_OK) return rc;
  double h[16];
  int it = 0, converged = 0;
  if ((rc = read_scalars(g, h, st)) != BSCT_OK) return rc;
  if ((rc = check_start(h[SC_RRP], h[SC_BB])) != BSCT_OK) return rc;
  if (rel_tol > 0.0 && (h[SC_BB] == 0.0 || sqrt(h[SC_RRP] / h[SC_BB]) <= rel_tol)) converged = 1;
  while (!converged && it < max_iter) {
    const int k = (rel_tol > 0.0) ? (check_every < max_iter - it ? check_every : max_iter - it) : max_iter - it;
    rc = f32 ? pcg_iter_t<float>(g, (float*)d_x, k, st) : pcg_iter_t<double>(g, (double*)d_x, k, st);
    if (rc != BSCT_OK) return rc;
    it += k;
    if (rel_tol > 0.0) {
      if ((rc = read_scalars(g, h, st)) != BSCT_OK) return rc;
      if (!isfinite(h[SC_RRP]) || !isfinite(h[SC_RR])) {
        bsct_set_last_message("PCG residual is not finite");
        return BSCT_ERR_NONFINITE;
      }
      if (sqrt(h[SC_RRP] / h[SC_BB]) <= rel_tol) converged = 1;
    }
  }
  if ((rc = read_scalars(g, h, st)) != BSCT_OK) return rc;
  const double rr = h[SC_RRP], bb = h[SC_BB];
  if (!isfinite(rr)) { bsct_set_last_message("PCG residual is not finite"); return BSCT_ERR_NONFINITE; }
  double tr = -1.0;
  if (rel_tol > 0.0) {
    rc = f32 ? true_residual_t<float>(g, (const float*)d_b, (const float*)d_x, &tr, st)
             : true_residual_t<double>(g, (const double*)d_b, (const double*)d_x, &tr, st);
    if (rc != BSCT_OK) return rc;
  }
  if (report) {
    report->iterations = it;
    report->converged = converged;
    report->rel_residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    report->true_rel_residual = tr;
  }
  return (rel_tol > 0.0 && !converged) ? BSCT_WARN_NOT_CONVERGED : BSCT_OK;
}

// ------------------------------------------------------------------------------------
// Whole solve in one CUDA graph.  The iterations run as the body of a conditional WHILE
// node; a one-thread kernel after every iteration counts it and decides on the device
// whether another follows (residual above the tolerance, fewer than max_iter so far), so
// a solve is one graph launch and one host synchronisation, not a host round trip per
// convergence check.  The executable graph is kept in the handle and rebuilt when the
// method, x, max_iter or the tolerance change.
// ------------------------------------------------------------------------------------
namespace bsct {
constexpr int SC_IT = 7;  // iterations run by the graph (unsigned 64-bit)

// after == 0: the decision before the first iteration; after == 1: after an iteration
__global__ void k_loop_ctl(double* sc, cudaGraphConditionalHandle h, int max_iter, double tol2, int rr_slot,
                           int after) {
  unsigned long long* it = reinterpret_cast<unsigned long long*>(sc + SC_IT);
  const unsigned long long n = after ? *it + 1ull : 0ull;
  *it = n;
  const double rr = __ldcg(sc + rr_slot), bb = __ldcg(sc + SC_BB);
  const bool more = (long long)n < (long long)max_iter && bb > 0.0 && isfinite(rr) && (tol2 <= 0.0 || rr > tol2 * bb);
  cudaGraphSetConditional(h, more ? 1u : 0u);
}
}  // namespace bsct

struct bsct_graph_solver {
  int method = -1, max_iter = -1;
  const void* x = nullptr;
  double tol2 = -1.0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;  // capture stream
};

void bsct_graph_solver_free(bsct_graph_solver* s) {
  if (!s) return;
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->cs) cudaStreamDestroy(s->cs);
  delete s;
}

template <typename T>
static int build_solve_graph(bsct_gram* g, int method, T* x, int max_iter, double tol2, bsct_graph_solver* sg) {
  if (sg->exec) { cudaGraphExecDestroy(sg->exec); sg->exec = nullptr; }
  if (!sg->cs) BSCT_CUDA_TRY(cudaStreamCreateWithFlags(&sg->cs, cudaStreamNonBlocking));
  cudaGraph_t parent = nullptr;
  BSCT_CUDA_TRY(cudaGraphCreate(&parent, 0));
  auto fail = [&](cudaError_t e) {
    bsct_set_last_cuda_error(e);
    cudaGraphDestroy(parent);
    return BSCT_ERR_CUDA;
  };
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, parent, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e);
  int rr_slot = method == 1 ? SC_RRP : SC_RR, zero = 0;
  double* scal = g->scal;
  void* init_args[] = {&scal, &h, &max_iter, &tol2, &rr_slot, &zero};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)k_loop_ctl;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = init_args;
  cudaGraphNode_t n_init = nullptr, n_loop = nullptr;
  if ((e = cudaGraphAddKernelNode(&n_init, parent, nullptr, 0, &kp)) != cudaSuccess) return fail(e);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&n_loop, parent, &n_init, nullptr, 1, &cp)) != cudaSuccess) return fail(e);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(sg->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return fail(e);
  int rc = method == 1 ? pcg_iter_t<T>(g, x, 1, sg->cs) : cg_iter_t<T, UPD_CG>(g, x, 1, sg->cs);
  k_loop_ctl<<<1, 1, 0, sg->cs>>>(g->scal, h, max_iter, tol2, rr_slot, 1);
  count_launch();
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(sg->cs, &captured);
  if (rc != BSCT_OK) { cudaGraphDestroy(parent); return rc; }
  if (e != cudaSuccess) return fail(e);
  if ((e = cudaGraphInstantiate(&sg->exec, parent, 0)) != cudaSuccess) return fail(e);
  cudaGraphDestroy(parent);
  sg->method = method;
  sg->x = x;
  sg->max_iter = max_iter;
  sg->tol2 = tol2;
  return BSCT_OK;
}

template <typename T>
static int solve_graph_t(bsct_gram* g, int method, double eps, const T* b, T* x, int max_iter, double rel_tol,
                         bsct_cg_report* report, cudaStream_t st) {
  int rc = BSCT_OK;
  if (method == 1) {
    rc = precond_ready(g, eps, st);
    if (rc == BSCT_OK) rc = pcg_begin_t<T>(g, b, x, 1, st);
  } else {
    rc = cg_begin_t<T>(g, b, x, 1, st);
  }
  if (rc != BSCT_OK) return rc;
  const double tol2 = rel_tol > 0.0 ? rel_tol * rel_tol : 0.0;
  if (!g->sgraph) g->sgraph = new bsct_graph_solver();
  bsct_graph_solver* sg = g->sgraph;
  if (!sg->exec || sg->method != method || sg->x != x || sg->max_iter != max_iter || sg->tol2 != tol2) {
    rc = build_solve_graph<T>(g, method, x, max_iter, tol2, sg);
    if (rc != BSCT_OK && g_overlap) {
      // a graph that cannot hold the programmatic launch edges is built without them (the
      // switch is process-wide while the graph is captured: do not build solve graphs
      // from several host threads at once)
      cudaGetLastError();
      g_overlap = false;
      rc = build_solve_graph<T>(g, method, x, max_iter, tol2, sg);
      g_overlap = true;
    }
    if (rc != BSCT_OK) return rc;
  }
  BSCT_CUDA_TRY(cudaGraphLaunch(sg->exec, st));
  double h[16];
  if ((rc = read_scalars(g, h, st)) != BSCT_OK) return rc;
  const double rr = h[method == 1 ? SC_RRP : SC_RR], bb = h[SC_BB];
  unsigned long long its = 0;
  memcpy(&its, &h[SC_IT], sizeof(its));
  if ((rc = check_start(0.0, bb)) != BSCT_OK) return rc;
  if (!isfinite(rr)) { bsct_set_last_message("residual is not finite"); return BSCT_ERR_NONFINITE; }
  const int converged = rel_tol > 0.0 && (bb == 0.0 || rr <= tol2 * bb);
  double tr = -1.0;
  if (rel_tol > 0.0) {
    rc = true_residual_t<T>(g, b, x, &tr, st);
    if (rc != BSCT_OK) return rc;
  }
  if (report) {
    report->iterations = (int)its;
    report->converged = converged;
    report->rel_residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    report->true_rel_residual = tr;
  }
  return (rel_tol > 0.0 && !converged) ? BSCT_WARN_NOT_CONVERGED : BSCT_OK;
}

extern "C" int bsct_solve_graph(bsct_gram* g, int method, double eps, const void* d_b, void* d_x, int max_iter,
                                double rel_tol, bsct_cg_report* report, void* stream) {
  if (!g || !d_b || !d_x || max_iter < 0 || (method != 0 && method != 1)) {
    bsct_set_last_message("invalid argument");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (g->precision == BSCT_F32)
    return solve_graph_t<float>(g, method, eps, (const float*)d_b, (float*)d_x, max_iter, rel_tol, report, st);
  return solve_graph_t<double>(g, method, eps, (const double*)d_b, (double*)d_x, max_iter, rel_tol, report, st);
}
