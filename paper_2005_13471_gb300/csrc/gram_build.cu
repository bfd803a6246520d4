// Gram filter build (Sec. 4) and the FFT-based Gram apply entry points.
//
//   k_view_keys, k_view_rank : views reduced to half turns in [0, 1) (theta and theta + pi
//                  give the same Gram kernel), cos/sin by cospi/sinpi (exact zeros on the
//                  axes), sorted by angle with a rank count (64-bit integer keys) so every
//                  tap can find its views by binary search.
//   k_gram_tables: per view, the Gram kernel A(t) = M_[c, c, s, s, zeta, zeta](t) as an
//                  exact piecewise polynomial between its kinks (FP64).
//   k_gram_taps  : one thread per tap d of the upper half plane:
//                    G[d] = sum_theta A_theta(d . u_theta)
//                  Only views with |d . u| < |c| + |s| + zeta contribute; for |d| larger
//                  than the widest support those views form one arc of angles around the
//                  normal of d, found by binary search.  FP64, mirrored to G[-d].
//   k_embed      : taps -> 2N x 2N circulant kernel (tap d at d mod 2N).
//   spectrum     : 2-D FFT of the circulant kernel in FP64 (same FFT kernels as the
//                  apply), real part kept.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "bsct_boxspline.cuh"
#include "bsct_fft.cuh"
#include "bsct_internal.h"

namespace bsct {

std::atomic<unsigned long long> g_launches{0};
KernelTimer g_timer;
bool g_overlap = true;

// ------------------------------------------------------------------------------------
// FFT dispatch over the supported sizes
// ------------------------------------------------------------------------------------
#define BSCT_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(384) X(512) X(768) X(1024) X(2048)

template <typename T> bool fft_ops_for(int N, FftOps<T>* out) {
  switch (N) {
#define BSCT_CASE(N_) case N_: *out = fft_ops<T, N_>(); return true;
    BSCT_SIZES(BSCT_CASE)
#undef BSCT_CASE
    default: return false;
  }
}
template bool fft_ops_for<float>(int, FftOps<float>*);
template bool fft_ops_for<double>(int, FftOps<double>*);

// ------------------------------------------------------------------------------------
// twiddles
// ------------------------------------------------------------------------------------
template <typename T> __global__ void k_twiddles(cpx<T>* tw, int L) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)L, &s, &c);
  tw[k] = mk(T(c), T(s));
}
struct StageDesc {
  int ns;
  int R[8], NSV[8], off[8];
};

// entry (Ns - 1) + (r - 1) Ns + jm of a plan's stage table: exp(-2 pi i r jm / (Ns R))
template <typename T> __global__ void k_stage_table(cpx<T>* out, StageDesc d, int n) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  int s = d.ns - 1;
  while (s > 0 && idx < d.off[s]) --s;
  const int local = idx - d.off[s];
  const int r = local / d.NSV[s] + 1, jm = local % d.NSV[s];
  double sn, cs;
  sincospi(-2.0 * (double)r * (double)jm / ((double)d.NSV[s] * (double)d.R[s]), &sn, &cs);
  out[idx] = mk(T(cs), T(sn));
}

template <typename T> static int stage_table(cpx<T>* out, int L, bool rev, cudaStream_t st) {
  PlanInfo p;
  if (!plan_info(L, rev, &p)) return BSCT_ERR_UNSUPPORTED_SIZE;
  StageDesc d;
  d.ns = p.ns;
  int nsv = 1;
  for (int i = 0; i < p.ns; ++i) {
    d.R[i] = p.R[i];
    d.NSV[i] = nsv;
    d.off[i] = nsv - 1;
    nsv *= p.R[i];
  }
  k_stage_table<T><<<(L + 255) / 256, 256, 0, st>>>(out, d, L - 1);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

template <typename T> int build_fft_tables(cpx<T>* tw, int N, cudaStream_t st) {
  k_twiddles<T><<<(2 * N + 255) / 256, 256, 0, st>>>(tw, 2 * N);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  int rc = stage_table<T>(tw + 2 * N, N, false, st);
  if (rc == BSCT_OK) rc = stage_table<T>(tw + 3 * N, N, true, st);
  if (rc == BSCT_OK) rc = stage_table<T>(tw + 4 * N, 2 * N, false, st);
  if (rc == BSCT_OK) rc = stage_table<T>(tw + 6 * N, 2 * N, true, st);
  return rc;
}
template int build_fft_tables<float>(cpx<float>*, int, cudaStream_t);
template int build_fft_tables<double>(cpx<double>*, int, cudaStream_t);

// ------------------------------------------------------------------------------------
// geometry (views sorted by angle in half turns, [0, 1))
// ------------------------------------------------------------------------------------
// reduced angle of each view (half turns in [0, 1)) and its bit pattern, which orders
// non-negative doubles like the values themselves
__global__ void k_view_keys(const double* __restrict__ ang, int na, double* __restrict__ red,
                            unsigned long long* __restrict__ key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= na) return;
  double a = ang[i];
  a = a - floor(a);
  if (a >= 1.0 || !(a > 0.0)) a = 0.0;  // also maps -0 to +0
  red[i] = a;
  key[i] = (unsigned long long)__double_as_longlong(a);
}
// rank of view i = #{j : key_j < key_i or (key_j == key_i and j < i)}, by 64-bit integer
// compares against key tiles in shared memory; writes the views in angle order (FP32 angle
// for the taps' window search, FP64 cos / sin)
constexpr int GEO_T = 256;
__global__ void __launch_bounds__(GEO_T) k_view_rank(const double* __restrict__ red,
                                                     const unsigned long long* __restrict__ key, int na,
                                                     float* __restrict__ thf_sorted, double2* __restrict__ cs_sorted) {
  __shared__ unsigned long long tile[GEO_T];
  const int i = blockIdx.x * GEO_T + threadIdx.x;
  const unsigned long long ki = i < na ? key[i] : 0ull;
  int rank = 0;
  for (int t0 = 0; t0 < na; t0 += GEO_T) {
    __syncthreads();
    if (t0 + threadIdx.x < na) tile[threadIdx.x] = key[t0 + threadIdx.x];
    __syncthreads();
    const int n = na - t0 < GEO_T ? na - t0 : GEO_T;
    for (int k = 0; k < n; ++k) {
      const unsigned long long kj = tile[k];
      rank += (kj < ki) || (kj == ki && t0 + k < i);
    }
  }
  if (i >= na) return;
  const double a = red[i];
  double s, c;
  sincospi(a, &s, &c);
  thf_sorted[rank] = (float)a;
  cs_sorted[rank] = make_double2(c, s);
}

// the per-view Gram kernel A(t) = M_[c,c,s,s,zeta,zeta](t)
__device__ __forceinline__ double gram_kernel(double t, double a, double b, double zeta) {
  BoxDirs D;
  D.ng = 0;
  if (a > 0.0) { D.a[D.ng] = a; D.m[D.ng] = 2; ++D.ng; }
  if (b > 0.0) { D.a[D.ng] = b; D.m[D.ng] = 2; ++D.ng; }
  if (zeta > 0.0) { D.a[D.ng] = zeta; D.m[D.ng] = 2; ++D.ng; }
  for (int g = D.ng; g < 4; ++g) { D.a[g] = 0.0; D.m[g] = 0; }
  int small = -1;
  if (a > 0.0 && b > 0.0) {
    if (b < BSCT_SHORT_DIR * a) small = 1;
    else if (a < BSCT_SHORT_DIR * b) small = 0;
  }
  return box_eval(t, D, small);
}

__device__ __forceinline__ int lower_bound_f(const float* __restrict__ v, int n, float x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Per-view table of the Gram kernel A(t) = M_[c,c,s,s,zeta,zeta](t) on t >= 0 (A is
// even): its kinks -S + i|c| + j|s| + k zeta (i, j, k in 0..2, S = |c|+|s|+zeta) cut
// [0, S] into <= 13 pieces on which A is a polynomial of degree <= 5; each piece is
// stored as monomials in v = (t - mid) / halfwidth in [-1, 1], obtained by Chebyshev
// interpolation at 6 nodes of exact FP64 values (gram_kernel, with the short-direction
// split near the axes).  Taps then cost a 4-step search and a 6-term Horner per view.
// Table layout per view: S, piece count, KMAX piece starts (padded with 1e300), centres,
// inverse half widths, then NC monomial coefficients per piece.  One detector box (or none):
// <= 13 pieces of degree <= 5; two boxes (Sec. 2's series of boxes): <= 41 pieces of degree 7.
template <int KMAX_, int NC_> struct GTab {
  static constexpr int KMAX = KMAX_, NC = NC_;
  static constexpr int S = 0, NK = 1, KN = 2, MID = KN + KMAX, IHW = MID + KMAX, COEF = IHW + KMAX,
                       STRIDE = COEF + NC * KMAX;
};
typedef GTab<16, 6> GT1;
typedef GTab<64, 8> GT2;

// Pieces [kn[q], kn[q+1]] (q < nk - 1) of a per-view table: the kernel values at the NC
// Chebyshev nodes of every piece are spread over all threads of the CTA (the near-axis
// views' short-direction evaluations are the costly ones), then one thread per piece turns
// its values into monomial coefficients.  fv: shared scratch of KMAX * NC doubles.
template <typename L, typename F>
__device__ void fit_table_pieces(double* __restrict__ T, const double* kn, int nk, double* fv, F kernel) {
  __shared__ double ck[L::NC * L::NC];
  cheb_cos_fill<L::NC>(ck);
  __syncthreads();
  const int items = (nk - 1) * L::NC;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int q = it / L::NC, i = it - q * L::NC;
    const double mid = 0.5 * (kn[q] + kn[q + 1]), hw = 0.5 * (kn[q + 1] - kn[q]);
    fv[it] = kernel(mid + hw * ck[L::NC + i]);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < L::KMAX; q += blockDim.x) {
    double* c = T + L::COEF + L::NC * q;
    if (q >= nk - 1) {
      T[L::MID + q] = 0.0;
      T[L::IHW + q] = 0.0;
      for (int i = 0; i < L::NC; ++i) c[i] = 0.0;
      continue;
    }
    const double* v = fv + q * L::NC;
    if constexpr (L::NC == 8) {
      cheb8_monomials(v, c, ck);
    } else {
      static_assert(L::NC == 6, "6 or 8 coefficients");
      double ch[6];
      for (int k = 0; k < 6; ++k) {
        double acc = 0.0;
        for (int i = 0; i < 6; ++i) acc += v[i] * ck[6 * k + i];
        ch[k] = acc * (k == 0 ? 1.0 / 6.0 : 2.0 / 6.0);
      }
      // Chebyshev -> monomial: T0=1, T1=v, T2=2v^2-1, T3=4v^3-3v, T4=8v^4-8v^2+1, T5=16v^5-20v^3+5v
      c[0] = ch[0] - ch[2] + ch[4];
      c[1] = ch[1] - 3.0 * ch[3] + 5.0 * ch[5];
      c[2] = 2.0 * ch[2] - 8.0 * ch[4];
      c[3] = 4.0 * ch[3] - 20.0 * ch[5];
      c[4] = 8.0 * ch[4];
      c[5] = 16.0 * ch[5];
    }
    T[L::MID + q] = 0.5 * (kn[q] + kn[q + 1]);
    T[L::IHW + q] = 2.0 / (kn[q + 1] - kn[q]);
  }
}

__global__ void __launch_bounds__(64) k_gram_tables(const double2* __restrict__ cs, double zeta, double merge_tol,
                                                    double* __restrict__ tab) {
  typedef GT1 L;
  const int j = blockIdx.x;
  const double a = fabs(cs[j].x), b = fabs(cs[j].y);
  const double S = a + b + zeta;
  __shared__ double kn[32];
  __shared__ double fv[L::KMAX * L::NC];
  __shared__ int nk_s;
  double* T = tab + (long)j * L::STRIDE;
  if (threadIdx.x == 0) {
    int n = 0;
    kn[n++] = 0.0;
    for (int i = 0; i <= 2; ++i)
      for (int jj = 0; jj <= 2; ++jj)
        for (int k = 0; k <= (zeta > 0.0 ? 2 : 0); ++k) {
          const double x = -S + i * a + jj * b + k * zeta;
          if (x > 0.0 && x < S) kn[n++] = x;
        }
    kn[n++] = S;
    for (int i = 1; i < n; ++i) {  // sort
      const double t = kn[i];
      int q = i - 1;
      while (q >= 0 && kn[q] > t) { kn[q + 1] = kn[q]; --q; }
      kn[q + 1] = t;
    }
    int m = 1;  // merge kinks closer than merge_tol (keep S as the last one)
    for (int i = 1; i < n; ++i)
      if (kn[i] - kn[m - 1] > merge_tol) kn[m++] = kn[i];
      else if (i == n - 1) kn[m - 1] = kn[i];
    nk_s = m;
    T[L::S] = S;
    T[L::NK] = m;
    for (int i = 0; i < L::KMAX; ++i) T[L::KN + i] = i < m ? kn[i] : 1e300;
  }
  __syncthreads();
  fit_table_pieces<L>(T, kn, nk_s, fv, [&](double t) { return gram_kernel(t, a, b, zeta); });
}

template <typename L = GT1>
__device__ __forceinline__ double gram_table_eval(const double* __restrict__ T, double t) {
  int q = 0;
#pragma unroll
  for (int step = L::KMAX / 2; step > 0; step >>= 1)
    if (T[L::KN + q + step] <= t) q += step;
  const double v = (t - T[L::MID + q]) * T[L::IHW + q];
  const double* c = T + L::COEF + L::NC * q;
  double r = c[L::NC - 1];
#pragma unroll
  for (int k = L::NC - 2; k >= 0; --k) r = fma(r, v, c[k]);
  return r;
}

// Two detector boxes: the per-view Gram kernel A = M_[c,c,s,s,w1,w1,w2,w2] is the
// autocorrelation h * h of the footprint h = M_[c,s,w1,w2] (FootPoly: exact cubic pieces);
// its kinks -S + i|c| + j|s| + k w1 + l w2 (i, j, k, l in 0..2) cut [0, S] into <= 41
// pieces of degree 7, fitted by Chebyshev interpolation at 8 nodes.
__global__ void __launch_bounds__(64) k_gram_tables2(const double2* __restrict__ cs, double w1, double w2,
                                                     double merge_tol, double* __restrict__ tab) {
  typedef GT2 L;
  const int j = blockIdx.x;
  const double a = fabs(cs[j].x), b = fabs(cs[j].y);
  const double S = a + b + w1 + w2;
  __shared__ double kn[96];
  __shared__ double fv[L::KMAX * L::NC];
  __shared__ int nk_s;
  double* T = tab + (long)j * L::STRIDE;
  if (threadIdx.x == 0) {
    int n = 0;
    kn[n++] = 0.0;
    for (int i = 0; i <= 2; ++i)
      for (int jj = 0; jj <= 2; ++jj)
        for (int k = 0; k <= 2; ++k)
          for (int l = 0; l <= 2; ++l) {
            const double x = -S + i * a + jj * b + k * w1 + l * w2;
            if (x > 0.0 && x < S && n < 94) kn[n++] = x;
          }
    kn[n++] = S;
    for (int i = 1; i < n; ++i) {  // sort
      const double t = kn[i];
      int q = i - 1;
      while (q >= 0 && kn[q] > t) { kn[q + 1] = kn[q]; --q; }
      kn[q + 1] = t;
    }
    int m = 1;  // merge kinks closer than merge_tol (keep S as the last one)
    for (int i = 1; i < n; ++i)
      if (kn[i] - kn[m - 1] > merge_tol) kn[m++] = kn[i];
      else if (i == n - 1) kn[m - 1] = kn[i];
    if (m > L::KMAX) m = L::KMAX;  // cannot happen: at most 41 distinct kinks in [0, S]
    nk_s = m;
    T[L::S] = S;
    T[L::NK] = m;
    for (int i = 0; i < L::KMAX; ++i) T[L::KN + i] = i < m ? kn[i] : 1e300;
  }
  __syncthreads();
  // A = h * h with h = M_[a, b, w1, w2] as exact cubic pieces (h is even)
  __shared__ FootPoly F;
  foot_build(F, a, b, w1, w2, 1e-13);
  fit_table_pieces<L>(T, kn, nk_s, fv, [&](double t) {
    return foot_conv(F, t, -F.hw, F.hw, F.kn, F.K + 1, [&](double v) { return foot_eval(F, v); });
  });
}

// Views that can reach tap d: those whose strip |d . u| < |c| + |s| + zeta contains d, bounded
// by the window |theta - (phi_d + pi/2)| <= asin(wmax / |d|).  The window only has to contain
// them (views outside the support are skipped by the caller), so it is computed in FP32 and
// widened by 1e-4 half turns - far more than the FP32 error, which is at most ~1e-5 here
// because asin's argument stays below 0.9999 - and found by binary search in the FP32 copy
// of the sorted angles (each within 6e-8 of its FP64 value), while the taps stay FP64.
// Writes up to two index ranges [lo, hi) of views; returns how many.
__device__ inline int tap_window(int d1, int d2, float r, int na, const float* __restrict__ th, float wmax,
                                 int rg[2][2]) {
  const float hw = (r > 1.0001f * wmax) ? asinf(wmax / r) * 0.318309886f + 1e-4f : 1.0f;
  if (hw >= 0.5f) {
    rg[0][0] = 0; rg[0][1] = na;
    return 1;
  }
  const float phi = atan2f((float)d2, (float)d1) * 0.318309886f;  // / pi, in [0, 1]
  float centre = phi + 0.5f;
  if (centre >= 1.0f) centre -= 1.0f;
  const float lo = centre - hw, hi = centre + hw;
  if (lo < 0.0f) {
    rg[0][0] = lower_bound_f(th, na, lo + 1.0f); rg[0][1] = na;
    rg[1][0] = 0; rg[1][1] = lower_bound_f(th, na, hi);
    return 2;
  }
  if (hi > 1.0f) {
    rg[0][0] = lower_bound_f(th, na, lo); rg[0][1] = na;
    rg[1][0] = 0; rg[1][1] = lower_bound_f(th, na, hi - 1.0f);
    return 2;
  }
  rg[0][0] = lower_bound_f(th, na, lo); rg[0][1] = lower_bound_f(th, na, hi);
  return 1;
}

// Taps closer to the origin than TAP_NEAR see up to all views (1800 at |d| < 2.4, ~40 at
// |d| = 64) and would hold a single thread for milliseconds, leaving the GPU idle around a few
// blocks; they are summed by k_gram_taps_near, one warp per tap, instead.
constexpr float TAP_NEAR = 64.0f;

// zeta: the sum of the detector box widths (bounds the strip of views that reach a tap)
template <typename L>
__global__ void k_gram_taps(int N, int na, const float* __restrict__ th, const double2* __restrict__ cs,
                            const double* __restrict__ tab, double zeta, double* __restrict__ G) {
  const long H = (long)(2 * N - 1) * (N - 1) + N;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  int d1, d2;
  if (h < N) { d2 = 0; d1 = (int)h; }
  else {
    const long q = h - N;
    d2 = 1 + (int)(q / (2 * N - 1));
    d1 = (int)(q % (2 * N - 1)) - (N - 1);
  }
  const float wmax = 1.41421356f + (float)zeta;  // >= |c| + |s| + zeta for every view
  const float r = hypotf((float)d1, (float)d2);
  if (r < TAP_NEAR) return;  // k_gram_taps_near
  double acc = 0.0;
  // two views per step as independent FP64 chains (the kernel waits on FP64 results,
  // not on issue); a view outside its support is evaluated at the support edge and
  // masked, and the sum keeps the view order
  auto visit = [&](int j0, int j1) {
    int j = j0;
    for (; j + 1 < j1; j += 2) {
      const double2 u0 = cs[j], u1 = cs[j + 1];
      const double t0 = fabs(d1 * u0.x + d2 * u0.y), t1 = fabs(d1 * u1.x + d2 * u1.y);
      const double* T0 = tab + (long)j * L::STRIDE;
      const double* T1 = T0 + L::STRIDE;
      const double s0 = T0[L::S], s1 = T1[L::S];
      const double e0 = gram_table_eval<L>(T0, fmin(t0, s0)), e1 = gram_table_eval<L>(T1, fmin(t1, s1));
      if (t0 < s0) acc += e0;
      if (t1 < s1) acc += e1;
    }
    if (j < j1) {
      const double2 u = cs[j];
      const double t = fabs(d1 * u.x + d2 * u.y);
      const double* T = tab + (long)j * L::STRIDE;
      if (t < T[L::S]) acc += gram_table_eval<L>(T, t);
    }
  };
  int rg[2][2];
  const int nr = tap_window(d1, d2, r, na, th, wmax, rg);
  for (int k = 0; k < nr; ++k) visit(rg[k][0], rg[k][1]);
  const int W = 2 * N - 1;
  G[(long)(d2 + N - 1) * W + (d1 + N - 1)] = acc;
  G[(long)(-d2 + N - 1) * W + (-d1 + N - 1)] = acc;
}

// The taps with |d| < TAP_NEAR (upper half plane, as k_gram_taps): one warp per candidate
// d of the square [-R0, R0) x [0, R0) (R0 = min(TAP_NEAR, N)); the lanes take the window's
// views in a strided order and the 32 partial sums are added by a fixed shuffle tree.
template <typename L>
__global__ void __launch_bounds__(128) k_gram_taps_near(int N, int R0, int na, const float* __restrict__ th,
                                                        const double2* __restrict__ cs, const double* __restrict__ tab,
                                                        double zeta, double* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const long w = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= (long)(2 * R0 - 1) * R0) return;
  const int d2 = (int)(w / (2 * R0 - 1)), d1 = (int)(w % (2 * R0 - 1)) - (R0 - 1);
  if (d2 == 0 && d1 < 0) return;  // lower half of the centre row: the mirror of d1 > 0
  const float r = hypotf((float)d1, (float)d2);
  if (!(r < TAP_NEAR)) return;   // the far kernel's taps
  const float wmax = 1.41421356f + (float)zeta;
  int rg[2][2];
  const int nr = tap_window(d1, d2, r, na, th, wmax, rg);
  double acc = 0.0;
  for (int k = 0; k < nr; ++k)
    for (int j = rg[k][0] + lane; j < rg[k][1]; j += 32) {
      const double2 u = cs[j];
      const double t = fabs(d1 * u.x + d2 * u.y);
      const double* T = tab + (long)j * L::STRIDE;
      const double s = T[L::S];
      const double e = gram_table_eval<L>(T, fmin(t, s));
      if (t < s) acc += e;
    }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const int W = 2 * N - 1;
    G[(long)(d2 + N - 1) * W + (d1 + N - 1)] = acc;
    G[(long)(-d2 + N - 1) * W + (-d1 + N - 1)] = acc;
  }
}

__global__ void k_embed(const double* __restrict__ G, int N, double* __restrict__ E) {
  const int L = 2 * N;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)L * L) return;
  const int a = (int)(i / L), b = (int)(i % L);
  double v = 0.0;
  if (a != N && b != N) {
    const int d2 = a < N ? a : a - L;
    const int d1 = b < N ? b : b - L;
    v = G[(long)(d2 + N - 1) * (2 * N - 1) + (d1 + N - 1)];
  }
  E[i] = v;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// [N+1][2N] scaled packed spectrum -> [2N][N+1] plain spectrum
__global__ void k_unpack_spectrum(const double* __restrict__ Gt, int N, double* __restrict__ out) {
  const int L = 2 * N;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)L * (N + 1)) return;
  const int u = (int)(i / (N + 1)), v = (int)(i % (N + 1));
  const double sc = (double)L * (double)L;
  double g;
  if (v == 0) g = Gt[u] + Gt[(long)N * L + u];
  else if (v == N) g = Gt[u] - Gt[(long)N * L + u];
  else g = Gt[(long)v * L + u];
  out[i] = g * sc;
}

}  // namespace bsct

using namespace bsct;

// ------------------------------------------------------------------------------------
// error reporting
// ------------------------------------------------------------------------------------
static thread_local char g_msg[512] = "no error";
void bsct_set_last_cuda_error(cudaError_t e) {
  snprintf(g_msg, sizeof(g_msg), "CUDA error %d: %s", (int)e, cudaGetErrorString(e));
}
void bsct_set_last_message(const char* msg) { snprintf(g_msg, sizeof(g_msg), "%s", msg); }

extern "C" const char* bsct_last_error_string(void) { return g_msg; }

extern "C" const char* bsct_status_string(int s) {
  switch (s) {
    case BSCT_OK: return "ok";
    case BSCT_ERR_INVALID_ARG: return "invalid argument";
    case BSCT_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case BSCT_ERR_CUDA: return "CUDA error";
    case BSCT_ERR_TIMEOUT: return "device wait timed out";
    case BSCT_ERR_NONFINITE: return "non-finite value";
    case BSCT_WARN_NOT_CONVERGED: return "not converged";
    default: return "unknown status";
  }
}

extern "C" uint64_t bsct_launch_count(void) { return (uint64_t)g_launches.load(); }

extern "C" int bsct_supported_size(int32_t N) {
  FftOps<float> o;
  return fft_ops_for<float>(N, &o) ? 1 : 0;
}

static int fail(int code, const char* msg) {
  bsct_set_last_message(msg);
  return code;
}
static int fail_msg(int code, const char* msg) { return fail(code, msg); }

extern "C" int bsct_set_kernel_timing(int on) {
  g_timer.on = on != 0;
  g_timer.n_recorded = 0;
  return BSCT_OK;
}

extern "C" int bsct_set_launch_overlap(int on) {
  g_overlap = on != 0;
  return BSCT_OK;
}

extern "C" int bsct_kernel_times(float* ms, int n) {
  if (!ms || n < 1) return fail_msg(BSCT_ERR_INVALID_ARG, "invalid argument");
  if (!g_timer.created || g_timer.n_recorded < 2) return fail_msg(BSCT_ERR_INVALID_ARG, "no timed launch recorded");
  const int k = g_timer.n_recorded - 1 < n ? g_timer.n_recorded - 1 : n;
  for (int i = 0; i < k; ++i) {
    BSCT_CUDA_TRY(cudaEventSynchronize(g_timer.ev[i + 1]));
    BSCT_CUDA_TRY(cudaEventElapsedTime(&ms[i], g_timer.ev[i], g_timer.ev[i + 1]));
  }
  return k;
}

int bsct_check_geom(const bsct_geom* g) {
  if (!g) return fail(BSCT_ERR_INVALID_ARG, "geom is NULL");
  if (!g->angles_pi) return fail(BSCT_ERR_INVALID_ARG, "angles_pi is NULL");
  if (g->n_angles < 1) return fail(BSCT_ERR_INVALID_ARG, "n_angles < 1");
  if (g->n_bins < 1) return fail(BSCT_ERR_INVALID_ARG, "n_bins < 1");
  if (!(g->lambda_y > 0.0) || !isfinite(g->lambda_y)) return fail(BSCT_ERR_INVALID_ARG, "lambda_y must be > 0");
  if (!(g->zeta_blur >= 0.0) || !isfinite(g->zeta_blur)) return fail(BSCT_ERR_INVALID_ARG, "zeta_blur must be >= 0");
  if (g->zeta_blur > 0.0 && g->zeta_blur < BSCT_SHORT_DIR)
    return fail(BSCT_ERR_INVALID_ARG, "0 < zeta_blur < 0.2 is not supported (short blur direction)");
  for (int i = 0; i < g->n_angles; ++i)
    if (!isfinite(g->angles_pi[i])) return fail(BSCT_ERR_INVALID_ARG, "angles_pi holds a non-finite value");
  if (g->n_blur < 0 || g->n_blur > 2) return fail(BSCT_ERR_INVALID_ARG, "n_blur must be 0, 1 or 2");
  if (g->n_blur > 0) {
    if (!g->blur_widths) return fail(BSCT_ERR_INVALID_ARG, "blur_widths is NULL");
    if (g->zeta_blur != 0.0) return fail(BSCT_ERR_INVALID_ARG, "zeta_blur must be 0 when blur_widths is given");
    for (int i = 0; i < g->n_blur; ++i)
      if (!isfinite(g->blur_widths[i]) || g->blur_widths[i] < BSCT_SHORT_DIR || g->blur_widths[i] > 4.0)
        return fail(BSCT_ERR_INVALID_ARG, "detector box widths must lie in [0.2, 4]");
  }
  return BSCT_OK;
}

int bsct_blur_boxes(const bsct_geom* g, double w[2]) {
  w[0] = w[1] = 0.0;
  if (g->n_blur > 0) {
    for (int i = 0; i < g->n_blur; ++i) w[i] = g->blur_widths[i];
    return g->n_blur;
  }
  if (g->zeta_blur > 0.0) {
    w[0] = g->zeta_blur;
    return 1;
  }
  return 0;
}

extern "C" void bsct_gram_free(bsct_gram* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  if (g->owns_filter) {
    cudaFree(g->taps);
    cudaFree(g->Gt64);
    cudaFree(g->Gt32);
    cudaFree(g->tw);
  }
  cudaFree(g->S);
  cudaFree(g->dg_work);
  cudaFree(g->z);
  bsct_host_pipe_free(g->pipe);
  bsct_graph_solver_free(g->sgraph);
  cudaFree(g->Mt64);
  cudaFree(g->Mt32);
  cudaFree(g->r);
  cudaFree(g->p);
  cudaFree(g->q);
  cudaFree(g->scal);
  cudaFree(g->partials);
  delete g;
}

#define TRY(expr)                                  \
  do {                                             \
    int _rc = (expr);                              \
    if (_rc != BSCT_OK) { cleanup(); return _rc; } \
  } while (0)
#define CTRY(expr)                                                             \
  do {                                                                         \
    cudaError_t _e = (expr);                                                   \
    if (_e != cudaSuccess) { bsct_set_last_cuda_error(_e); cleanup(); return BSCT_ERR_CUDA; } \
  } while (0)

extern "C" int bsct_gram_build(const bsct_geom* geom, int precision, bsct_gram** out, void* stream) {
  int rc = bsct_check_geom(geom);
  if (rc != BSCT_OK) return rc;
  if (!out) return fail(BSCT_ERR_INVALID_ARG, "out is NULL");
  if (precision != BSCT_F32 && precision != BSCT_F64) return fail(BSCT_ERR_INVALID_ARG, "precision");
  const int N = geom->N;
  FftOps<double> o64;
  FftOps<float> o32;
  if (!fft_ops_for<double>(N, &o64) || !fft_ops_for<float>(N, &o32))
    return fail(BSCT_ERR_UNSUPPORTED_SIZE, "unsupported N (see bsct_supported_size)");
  cudaStream_t st = (cudaStream_t)stream;
  const int na = geom->n_angles;
  const int L = 2 * N;
  const long ntap = (long)(2 * N - 1) * (2 * N - 1);

  bsct_gram* g = new bsct_gram();
  g->N = N;
  g->precision = precision;
  g->n_angles = na;
  {
    double w[2];
    bsct_blur_boxes(geom, w);
    g->zeta = w[0] + w[1];  // total detector width (informational)
  }
  g->lambda = geom->lambda_y;
  double *d_ang = nullptr, *d_emb = nullptr, *d_gtab = nullptr, *d_red = nullptr;
  float* d_thf = nullptr;
  unsigned long long* d_key = nullptr;
  double2* d_cs = nullptr;
  void* d_S2 = nullptr;
  cpx<double>* tw64 = nullptr;
  char* d_tmp = nullptr;  // every temporary of the build in one allocation
  auto cleanup = [&]() {
    cudaFree(d_tmp);
    cudaFree(tw64);
    if (g) { bsct_gram_free(g); g = nullptr; }
  };
  const size_t T = precision == BSCT_F32 ? sizeof(float) : sizeof(double);
  double wb[2];
  const int nbox = bsct_blur_boxes(geom, wb);
  {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_ang = al(na * sizeof(double)), b_red = al(na * sizeof(double)), b_thf = al(na * sizeof(float)),
                 b_key = al(na * sizeof(unsigned long long)), b_cs = al(na * sizeof(double2)),
                 b_gtab = al((size_t)na * (nbox == 2 ? GT2::STRIDE : GT1::STRIDE) * sizeof(double)),
                 b_emb = al((size_t)L * L * sizeof(double)), b_S2 = al((size_t)L * N * 2 * sizeof(double));
    CTRY(cudaMalloc(&d_tmp, b_ang + b_red + b_thf + b_key + b_cs + b_gtab + b_emb + b_S2));
    char* q = d_tmp;
    d_ang = (double*)q; q += b_ang;
    d_red = (double*)q; q += b_red;
    d_thf = (float*)q; q += b_thf;
    d_key = (unsigned long long*)q; q += b_key;
    d_cs = (double2*)q; q += b_cs;
    d_gtab = (double*)q; q += b_gtab;
    d_emb = (double*)q; q += b_emb;
    d_S2 = q;
  }
  CTRY(cudaMalloc(&g->taps, ntap * sizeof(double)));
  CTRY(cudaMalloc(&g->Gt64, (size_t)(N + 1) * L * sizeof(double)));
  CTRY(cudaMalloc(&tw64, (size_t)fft_table_elems(N) * sizeof(cpx<double>)));
  CTRY(cudaMemcpyAsync(d_ang, geom->angles_pi, na * sizeof(double), cudaMemcpyHostToDevice, st));

  k_view_keys<<<(na + 255) / 256, 256, 0, st>>>(d_ang, na, d_red, d_key);
  k_view_rank<<<(na + GEO_T - 1) / GEO_T, GEO_T, 0, st>>>(d_red, d_key, na, d_thf, d_cs);
  const long H = (long)(2 * N - 1) * (N - 1) + N;
  const int R0 = N < (int)TAP_NEAR ? N : (int)TAP_NEAR;  // near taps: |d1|, d2 < R0
  if (nbox == 2) {
    k_gram_tables2<<<na, 64, 0, st>>>(d_cs, wb[0], wb[1], 1e-13, d_gtab);
    k_gram_taps<GT2><<<(unsigned)((H + 127) / 128), 128, 0, st>>>(N, na, d_thf, d_cs, d_gtab, wb[0] + wb[1], g->taps);
    k_gram_taps_near<GT2><<<(unsigned)(((long)(2 * R0 - 1) * R0 + 3) / 4), 128, 0, st>>>(N, R0, na, d_thf, d_cs, d_gtab,
                                                                                      wb[0] + wb[1], g->taps);
  } else {
    k_gram_tables<<<na, 64, 0, st>>>(d_cs, wb[0], 1e-13, d_gtab);
    k_gram_taps<GT1><<<(unsigned)((H + 127) / 128), 128, 0, st>>>(N, na, d_thf, d_cs, d_gtab, wb[0], g->taps);
    k_gram_taps_near<GT1><<<(unsigned)(((long)(2 * R0 - 1) * R0 + 3) / 4), 128, 0, st>>>(N, R0, na, d_thf, d_cs, d_gtab,
                                                                                      wb[0], g->taps);
  }
  k_embed<<<(unsigned)(((long)L * L + 255) / 256), 256, 0, st>>>(g->taps, N, d_emb);
  count_launch(6);
  CTRY(cudaGetLastError());
  TRY(build_fft_tables<double>(tw64, N, st));
  TRY(o64.spectrum(d_emb, (cpx<double>*)d_S2, g->Gt64, tw64, st));

  // per-precision apply state
  CTRY(cudaMalloc(&g->S, (size_t)N * N * 2 * T));
  CTRY(cudaMalloc(&g->r, (size_t)N * N * T));
  CTRY(cudaMalloc(&g->p, (size_t)N * N * T));
  CTRY(cudaMalloc(&g->q, (size_t)N * N * T));
  g->n_partials = 1024;
  CTRY(cudaMalloc(&g->partials, (size_t)g->n_partials * sizeof(double) * 2));
  CTRY(cudaMalloc(&g->scal, 16 * sizeof(double)));
  CTRY(cudaMemsetAsync(g->scal, 0, 16 * sizeof(double), st));
  if (precision == BSCT_F32) {
    const long ng = (long)(N + 1) * L;
    CTRY(cudaMalloc(&g->Gt32, ng * sizeof(float)));
    k_to_f32<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(g->Gt64, g->Gt32, ng);
    count_launch();
    CTRY(cudaMalloc(&g->tw, (size_t)fft_table_elems(N) * sizeof(cpx<float>)));
    TRY(build_fft_tables<float>((cpx<float>*)g->tw, N, st));
  } else {
    g->tw = tw64;
    tw64 = nullptr;
  }
  CTRY(cudaGetLastError());
  CTRY(cudaStreamSynchronize(st));
  cudaFree(d_tmp);
  cudaFree(tw64);
  *out = g;
  return BSCT_OK;
}
#undef TRY
#undef CTRY

extern "C" int bsct_gram_taps(const bsct_gram* g, double* d_out, void* stream) {
  if (!g || !d_out) return fail(BSCT_ERR_INVALID_ARG, "NULL argument");
  const long ntap = (long)(2 * g->N - 1) * (2 * g->N - 1);
  BSCT_CUDA_TRY(cudaMemcpyAsync(d_out, g->taps, ntap * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return BSCT_OK;
}

extern "C" int bsct_gram_spectrum(const bsct_gram* g, double* d_out, void* stream) {
  if (!g || !d_out) return fail(BSCT_ERR_INVALID_ARG, "NULL argument");
  const long n = (long)2 * g->N * (g->N + 1);
  k_unpack_spectrum<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(g->Gt64, g->N, d_out);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

extern "C" int bsct_gram_apply(const bsct_gram* g, const void* d_x, void* d_y, int mode, void* stream) {
  if (!g || !d_x || !d_y) return fail(BSCT_ERR_INVALID_ARG, "NULL argument");
  if (d_x == d_y) return fail(BSCT_ERR_INVALID_ARG, "x and y may not alias");
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == BSCT_APPLY_FFT32) {
    if (g->precision != BSCT_F32) return fail(BSCT_ERR_INVALID_ARG, "FFT32 apply needs an F32 handle");
    FftOps<float> o;
    fft_ops_for<float>(g->N, &o);
    return o.apply((const float*)d_x, (float*)d_y, (cpx<float>*)g->S, g->Gt32, (const cpx<float>*)g->tw, st);
  }
  if (mode == BSCT_APPLY_F64) {
    if (g->precision != BSCT_F64) return fail(BSCT_ERR_INVALID_ARG, "F64 apply needs an F64 handle");
    FftOps<double> o;
    fft_ops_for<double>(g->N, &o);
    return o.apply((const double*)d_x, (double*)d_y, (cpx<double>*)g->S, g->Gt64, (const cpx<double>*)g->tw, st);
  }
  if (mode == BSCT_APPLY_DFTGEMM_BF16) {
    if (g->precision != BSCT_F32) return fail(BSCT_ERR_INVALID_ARG, "DFT-GEMM apply needs an F32 handle");
    int P, Q;
    if (!dftgemm_factor(2 * g->N, &P, &Q)) return fail(BSCT_ERR_UNSUPPORTED_SIZE, "no DFT-GEMM factorisation for 2N");
    bsct_gram* gm = const_cast<bsct_gram*>(g);
    if (!gm->dg_work) {
      const size_t bytes = dftgemm_scratch_bytes(g->N);
      BSCT_CUDA_TRY(cudaMalloc(&gm->dg_work, bytes));
      gm->dg_bytes = bytes;
    }
    const int rc = check_finite_async<float>((const float*)d_x, (long)g->N * g->N, st);
    if (rc != BSCT_OK) return rc;
    return dftgemm_apply(g->N, (const float*)d_x, (float*)d_y, g->Gt32, (const float2*)g->tw, gm->dg_work, st);
  }
  return fail(BSCT_ERR_INVALID_ARG, "unknown apply mode");
}
