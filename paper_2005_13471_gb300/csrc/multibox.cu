// Detector kernels made of two boxes: back projection and forward projection.
//
// Sec. 2 models the detector cell's response as a convolution of boxes and works with one;
// with two unit-mass boxes of widths w1, w2 the footprint of a pixel in view theta becomes
//     h_theta = M_[|c|, |s|, w1, w2]   (c, s = cos theta, sin theta),
// one box-spline direction more than the one-box case, and everything downstream gains a
// degree: the sinogram interpolant of Sec. 5 has degree d = (non-zero directions) - 1, i.e.
// 3 for oblique views and 2 for axis-aligned ones, with the correction filter of Eq. 5 for
// that degree (q[m] = sqrt(3) (sqrt(3) - 2)^|m| for d = 3, sqrt(2) (2 sqrt(2) - 3)^|m| for
// d = 2, |m| <= 40, zero outside the detector).
//
// Back projection, per view (same scheme as the one-box path, wider tables):
//   the weight of sample m0 + J0 + j for a pixel at detector coordinate p = m0 + f is
//   phi_j(f) = K((J0 + j - f) lambda), K = lambda M_[|c|, |s|, w1, w2, lambda x (d+1)]; each
//   phi_j is one polynomial of degree <= 7 between consecutive points of
//   {0} U {frac(-kink(K) / lambda)} (<= 17 pieces).  k_mb_bp_tables fits them in FP64 by
//   Chebyshev interpolation at 8 nodes of exact kernel values - K is evaluated as the
//   convolution of the trapezoid M_[|c|, |s|] (short-direction split near the axes) with
//   M_[w1, w2, lambda x (d+1)] (box_conv) - and k_mb_bp_gather sums, per pixel and view,
//   sum_j c~[m0 + J0 + j] poly_{q,j}(v).
// Forward projection, per view: h_theta is one cubic between consecutive kinks
//   -W/2 + k0 |c| + k1 |s| + k2 w1 + k3 w2 (<= 15 pieces, W = |c| + |s| + w1 + w2), fitted in
//   FP64 at 4 Chebyshev nodes; one thread per (view, sample) walks the image lines along the
//   view's major axis and sums h(y_m - x_k . u) c_k over the pixels of each line inside the
//   support.
// Detector coordinates are formed in FP64 in both precisions; FP32 evaluates the
// polynomials and accumulates in FP32, folded into FP64 sums per view block / image line.
#include <math.h>

#include "bsct_boxspline.cuh"
#include "bsct_internal.h"

namespace bsct {

constexpr int MB_QMAX = 20;   // pieces of f per view (<= 17 occur)
constexpr int MB_NJMAX = 48;  // samples touching one pixel
constexpr int MB_NC = 8;      // coefficients per (piece, offset): degree <= 7
// per-view FP64 header: p00, c/lambda, s/lambda, Q, J0, nJ, degree, pad; piece starts
// sigma[0..Q] (padded to 24 with 2.0); centres mid[QMAX]; inverse half widths ihw[QMAX]
constexpr int MB_P00 = 0, MB_CL = 1, MB_SL = 2, MB_Q = 3, MB_J0 = 4, MB_NJ = 5, MB_DEG = 6;
constexpr int MB_SIG = 8, MB_MID = MB_SIG + 24, MB_IHW = MB_MID + MB_QMAX, MB_DH = MB_IHW + MB_QMAX;
constexpr long MB_CSTRIDE = (long)MB_QMAX * MB_NJMAX * MB_NC;  // T coefficients per view
constexpr int MB_PF_T = 256, MB_PF_H = 40;
constexpr int MB_TX = 16, MB_TY = 16;

__host__ __device__ inline void mb_jrange(double W, double lam, int* J0, int* nJ) {
  const double h = 0.5 * W / lam;
  const int j0 = (int)floor(-h) + 1;
  const int j1 = (int)ceil(h + 1.0) - 1;
  *J0 = j0;
  *nJ = j1 - j0 + 1;
}

// P = {|c|, |s|} (non-zero ones, with the short-direction split), Q = {w1, w2, lambda x (d+1)}
__device__ inline void mb_bp_dirs(double A, double B, double w1, double w2, double lam, int d, BoxDirs* P,
                                  int* small, BoxDirs* Q) {
  P->ng = 0;
  if (A > 0.0) { P->a[P->ng] = A; P->m[P->ng] = 1; ++P->ng; }
  if (B > 0.0) { P->a[P->ng] = B; P->m[P->ng] = 1; ++P->ng; }
  for (int g = P->ng; g < 4; ++g) { P->a[g] = 0.0; P->m[g] = 0; }
  *small = -1;
  if (A > 0.0 && B > 0.0) {
    if (B < BSCT_SHORT_DIR * A) *small = 1;
    else if (A < BSCT_SHORT_DIR * B) *small = 0;
  }
  Q->ng = 0;
  if (w1 == w2) { Q->a[0] = w1; Q->m[0] = 2; Q->ng = 1; }
  else { Q->a[0] = w1; Q->m[0] = 1; Q->a[1] = w2; Q->m[1] = 1; Q->ng = 2; }
  Q->a[Q->ng] = lam; Q->m[Q->ng] = d + 1; ++Q->ng;
  for (int g = Q->ng; g < 4; ++g) { Q->a[g] = 0.0; Q->m[g] = 0; }
}

// one CTA (256 threads) per view
template <typename T>
__global__ void __launch_bounds__(256) k_mb_bp_tables(const double* __restrict__ ang, int N, int M, double lam,
                                                      double w1, double w2, double merge_tol,
                                                      double* __restrict__ hdr, T* __restrict__ coef,
                                                      int* __restrict__ status) {
  const int a = blockIdx.x;
  __shared__ double sig[MB_QMAX + 4];
  __shared__ int s_q;
  double s_, c_;
  sincospi(ang[a], &s_, &c_);
  const double A = fabs(c_), B = fabs(s_);
  const int d = (A > 0.0) + (B > 0.0) + 1;  // directions |c|, |s|, w1, w2 (non-zero) - 1
  BoxDirs P, Q;
  int small;
  mb_bp_dirs(A, B, w1, w2, lam, d, &P, &small, &Q);
  const double W = A + B + w1 + w2 + (d + 1) * lam;
  int J0, nJ;
  mb_jrange(W, lam, &J0, &nJ);
  double* h = hdr + (long)a * MB_DH;
  if (threadIdx.x == 0) {
    // kinks of K: -W/2 + k0 A + k1 B + k2 w1 + k3 w2 (+ multiples of lambda); in f they sit
    // at frac(-kink / lambda)
    double fk[17];
    int n = 0;
    fk[n++] = 0.0;
    for (int k0 = 0; k0 <= (A > 0.0); ++k0)
      for (int k1 = 0; k1 <= (B > 0.0); ++k1)
        for (int k2 = 0; k2 <= 1; ++k2)
          for (int k3 = 0; k3 <= 1; ++k3) {
            const double kink = -0.5 * W + k0 * A + k1 * B + k2 * w1 + k3 * w2;
            double f = -kink / lam;
            f -= floor(f);
            if (f >= 1.0) f = 0.0;
            fk[n++] = f;
          }
    for (int i = 1; i < n; ++i) {  // insertion sort
      const double t = fk[i];
      int j = i - 1;
      while (j >= 0 && fk[j] > t) { fk[j + 1] = fk[j]; --j; }
      fk[j + 1] = t;
    }
    int q = 1;  // merge kinks closer than merge_tol, drop those within merge_tol of 1
    for (int i = 1; i < n; ++i)
      if (fk[i] - fk[q - 1] > merge_tol && 1.0 - fk[i] > merge_tol) fk[q++] = fk[i];
    for (int i = 0; i < q; ++i) sig[i] = fk[i];
    sig[q] = 1.0;
    s_q = q;
    const double x0 = -0.5 * (N - 1);
    h[MB_P00] = (x0 * c_ + x0 * s_) / lam + 0.5 * (M - 1);
    h[MB_CL] = c_ / lam;
    h[MB_SL] = s_ / lam;
    h[MB_Q] = q;
    h[MB_J0] = J0;
    h[MB_NJ] = nJ;
    h[MB_DEG] = d;
    h[7] = 0.0;
    for (int i = 0; i < 24; ++i) h[MB_SIG + i] = i <= q ? sig[i] : 2.0;
    if (nJ > MB_NJMAX) atomicExch(status, 1);
  }
  __syncthreads();
  const int Qn = s_q;
  for (int i = threadIdx.x; i < MB_QMAX; i += blockDim.x) {
    h[MB_MID + i] = i < Qn ? 0.5 * (sig[i] + sig[i + 1]) : 0.0;
    h[MB_IHW + i] = i < Qn ? 2.0 / (sig[i + 1] - sig[i]) : 0.0;
  }
  T* cv = coef + (long)a * MB_CSTRIDE;
  for (int w = threadIdx.x; w < MB_QMAX * MB_NJMAX; w += blockDim.x) {
    const int q = w / MB_NJMAX, j = w % MB_NJMAX;
    T* c = cv + (long)w * MB_NC;
    if (q >= Qn || j >= nJ || nJ > MB_NJMAX) {
      for (int i = 0; i < MB_NC; ++i) c[i] = T(0);
      continue;
    }
    const double mid = 0.5 * (sig[q] + sig[q + 1]), hw = 0.5 * (sig[q + 1] - sig[q]);
    double fv[8], mono[8];
    for (int i = 0; i < 8; ++i) {
      const double f = mid + hw * cospi((2.0 * i + 1.0) / 16.0);
      const double u = (J0 + j - f) * lam;
      fv[i] = fabs(u) < 0.5 * W ? lam * box_conv(u, P, small, Q) : 0.0;
    }
    cheb8_monomials(fv, mono);
    for (int i = 0; i < MB_NC; ++i) c[i] = T(mono[i]);
  }
}

// c~ = g_s * q (Eq. 5) for the view's degree (2 or 3); one CTA per 256 outputs of one view
template <typename T>
__global__ void __launch_bounds__(MB_PF_T) k_mb_prefilter(const double* __restrict__ hdr, const T* __restrict__ g,
                                                          int M, T* __restrict__ ct) {
  __shared__ T qs[MB_PF_H + 1];
  __shared__ T seg[MB_PF_T + 2 * MB_PF_H];
  const int a = blockIdx.y, m0 = blockIdx.x * MB_PF_T;
  const T* gr = g + (long)a * M;
  const int d = (int)hdr[(long)a * MB_DH + MB_DEG];
  if (threadIdx.x <= MB_PF_H) {
    const double r = d == 3 ? 1.7320508075688772 : 1.4142135623730951;   // sqrt(3) / sqrt(2)
    const double z1 = d == 3 ? 1.7320508075688772 - 2.0 : 2.0 * 1.4142135623730951 - 3.0;
    qs[threadIdx.x] = T(r * pow(z1, (double)threadIdx.x));
  }
  for (int i = threadIdx.x; i < MB_PF_T + 2 * MB_PF_H; i += MB_PF_T) {
    const int mm = m0 - MB_PF_H + i;
    seg[i] = (mm >= 0 && mm < M) ? gr[mm] : T(0);
  }
  __syncthreads();
  const int m = m0 + threadIdx.x;
  if (m >= M) return;
  const T* c = seg + MB_PF_H + threadIdx.x;
  T acc = T(0);
  for (int j = MB_PF_H; j >= 1; --j) acc = fma(qs[j], c[-j] + c[j], acc);
  ct[(long)a * M + m] = fma(qs[0], c[0], acc);
}

template <typename T> struct MbVec;
template <> struct MbVec<float> {
  static __device__ __forceinline__ void load8(const float* p, float c[8]) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p)), y = __ldg(reinterpret_cast<const float4*>(p + 4));
    c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w; c[4] = y.x; c[5] = y.y; c[6] = y.z; c[7] = y.w;
  }
};
template <> struct MbVec<double> {
  static __device__ __forceinline__ void load8(const double* p, double c[8]) {
    for (int i = 0; i < 4; ++i) {
      const double2 x = __ldg(reinterpret_cast<const double2*>(p) + i);
      c[2 * i] = x.x;
      c[2 * i + 1] = x.y;
    }
  }
};

// one thread per pixel, every view
template <typename T>
__global__ void __launch_bounds__(MB_TX* MB_TY) k_mb_bp_gather(const double* __restrict__ hdr,
                                                               const T* __restrict__ coef, const T* __restrict__ ct,
                                                               int na, int N, int M, T* __restrict__ b) {
  const int k1 = blockIdx.x * MB_TX + threadIdx.x, k2 = blockIdx.y * MB_TY + threadIdx.y;
  if (k1 >= N || k2 >= N) return;
  double total = 0.0;
  T part = T(0);
  for (int a = 0; a < na; ++a) {
    const double* h = hdr + (long)a * MB_DH;
    const double p = h[MB_P00] + (double)k1 * h[MB_CL] + (double)k2 * h[MB_SL];
    const double mf = floor(p);
    const double f = p - mf;
    const int Q = (int)h[MB_Q], J0 = (int)h[MB_J0], nJ = (int)h[MB_NJ];
    int q = 0;
    while (q + 1 < Q && h[MB_SIG + q + 1] <= f) ++q;
    const T v = T((f - h[MB_MID + q]) * h[MB_IHW + q]);
    const T* cq = coef + (long)a * MB_CSTRIDE + (long)q * MB_NJMAX * MB_NC;
    const T* cr = ct + (long)a * M;
    const int mb = (int)mf + J0;
    for (int j = 0; j < nJ; ++j) {
      const int m = mb + j;
      if ((unsigned)m >= (unsigned)M) continue;
      T c[8];
      MbVec<T>::load8(cq + j * MB_NC, c);
      T w = c[7];
#pragma unroll
      for (int i = 6; i >= 0; --i) w = fma(w, v, c[i]);
      part = fma(w, cr[m], part);
    }
    if ((a & 31) == 31) { total += (double)part; part = T(0); }
  }
  total += (double)part;
  b[(long)k2 * N + k1] = T(total);
}

// ---------------------------------------------------------------------------------------
// Forward projection
// ---------------------------------------------------------------------------------------
constexpr int MBF_KMAX = 16;  // pieces of h (<= 15 occur)
// per-view FP64 header: c, s, rows (1: lines are image rows), W/2, pieces; kinks kn[0..K]
// (padded to 20 with 1e300); centres mid[KMAX]; inverse half widths ihw[KMAX]; then
// 4 monomial coefficients per piece (FP64 here; T copies in the coefficient table)
constexpr int MBF_C = 0, MBF_S = 1, MBF_ROWS = 2, MBF_HW = 3, MBF_K = 4;
constexpr int MBF_KN = 8, MBF_MID = MBF_KN + 20, MBF_IHW = MBF_MID + MBF_KMAX, MBF_DH = MBF_IHW + MBF_KMAX;
constexpr int MBF_CSTRIDE = MBF_KMAX * 4;
constexpr int MBF_THREADS = 128;

__device__ inline double mb_footprint(double u, double A, double B, double w1, double w2) {
  BoxDirs P, Q;
  P.ng = 0;
  if (A > 0.0) { P.a[P.ng] = A; P.m[P.ng] = 1; ++P.ng; }
  if (B > 0.0) { P.a[P.ng] = B; P.m[P.ng] = 1; ++P.ng; }
  for (int g = P.ng; g < 4; ++g) { P.a[g] = 0.0; P.m[g] = 0; }
  int small = -1;
  if (A > 0.0 && B > 0.0) {
    if (B < BSCT_SHORT_DIR * A) small = 1;
    else if (A < BSCT_SHORT_DIR * B) small = 0;
  }
  Q.ng = 0;
  if (w1 == w2) { Q.a[0] = w1; Q.m[0] = 2; Q.ng = 1; }
  else { Q.a[0] = w1; Q.m[0] = 1; Q.a[1] = w2; Q.m[1] = 1; Q.ng = 2; }
  for (int g = Q.ng; g < 4; ++g) { Q.a[g] = 0.0; Q.m[g] = 0; }
  return box_conv(u, P, small, Q);
}

// one CTA (32 threads) per view; thread q fits piece q
template <typename T>
__global__ void __launch_bounds__(32) k_mb_fp_tables(const double* __restrict__ ang, double w1, double w2,
                                                     double merge_tol, double* __restrict__ hdr,
                                                     T* __restrict__ coef) {
  const int a = blockIdx.x;
  __shared__ double kn[20];
  __shared__ int s_k;
  double s_, c_;
  sincospi(ang[a], &s_, &c_);
  const double A = fabs(c_), B = fabs(s_);
  const double W = A + B + w1 + w2;
  double* h = hdr + (long)a * MBF_DH;
  if (threadIdx.x == 0) {
    double k[16];
    int n = 0;
    for (int k0 = 0; k0 <= (A > 0.0); ++k0)
      for (int k1 = 0; k1 <= (B > 0.0); ++k1)
        for (int k2 = 0; k2 <= 1; ++k2)
          for (int k3 = 0; k3 <= 1; ++k3) k[n++] = -0.5 * W + k0 * A + k1 * B + k2 * w1 + k3 * w2;
    for (int i = 1; i < n; ++i) {  // insertion sort
      const double t = k[i];
      int j = i - 1;
      while (j >= 0 && k[j] > t) { k[j + 1] = k[j]; --j; }
      k[j + 1] = t;
    }
    // merge kinks closer than merge_tol (the ends -W/2 and W/2 stay)
    int m = 1;
    for (int i = 1; i < n; ++i)
      if (k[i] - k[m - 1] > merge_tol) k[m++] = k[i];
      else if (i == n - 1) k[m - 1] = k[i];
    for (int i = 0; i < 20; ++i) kn[i] = i < m ? k[i] : 1e300;
    s_k = m - 1;
    const bool rows = A >= B;
    h[MBF_C] = c_;
    h[MBF_S] = s_;
    h[MBF_ROWS] = rows ? 1.0 : 0.0;
    h[MBF_HW] = 0.5 * W;
    h[MBF_K] = m - 1;
    for (int i = 5; i < MBF_KN; ++i) h[i] = 0.0;
    for (int i = 0; i < 20; ++i) h[MBF_KN + i] = kn[i];
  }
  __syncthreads();
  const int K = s_k, q = threadIdx.x;
  if (q >= MBF_KMAX) return;
  T* c = coef + (long)a * MBF_CSTRIDE + 4 * q;
  if (q >= K) {
    h[MBF_MID + q] = 0.0;
    h[MBF_IHW + q] = 0.0;
    for (int i = 0; i < 4; ++i) c[i] = T(0);
    return;
  }
  const double mid = 0.5 * (kn[q] + kn[q + 1]), hw = 0.5 * (kn[q + 1] - kn[q]);
  // cubic through the 4 Chebyshev nodes cos(pi (2i + 1) / 8), then monomials in v
  double fv[4], ch[4];
  for (int i = 0; i < 4; ++i) fv[i] = mb_footprint(mid + hw * cospi((2.0 * i + 1.0) / 8.0), A, B, w1, w2);
  for (int k = 0; k < 4; ++k) {
    double acc = 0.0;
    for (int i = 0; i < 4; ++i) acc += fv[i] * cospi(k * (2.0 * i + 1.0) / 8.0);
    ch[k] = acc * (k == 0 ? 0.25 : 0.5);
  }
  c[0] = T(ch[0] - ch[2]);
  c[1] = T(ch[1] - 3.0 * ch[3]);
  c[2] = T(2.0 * ch[2]);
  c[3] = T(4.0 * ch[3]);
  h[MBF_MID + q] = mid;
  h[MBF_IHW + q] = 1.0 / hw;
}

template <typename T>
__global__ void k_mb_transpose(const T* __restrict__ a, int N, T* __restrict__ at) {
  __shared__ T t[32][33];
  const int x = blockIdx.x * 32 + threadIdx.x;
  for (int y = blockIdx.y * 32 + threadIdx.y, r = threadIdx.y; r < 32; y += 8, r += 8)
    if (x < N && y < N) t[r][threadIdx.x] = a[(long)y * N + x];
  __syncthreads();
  const int xo = blockIdx.y * 32 + threadIdx.x;
  for (int yo = blockIdx.x * 32 + threadIdx.y, r = threadIdx.y; r < 32; yo += 8, r += 8)
    if (xo < N && yo < N) at[(long)yo * N + xo] = t[threadIdx.x][r];
}

// one thread per (view, detector sample)
template <typename T>
__global__ void __launch_bounds__(MBF_THREADS) k_mb_fp_gather(const T* __restrict__ img, const T* __restrict__ imgT,
                                                              const double* __restrict__ hdr,
                                                              const T* __restrict__ coef, int N, int M, double lam,
                                                              T* __restrict__ sino) {
  const int a = blockIdx.y, m = blockIdx.x * MBF_THREADS + threadIdx.x;
  if (m >= M) return;
  const double* h = hdr + (long)a * MBF_DH;
  const bool rows = h[MBF_ROWS] != 0.0;
  const double major = rows ? h[MBF_C] : h[MBF_S], minor = rows ? h[MBF_S] : h[MBF_C];
  const double hW = h[MBF_HW];
  const int K = (int)h[MBF_K];
  const T* src = rows ? img : imgT;  // line L, position X: src[L N + X]
  const T* cf = coef + (long)a * MBF_CSTRIDE;
  const double hN = 0.5 * (N - 1);
  const double y = (m - 0.5 * (M - 1)) * lam;
  const double ihalf = hW / fabs(major);
  double total = 0.0;
  for (int L = 0; L < N; ++L) {
    // |y - (X - hN) major - (L - hN) minor| < W / 2
    const double base = y - (L - hN) * minor;
    const double ctr = base / major + hN;
    int x0 = (int)ceil(ctr - ihalf), x1 = (int)floor(ctr + ihalf);
    x0 = x0 < 0 ? 0 : x0;
    x1 = x1 > N - 1 ? N - 1 : x1;
    T part = T(0);
    const T* line = src + (long)L * N;
    for (int X = x0; X <= x1; ++X) {
      const double u = base - (X - hN) * major;
      if (!(fabs(u) < hW)) continue;
      int q = 0;
      while (q + 1 < K && h[MBF_KN + q + 1] <= u) ++q;
      const T v = T((u - h[MBF_MID + q]) * h[MBF_IHW + q]);
      const T* c = cf + 4 * q;
      T w = fma(fma(fma(c[3], v, c[2]), v, c[1]), v, c[0]);
      part = fma(w, line[X], part);
    }
    total += (double)part;
  }
  sino[(long)a * M + m] = T(total);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static size_t mb_al(size_t x) { return (x + 255) & ~(size_t)255; }

int mb_check_bp(const bsct_geom* g) {
  double w[2];
  bsct_blur_boxes(g, w);
  // widest kernel: |c| + |s| <= sqrt(2), degree 3
  int J0, nJ;
  mb_jrange(1.4142135623730951 + w[0] + w[1] + 4.0 * g->lambda_y, g->lambda_y, &J0, &nJ);
  if (nJ > MB_NJMAX) {
    bsct_set_last_message("two detector boxes: too many samples per pixel (lambda_y too small for the box widths)");
    return BSCT_ERR_UNSUPPORTED_SIZE;
  }
  return BSCT_OK;
}

size_t mb_bp_workspace(const bsct_geom* g, int precision) {
  const size_t T = precision == BSCT_F32 ? 4 : 8;
  const size_t na = (size_t)g->n_angles;
  return mb_al(na * sizeof(double)) + mb_al(na * MB_DH * sizeof(double)) + mb_al(na * MB_CSTRIDE * T) +
         mb_al(na * (size_t)g->n_bins * T) + mb_al(sizeof(int));
}

template <typename T> int mb_bp_run(const bsct_geom* g, const T* sino, T* b, char* w, cudaStream_t st) {
  const int N = g->N, M = g->n_bins, na = g->n_angles;
  double wb[2];
  bsct_blur_boxes(g, wb);
  double* ang = (double*)w;
  w += mb_al((size_t)na * sizeof(double));
  double* hdr = (double*)w;
  w += mb_al((size_t)na * MB_DH * sizeof(double));
  T* coef = (T*)w;
  w += mb_al((size_t)na * MB_CSTRIDE * sizeof(T));
  T* ct = (T*)w;
  w += mb_al((size_t)na * M * sizeof(T));
  int* status = (int*)w;
  BSCT_CUDA_TRY(cudaMemcpyAsync(ang, g->angles_pi, (size_t)na * sizeof(double), cudaMemcpyHostToDevice, st));
  BSCT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  const double tol = sizeof(T) == 4 ? 1e-6 : 1e-12;
  k_mb_bp_tables<T><<<na, 256, 0, st>>>(ang, N, M, g->lambda_y, wb[0], wb[1], tol, hdr, coef, status);
  dim3 gp((M + MB_PF_T - 1) / MB_PF_T, na);
  k_mb_prefilter<T><<<gp, MB_PF_T, 0, st>>>(hdr, sino, M, ct);
  dim3 gg((N + MB_TX - 1) / MB_TX, (N + MB_TY - 1) / MB_TY), tb(MB_TX, MB_TY);
  k_mb_bp_gather<T><<<gg, tb, 0, st>>>(hdr, coef, ct, na, N, M, b);
  count_launch(3);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}
template int mb_bp_run<float>(const bsct_geom*, const float*, float*, char*, cudaStream_t);
template int mb_bp_run<double>(const bsct_geom*, const double*, double*, char*, cudaStream_t);

size_t mb_fp_workspace(const bsct_geom* g, int precision) {
  const size_t T = precision == BSCT_F32 ? 4 : 8;
  const size_t na = (size_t)g->n_angles;
  return mb_al(na * sizeof(double)) + mb_al(na * MBF_DH * sizeof(double)) + mb_al(na * MBF_CSTRIDE * T) +
         mb_al((size_t)g->N * g->N * T);
}

template <typename T> int mb_fp_run(const bsct_geom* g, const T* c, T* sino, char* w, cudaStream_t st) {
  const int N = g->N, M = g->n_bins, na = g->n_angles;
  double wb[2];
  bsct_blur_boxes(g, wb);
  double* ang = (double*)w;
  w += mb_al((size_t)na * sizeof(double));
  double* hdr = (double*)w;
  w += mb_al((size_t)na * MBF_DH * sizeof(double));
  T* coef = (T*)w;
  w += mb_al((size_t)na * MBF_CSTRIDE * sizeof(T));
  T* cT = (T*)w;
  BSCT_CUDA_TRY(cudaMemcpyAsync(ang, g->angles_pi, (size_t)na * sizeof(double), cudaMemcpyHostToDevice, st));
  k_mb_fp_tables<T><<<na, 32, 0, st>>>(ang, wb[0], wb[1], 1e-13, hdr, coef);
  dim3 tb(32, 8), tg((N + 31) / 32, (N + 31) / 32);
  k_mb_transpose<T><<<tg, tb, 0, st>>>(c, N, cT);
  dim3 gg((M + MBF_THREADS - 1) / MBF_THREADS, na);
  k_mb_fp_gather<T><<<gg, MBF_THREADS, 0, st>>>(c, cT, hdr, coef, N, M, g->lambda_y, sino);
  count_launch(3);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}
template int mb_fp_run<float>(const bsct_geom*, const float*, float*, char*, cudaStream_t);
template int mb_fp_run<double>(const bsct_geom*, const double*, double*, char*, cudaStream_t);

}  // namespace bsct
