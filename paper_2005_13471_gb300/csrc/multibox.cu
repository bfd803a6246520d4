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
//   Chebyshev interpolation at 8 nodes of exact kernel values - K = lambda (h * beta_d),
//   the footprint h held as exact cubic pieces (FootPoly) convolved with the B-spline
//   beta_d = M_[lambda x (d+1)] by Gauss-Legendre between the kinks of both - and
//   k_mb_bp_gather sums, per pixel and view, sum_j c~[m0 + J0 + j] poly_{q,j}(v).
// Forward projection, per view: h_theta is one cubic between consecutive kinks
//   -W/2 + k0 |c| + k1 |s| + k2 w1 + k3 w2 (<= 15 pieces, W = |c| + |s| + w1 + w2), the same
//   FootPoly pieces; one thread per (view, sample) walks the image lines along the view's
//   major axis and sums h(y_m - x_k . u) c_k over the pixels of each line inside the
//   support.
// The back projection forms detector coordinates in FP64 in both precisions; the FP32
// forward projection forms each line's first footprint argument in FP64 and steps it in
// FP32.  FP32 evaluates the polynomials and accumulates in FP32, folded into FP64 sums per
// view block / image line.
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
constexpr int MB_SIG = 8, MB_MID = MB_SIG + 24, MB_IHW = MB_MID + MB_QMAX, MB_F = MB_IHW + MB_QMAX;
// then FP32 copies for the FP32 gather (72 floats in 36 doubles): floor(p00), frac(p00),
// c/lambda = c_hi + c_lo, s/lambda = s_hi + s_lo (hi parts short enough that X c_hi and
// Y s_hi are exact in FP32 for every pixel index), 2 pads, sigma[24], mid[20], 1/hw[20]
constexpr int MBF_P0 = 0, MBF_SIGF = 8, MBF_MIDF = MBF_SIGF + 24, MBF_IHWF = MBF_MIDF + MB_QMAX;
constexpr int MB_DH = MB_F + 36;
constexpr long MB_CSTRIDE = (long)MB_QMAX * MB_NJMAX * MB_NC;  // T coefficients per view
constexpr int MB_PF_T = 256, MB_PF_H = 40;
constexpr int MB_TX = 16, MB_TY = 16;
constexpr int MB_CHUNK = 128;  // (piece, offset) pairs fitted per round of the table kernel

__host__ __device__ inline void mb_jrange(double W, double lam, int* J0, int* nJ) {
  const double h = 0.5 * W / lam;
  const int j0 = (int)floor(-h) + 1;
  const int j1 = (int)ceil(h + 1.0) - 1;
  *J0 = j0;
  *nJ = j1 - j0 + 1;
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
  __shared__ FootPoly F;
  double s_, c_;
  sincospi(ang[a], &s_, &c_);
  const double A = fabs(c_), B = fabs(s_);
  const int d = (A > 0.0) + (B > 0.0) + 1;  // directions |c|, |s|, w1, w2 (non-zero) - 1
  foot_build(F, A, B, w1, w2, 1e-13);       // the view's footprint h as exact cubic pieces
  BoxDirs Q;                                // beta_d = M_[lambda x (d+1)]
  Q.a[0] = lam; Q.m[0] = d + 1; Q.ng = 1;
  for (int g = 1; g < 4; ++g) { Q.a[g] = 0.0; Q.m[g] = 0; }
  const double bh = 0.5 * (d + 1) * lam;
  double bk[5];
  for (int k = 0; k <= d + 1; ++k) bk[k] = -bh + k * lam;
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
    float* hf = reinterpret_cast<float*>(h + MB_F);
    const double pz = h[MB_P00], nz = floor(pz);
    hf[MBF_P0 + 0] = (float)nz;
    hf[MBF_P0 + 1] = (float)(pz - nz);
    int nb = 1;  // pixel indices < 2^nb
    while ((1 << nb) < N) ++nb;
    const double cs[2] = {c_ / lam, s_ / lam};
    for (int k = 0; k < 2; ++k) {
      int e;
      const double mm = frexp(cs[k], &e);
      const double hi = ldexp(trunc(ldexp(mm, 24 - nb)), e - (24 - nb));
      hf[MBF_P0 + 2 + 2 * k] = (float)hi;
      hf[MBF_P0 + 3 + 2 * k] = (float)(cs[k] - hi);
    }
    hf[6] = hf[7] = 0.f;
    for (int i = 0; i < 24; ++i) hf[MBF_SIGF + i] = i <= q ? (float)sig[i] : 2.f;
  }
  __syncthreads();
  const int Qn = s_q;
  for (int i = threadIdx.x; i < MB_QMAX; i += blockDim.x) {
    h[MB_MID + i] = i < Qn ? 0.5 * (sig[i] + sig[i + 1]) : 0.0;
    h[MB_IHW + i] = i < Qn ? 2.0 / (sig[i + 1] - sig[i]) : 0.0;
    float* hf = reinterpret_cast<float*>(h + MB_F);
    hf[MBF_MIDF + i] = (float)h[MB_MID + i];
    hf[MBF_IHWF + i] = (float)h[MB_IHW + i];
  }
  T* cv = coef + (long)a * MB_CSTRIDE;
  // unused (piece, offset) slots are zero
  for (int w = threadIdx.x; w < MB_QMAX * MB_NJMAX; w += blockDim.x) {
    const int q = w / MB_NJMAX, j = w % MB_NJMAX;
    if (q >= Qn || j >= nJ || nJ > MB_NJMAX)
      for (int i = 0; i < MB_NC; ++i) cv[(long)w * MB_NC + i] = T(0);
  }
  if (nJ > MB_NJMAX) return;  // uniform over the CTA (rejected on the host)
  // the used slots in chunks of MB_CHUNK (piece, offset) pairs: the 8 node values of every
  // pair of the chunk spread over all threads, then one thread per pair fits them
  __shared__ double fvs[MB_CHUNK * 8];
  __shared__ double ck[64];
  cheb_cos_fill<8>(ck);  // read after the first barrier of the chunk loop
  const int items = Qn * nJ;
  for (int c0 = 0; c0 < items; c0 += MB_CHUNK) {
    const int nc = items - c0 < MB_CHUNK ? items - c0 : MB_CHUNK;
    __syncthreads();  // the previous chunk's values have been fitted
    for (int it = threadIdx.x; it < nc * 8; it += blockDim.x) {
      const int w = c0 + (it >> 3), i = it & 7, q = w / nJ, j = w - q * nJ;
      const double mid = 0.5 * (sig[q] + sig[q + 1]), hw = 0.5 * (sig[q + 1] - sig[q]);
      const double f = mid + hw * ck[8 + i];
      const double u = (J0 + j - f) * lam;
      fvs[it] = fabs(u) < 0.5 * W
                    ? lam * foot_conv(F, u, -bh, bh, bk, d + 2, [&](double v) { return box_tp(-fabs(v), Q); })
                    : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      const int w = c0 + k, q = w / nJ, j = w - q * nJ;
      double mono[8];
      cheb8_monomials(fvs + 8 * k, mono, ck);
      T* c = cv + ((long)q * MB_NJMAX + j) * MB_NC;
      for (int i = 0; i < MB_NC; ++i) c[i] = T(mono[i]);
    }
  }
}

// c~ = g_s * q (Eq. 5) for the view's degree (2 or 3); one CTA per 256 outputs of one view
// the taps of both filters, formed once on the host
struct MbPfTaps {
  double q2[MB_PF_H + 1], q3[MB_PF_H + 1];
};
static MbPfTaps mb_pf_taps() {
  MbPfTaps t;
  for (int i = 0; i <= MB_PF_H; ++i) {
    t.q2[i] = 1.4142135623730951 * pow(2.0 * 1.4142135623730951 - 3.0, (double)i);  // sqrt(2) (2 sqrt(2) - 3)^i
    t.q3[i] = 1.7320508075688772 * pow(1.7320508075688772 - 2.0, (double)i);        // sqrt(3) (sqrt(3) - 2)^i
  }
  return t;
}
template <typename T>
__global__ void __launch_bounds__(MB_PF_T) k_mb_prefilter(const double* __restrict__ hdr, const T* __restrict__ g,
                                                          int M, T* __restrict__ ct, MbPfTaps taps) {
  __shared__ T qs[MB_PF_H + 1];
  __shared__ T seg[MB_PF_T + 2 * MB_PF_H];
  const int a = blockIdx.y, m0 = blockIdx.x * MB_PF_T;
  const T* gr = g + (long)a * M;
  const int d = (int)hdr[(long)a * MB_DH + MB_DEG];
  if (threadIdx.x <= MB_PF_H) qs[threadIdx.x] = T(d == 3 ? taps.q3[threadIdx.x] : taps.q2[threadIdx.x]);
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

// one thread per pixel, every view; each view's used coefficients (Q x nJ rows of 8) are
// staged in shared memory by the whole CTA, so the pixels' data-dependent row reads hit
// shared memory instead of L1
template <typename T> __host__ __device__ constexpr size_t mb_gather_smem() {
  return (size_t)(MB_QMAX - 3) * (MB_NJMAX * MB_NC + 1) * sizeof(T);  // <= 17 pieces occur
}
template <typename T>
__global__ void __launch_bounds__(MB_TX* MB_TY) k_mb_bp_gather(const double* __restrict__ hdr,
                                                               const T* __restrict__ coef, const T* __restrict__ ct,
                                                               int na, int N, int M, T* __restrict__ b) {
  extern __shared__ __align__(16) unsigned char mb_raw[];
  T* sc = reinterpret_cast<T*>(mb_raw);  // [q][j][8], j < nJ; piece rows padded by one (banks)
  const int tid = threadIdx.y * MB_TX + threadIdx.x;
  const int k1 = blockIdx.x * MB_TX + threadIdx.x, k2 = blockIdx.y * MB_TY + threadIdx.y;
  const bool inside = k1 < N && k2 < N;
  double total = 0.0;
  T part = T(0);
  for (int a = 0; a < na; ++a) {
    const double* h = hdr + (long)a * MB_DH;
    const int Q = (int)h[MB_Q], J0 = (int)h[MB_J0], nJ = (int)h[MB_NJ];
    const int row = nJ * MB_NC, rs = row + 1;
    __syncthreads();  // the previous view's coefficients have been read
    const T* src = coef + (long)a * MB_CSTRIDE;
    for (int e = tid; e < Q * row; e += MB_TX * MB_TY) {
      const int q = e / row, r = e - q * row;
      sc[q * rs + r] = src[(long)q * MB_NJMAX * MB_NC + r];
    }
    __syncthreads();
    if (inside) {
      int q = 0, mb;
      T v;
      if constexpr (sizeof(T) == 8) {
        const double p = h[MB_P00] + (double)k1 * h[MB_CL] + (double)k2 * h[MB_SL];
        const double mf = floor(p);
        const double f = p - mf;
        for (int step = 16; step > 0; step >>= 1)
          if (q + step < Q && h[MB_SIG + q + step] <= f) q += step;
        v = (f - h[MB_MID + q]) * h[MB_IHW + q];
        mb = (int)mf + J0;
      } else {
        // p = floor(p00) + frac(p00) + X c_hi + Y s_hi + (X c_lo + Y s_lo): the hi products
        // are exact, so their integer and fractional parts separate exactly in FP32
        const float* hf = reinterpret_cast<const float*>(h + MB_F);
        const float X = (float)k1, Y = (float)k2;
        const float a1 = X * hf[MBF_P0 + 2], a2 = Y * hf[MBF_P0 + 4];
        const float n1 = floorf(a1), n2 = floorf(a2);
        const float fr = (hf[MBF_P0 + 1] + (a1 - n1)) + ((a2 - n2) + fmaf(Y, hf[MBF_P0 + 5], X * hf[MBF_P0 + 3]));
        const float n3 = floorf(fr);
        const float f = fr - n3;
        for (int step = 16; step > 0; step >>= 1)
          if (q + step < Q && hf[MBF_SIGF + q + step] <= f) q += step;
        v = (f - hf[MBF_MIDF + q]) * hf[MBF_IHWF + q];
        mb = (int)hf[MBF_P0] + (int)n1 + (int)n2 + (int)n3 + J0;
      }
      const T* cq = sc + q * rs;
      const T* cr = ct + (long)a * M;
      for (int j = 0; j < nJ; ++j) {
        const int m = mb + j;
        if ((unsigned)m >= (unsigned)M) continue;
        const T* c = cq + j * MB_NC;
        T w = c[7];
#pragma unroll
        for (int i = 6; i >= 0; --i) w = fma(w, v, c[i]);
        part = fma(w, cr[m], part);
      }
    }
    if ((a & 31) == 31) { total += (double)part; part = T(0); }
  }
  total += (double)part;
  if (inside) b[(long)k2 * N + k1] = T(total);
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

// one CTA (32 threads) per view: the footprint's exact cubic pieces (foot_build), stored
// for the gather (coefficients in T)
template <typename T>
__global__ void __launch_bounds__(32) k_mb_fp_tables(const double* __restrict__ ang, double w1, double w2,
                                                     double merge_tol, double* __restrict__ hdr,
                                                     T* __restrict__ coef) {
  const int a = blockIdx.x;
  __shared__ FootPoly F;
  double s_, c_;
  sincospi(ang[a], &s_, &c_);
  const double A = fabs(c_), B = fabs(s_);
  foot_build(F, A, B, w1, w2, merge_tol);
  double* h = hdr + (long)a * MBF_DH;
  if (threadIdx.x == 0) {
    h[MBF_C] = c_;
    h[MBF_S] = s_;
    h[MBF_ROWS] = A >= B ? 1.0 : 0.0;
    h[MBF_HW] = F.hw;
    h[MBF_K] = F.K;
    for (int i = 5; i < MBF_KN; ++i) h[i] = 0.0;
    for (int i = 0; i < 20; ++i) h[MBF_KN + i] = i < 17 ? F.kn[i] : 1e300;
  }
  const int q = threadIdx.x;
  if (q >= MBF_KMAX) return;
  T* c = coef + (long)a * MBF_CSTRIDE + 4 * q;
  const bool on = q < F.K;
  h[MBF_MID + q] = on ? F.mid[q] : 0.0;
  h[MBF_IHW + q] = on ? F.ihw[q] : 0.0;
  for (int i = 0; i < 4; ++i) c[i] = on ? T(F.c[q][i]) : T(0);
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

// one thread per (view, detector sample); the view's pieces are staged in shared memory.
// FP64: every footprint argument u = y - x . u_theta in FP64.  FP32: u in FP64 at the first
// pixel of each line, then stepped by the FP32 pixel increment (<= ~6 steps: |error| below
// 1e-6 of a pixel), piece search and Horner in FP32.
template <typename T>
__global__ void __launch_bounds__(MBF_THREADS) k_mb_fp_gather(const T* __restrict__ img, const T* __restrict__ imgT,
                                                              const double* __restrict__ hdr,
                                                              const T* __restrict__ coef, int N, int M, double lam,
                                                              T* __restrict__ sino) {
  const int a = blockIdx.y, m = blockIdx.x * MBF_THREADS + threadIdx.x;
  __shared__ double s_kn[MBF_KMAX + 1], s_mid[MBF_KMAX], s_ihw[MBF_KMAX];
  __shared__ T s_c[MBF_KMAX][4];
  __shared__ T s_knt[MBF_KMAX + 1], s_midt[MBF_KMAX], s_ihwt[MBF_KMAX];
  const double* h = hdr + (long)a * MBF_DH;
  const int K = (int)h[MBF_K];
  for (int i = threadIdx.x; i <= MBF_KMAX; i += blockDim.x) {
    const double kn = i <= K ? h[MBF_KN + i] : 1e300;
    s_kn[i] = kn;
    s_knt[i] = i <= K ? T(kn) : T(3.0e38);
    if (i < MBF_KMAX) {
      s_mid[i] = h[MBF_MID + i];
      s_ihw[i] = h[MBF_IHW + i];
      s_midt[i] = T(h[MBF_MID + i]);
      s_ihwt[i] = T(h[MBF_IHW + i]);
      for (int k = 0; k < 4; ++k) s_c[i][k] = coef[(long)a * MBF_CSTRIDE + 4 * i + k];
    }
  }
  __syncthreads();
  if (m >= M) return;
  const bool rows = h[MBF_ROWS] != 0.0;
  const double major = rows ? h[MBF_C] : h[MBF_S], minor = rows ? h[MBF_S] : h[MBF_C];
  const double hW = h[MBF_HW];
  const T* src = rows ? img : imgT;  // line L, position X: src[L N + X]
  const double hN = 0.5 * (N - 1);
  const double y = (m - 0.5 * (M - 1)) * lam;
  const double ihalf = hW / fabs(major), imaj = 1.0 / major;
  const T majt = T(major), hWt = T(hW);
  double total = 0.0;
  for (int L = 0; L < N; ++L) {
    // |y - (X - hN) major - (L - hN) minor| < W / 2
    const double base = y - (L - hN) * minor;
    const double ctr = base * imaj + hN;  // the pixels at the support's ends carry h ~ 0
    int x0 = (int)ceil(ctr - ihalf), x1 = (int)floor(ctr + ihalf);
    x0 = x0 < 0 ? 0 : x0;
    x1 = x1 > N - 1 ? N - 1 : x1;
    T part = T(0);
    const T* line = src + (long)L * N;
    const T u0 = T(base - (x0 - hN) * major);
    for (int X = x0; X <= x1; ++X) {
      T w;
      if constexpr (sizeof(T) == 8) {
        const double u = base - (X - hN) * major;
        if (!(fabs(u) < hW)) continue;
        int q = 0;
        for (int step = 8; step > 0; step >>= 1)
          if (q + step < K && s_kn[q + step] <= u) q += step;
        const double v = (u - s_mid[q]) * s_ihw[q];
        w = fma(fma(fma(s_c[q][3], v, s_c[q][2]), v, s_c[q][1]), v, s_c[q][0]);
      } else {
        const T u = u0 - T(X - x0) * majt;
        if (!(fabsf(u) < hWt)) continue;
        int q = 0;
        for (int step = 8; step > 0; step >>= 1)
          if (q + step < K && s_knt[q + step] <= u) q += step;
        const T v = (u - s_midt[q]) * s_ihwt[q];
        w = fmaf(fmaf(fmaf(s_c[q][3], v, s_c[q][2]), v, s_c[q][1]), v, s_c[q][0]);
      }
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
  static const MbPfTaps taps = mb_pf_taps();
  k_mb_prefilter<T><<<gp, MB_PF_T, 0, st>>>(hdr, sino, M, ct, taps);
  dim3 gg((N + MB_TX - 1) / MB_TX, (N + MB_TY - 1) / MB_TY), tb(MB_TX, MB_TY);
  BSCT_CUDA_TRY(cudaFuncSetAttribute(k_mb_bp_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)mb_gather_smem<T>()));
  k_mb_bp_gather<T><<<gg, tb, mb_gather_smem<T>(), st>>>(hdr, coef, ct, na, N, M, b);
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
