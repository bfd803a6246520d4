// Back projection b = H^T g_hat with B-spline sinogram interpolation (Sec. 5).
//
// For view theta with footprint directions [|c|, |s|, zeta] and interpolation degree
// d (Sec. 5 degree rule), sample m contributes to pixel k with weight
//     K(y_m - t_k),  K(u) = lambda * M_[|c|, |s|, zeta, lambda x (d+1)](u),  t_k = x_k . u
// (beta_d((y - y_m)/lambda) = lambda M_[lambda^(d+1)](y - y_m), correlated with the
// footprint M_[c, s, zeta]).  Write p = (t_k - y_0)/lambda = m0 + f with m0 integer and
// f in [0, 1); then y_{m0+j} - t_k = (j - f) lambda and the weight of sample m0 + j is
// phi_j(f) = K((j - f) lambda).  Each phi_j is a piecewise polynomial in f whose kinks
// all sit in one set {0} U {frac(-kink(K) / lambda)}, so per view:
//
//   k_bp_tables (FP64): kinks sigma_0 = 0 < ... < sigma_Q = 1, and for every piece q and
//       offset j the degree-<=5 polynomial of phi_j on piece q, by Chebyshev interpolation
//       at 6 nodes of exact FP64 kernel values (the kernel is evaluated with the
//       short-direction split of bsct_boxspline.cuh, so views near the axes lose no
//       digits), stored as monomials in v = (f - mid_q) / halfwidth_q in [-1, 1];
//   k_prefilter: c~ = g_s * q for degree-2 views (Eq. 5 correction filter,
//       q[m] = sqrt(2) (2 sqrt(2) - 3)^|m|, |m| <= 40, zero outside the detector);
//   k_bp_gather: one thread per pixel, loop over views: locate f's piece, then
//       b_k += sum_j c~[m0 + j] * poly_{q,j}(v).  The detector coordinate of each warp's
//       8 x 4 pixel sub-tile is computed once per view in FP64 and the pixel offsets are
//       added in T, so FP32 keeps ~1e-6 absolute accuracy in f.
#include <math.h>

#include "bsct_boxspline.cuh"
#include "bsct_internal.h"

namespace bsct {

constexpr int BP_QMAX = 12;   // pieces per view (<= 9 occur)
constexpr int BP_NJMAX = 16;  // samples touching one pixel (lambda_y >= ~0.2)
// header: c/lambda, s/lambda, Q, J0, nJ, then the FP32 split of the detector coordinate
// p = p00 + X c/lambda + Y s/lambda (pixel X, Y): floor(p00), p00 - floor(p00), and
// c/lambda = c_hi + c_lo, s/lambda = s_hi + s_lo with hi parts short enough that
// X c_hi and Y s_hi are exact in FP32 for every pixel index of the image; last, E (below)
constexpr int BP_HDR = 12;
constexpr int BP_SIG = BP_HDR;                      // sigma[16] (padded with 2, for a 4-step search)
constexpr int BP_MI = BP_SIG + 16;                  // (mid, 1/halfwidth) of piece q at BP_MI + 2 q
// piece lookup: byte c of the BP_NL bytes at BP_LUT is the piece holding f = c / BP_NL, and
// E = header[11] is the largest number of kinks strictly inside one cell [c, c + 1) / BP_NL
// (both in T's comparisons), so with E <= 1 the piece of f is lut[cell] + (sigma[that + 1] <= f)
constexpr int BP_NL = 128;
constexpr int BP_LUT = BP_MI + 2 * BP_QMAX;
// coefficients of piece q, offset j: (c0..c3) at BP_CA + q BP_QA + 4 j, (c4, c5) at
// BP_CB + q BP_QB + 2 j; the +4 / +2 pads put the pieces one warp touches on different
// banks for the 16-byte and 8-byte reads
constexpr int BP_CA = BP_LUT + BP_NL / 4;  // 84: 16-byte aligned
constexpr int BP_QA = BP_NJMAX * 4 + 4;
constexpr int BP_CB = BP_CA + BP_QMAX * BP_QA;
constexpr int BP_QB = BP_NJMAX * 2 + 2;
constexpr int BP_STRIDE = BP_CB + BP_QMAX * BP_QB;
constexpr int BP_TX = 32, BP_TY = 8;

__host__ __device__ inline int bp_degree(double c, double s, double zeta) {
  return (c != 0.0) + (s != 0.0) + (zeta > 0.0) - 1;
}
__host__ __device__ inline void bp_jrange(double W, double lam, int* J0, int* nJ) {
  const double h = 0.5 * W / lam;
  const int j0 = (int)floor(-h) + 1;
  const int j1 = (int)ceil(h + 1.0) - 1;
  *J0 = j0;
  *nJ = j1 - j0 + 1;
}

__device__ inline void bp_dirs(double A, double B, double zeta, double lam, int d, BoxDirs* D, int* small) {
  D->ng = 0;
  if (A > 0.0) { D->a[D->ng] = A; D->m[D->ng] = 1; ++D->ng; }
  if (B > 0.0) { D->a[D->ng] = B; D->m[D->ng] = 1; ++D->ng; }
  if (zeta > 0.0) { D->a[D->ng] = zeta; D->m[D->ng] = 1; ++D->ng; }
  D->a[D->ng] = lam; D->m[D->ng] = d + 1; ++D->ng;
  for (int g = D->ng; g < 4; ++g) { D->a[g] = 0.0; D->m[g] = 0; }
  *small = -1;
  if (A > 0.0 && B > 0.0) {
    if (B < BSCT_SHORT_DIR * A) *small = 1;
    else if (A < BSCT_SHORT_DIR * B) *small = 0;
  }
}

// one CTA (256 threads) per view
template <typename T>
__global__ void __launch_bounds__(256) k_bp_tables(const double* __restrict__ ang, int N, int M, double lam,
                                                   double zeta, double merge_tol, T* __restrict__ tab,
                                                   double* __restrict__ p00, double2* __restrict__ csl,
                                                   int* __restrict__ status) {
  const int a = blockIdx.x;
  __shared__ double sig[64];
  __shared__ int Qs, Es;
  // cos(pi k (2i + 1) / 12), k, i < 6: the Chebyshev nodes (k = 1) and the fit's cosines,
  // formed once per view
  __shared__ double cosk[36];
  if (threadIdx.x < 36) cosk[threadIdx.x] = cospi((threadIdx.x / 6) * (2.0 * (threadIdx.x % 6) + 1.0) / 12.0);
  double s_, c_;
  sincospi(ang[a], &s_, &c_);
  const double A = fabs(c_), B = fabs(s_);
  const int d = bp_degree(c_, s_, zeta);
  BoxDirs D;
  int small;
  bp_dirs(A, B, zeta, lam, d, &D, &small);
  double W = 0.0;
  for (int g = 0; g < D.ng; ++g) W += D.m[g] * D.a[g];
  int J0, nJ;
  bp_jrange(W, lam, &J0, &nJ);
  if (threadIdx.x == 0) {
    // kinks of K: -W/2 + sum_g k_g a_g ; their positions in f are frac(-kink / lam)
    int n = 0;
    sig[n++] = 0.0;
    const int m0 = D.m[0], m1 = D.ng > 1 ? D.m[1] : 0, m2 = D.ng > 2 ? D.m[2] : 0, m3 = D.ng > 3 ? D.m[3] : 0;
    for (int k0 = 0; k0 <= m0; ++k0)
      for (int k1 = 0; k1 <= m1; ++k1)
        for (int k2 = 0; k2 <= m2; ++k2)
          for (int k3 = 0; k3 <= m3; ++k3) {
            double kink = -0.5 * W + k0 * D.a[0] + k1 * D.a[1] + k2 * D.a[2] + k3 * D.a[3];
            double fpos = -kink / lam;
            fpos -= floor(fpos);
            if (fpos >= 1.0) fpos = 0.0;
            if (n < 63) sig[n++] = fpos;
          }
    for (int i = 1; i < n; ++i) {  // sort
      double t = sig[i];
      int j = i - 1;
      while (j >= 0 && sig[j] > t) { sig[j + 1] = sig[j]; --j; }
      sig[j + 1] = t;
    }
    int q = 1;  // merge kinks closer than merge_tol, drop those within merge_tol of 1
    for (int i = 1; i < n; ++i)
      if (sig[i] - sig[q - 1] > merge_tol && 1.0 - sig[i] > merge_tol) sig[q++] = sig[i];
    sig[q] = 1.0;
    Qs = q;
    T* h = tab + (long)a * BP_STRIDE;
    h[0] = T(c_ / lam);
    h[1] = T(s_ / lam);
    h[2] = T(q < BP_QMAX ? q : BP_QMAX);
    h[3] = T(J0);
    h[4] = T(nJ);
    for (int i = 0; i < 16; ++i) h[BP_SIG + i] = i <= q ? T(sig[i]) : T(2.0);
    if (q > BP_QMAX || nJ > BP_NJMAX) atomicExch(status, 1);
    // detector coordinate of pixel (0, 0) in bin units, FP64
    const double x0 = -0.5 * (N - 1);
    const double pz = (x0 * c_ + x0 * s_) / lam + 0.5 * (M - 1);
    p00[a] = pz;
    csl[a] = make_double2(c_ / lam, s_ / lam);
    // FP32 split (pixel indices < 2^nb need hi parts of 24 - nb significant bits; the
    // indices reach the end of the last 64-pixel tile)
    int nb = 1;
    while ((1 << nb) < (N + 63) / 64 * 64) ++nb;
    const double nz = floor(pz);
    h[5] = T(nz);
    h[6] = T(pz - nz);
    const double cs[2] = {c_ / lam, s_ / lam};
    for (int k = 0; k < 2; ++k) {
      int e;
      const double m = frexp(cs[k], &e);                        // cs = m 2^e, 0.5 <= |m| < 1
      const double hi = ldexp(trunc(ldexp(m, 24 - nb)), e - (24 - nb));
      h[7 + 2 * k] = T(hi);
      h[8 + 2 * k] = T(cs[k] - hi);
    }
    Es = 0;
  }
  __syncthreads();
  const int Q = Qs;
  if (Q > BP_QMAX || nJ > BP_NJMAX) return;
  T* h = tab + (long)a * BP_STRIDE;
  // piece lookup, one cell a thread, with T's comparisons (those of the gathers): the
  // piece holding the cell's left end and the kinks strictly inside the cell
  if (threadIdx.x < BP_NL) {
    const T x0 = T(threadIdx.x) * T(1.0 / BP_NL), x1 = T(threadIdx.x + 1) * T(1.0 / BP_NL);
    int q0 = 0, e = 0;
    for (int r = 1; r < 16; ++r) {
      const T sr = h[BP_SIG + r];
      q0 += sr <= x0 ? 1 : 0;
      e += (x0 < sr && sr < x1) ? 1 : 0;
    }
    reinterpret_cast<unsigned char*>(h + BP_LUT)[threadIdx.x] = (unsigned char)q0;
    atomicMax(&Es, e);
  }
  for (int i = threadIdx.x; i < BP_QMAX * 6; i += blockDim.x) {  // pads
    if (i < BP_QMAX * 4) h[BP_CA + (i / 4) * BP_QA + BP_NJMAX * 4 + i % 4] = T(0);
    else h[BP_CB + ((i - BP_QMAX * 4) / 2) * BP_QB + BP_NJMAX * 2 + i % 2] = T(0);
  }
  // kernel values at the 6 Chebyshev nodes x_i = cos(pi (2i+1) / 12) of every (piece,
  // offset), spread over all threads (the near-axis views' split evaluations are costly)
  __shared__ double fvs[BP_QMAX * BP_NJMAX * 6];
  for (int it = threadIdx.x; it < Q * nJ * 6; it += blockDim.x) {
    const int i = it % 6, w = it / 6, q = w / nJ, j = w - q * nJ;
    const double mid = 0.5 * (sig[q] + sig[q + 1]), hw = 0.5 * (sig[q + 1] - sig[q]);
    const double f = mid + hw * cosk[6 + i];
    const double u = (J0 + j - f) * lam;
    fvs[it] = (fabs(u) < 0.5 * W) ? lam * box_eval(u, D, small) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) h[11] = T(Es);
  for (int w = threadIdx.x; w < BP_QMAX * BP_NJMAX; w += blockDim.x) {
    const int q = w / BP_NJMAX, j = w % BP_NJMAX;
    T* ca = h + BP_CA + q * BP_QA + j * 4;
    T* cb = h + BP_CB + q * BP_QB + j * 2;
    if (q >= Q || j >= nJ) {
      for (int i = 0; i < 4; ++i) ca[i] = T(0);
      cb[0] = T(0);
      cb[1] = T(0);
      if (j == 0 && q < BP_QMAX) { h[BP_MI + 2 * q] = T(0); h[BP_MI + 2 * q + 1] = T(0); }
      continue;
    }
    const double lo = sig[q], hi = sig[q + 1];
    const double mid = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
    if (j == 0) { h[BP_MI + 2 * q] = T(mid); h[BP_MI + 2 * q + 1] = T(1.0 / hw); }
    const double* fv = fvs + (q * nJ + j) * 6;
    double ch[6];
    for (int k = 0; k < 6; ++k) {
      double acc = 0.0;
      for (int i = 0; i < 6; ++i) acc += fv[i] * cosk[6 * k + i];
      ch[k] = acc * (k == 0 ? 1.0 / 6.0 : 2.0 / 6.0);
    }
    // Chebyshev -> monomial: T0=1, T1=v, T2=2v^2-1, T3=4v^3-3v, T4=8v^4-8v^2+1, T5=16v^5-20v^3+5v
    const double m0 = ch[0] - ch[2] + ch[4];
    const double m1 = ch[1] - 3.0 * ch[3] + 5.0 * ch[5];
    const double m2 = 2.0 * ch[2] - 8.0 * ch[4];
    const double m3 = 4.0 * ch[3] - 20.0 * ch[5];
    const double m4 = 8.0 * ch[4];
    const double m5 = 16.0 * ch[5];
    ca[0] = T(m0); ca[1] = T(m1); ca[2] = T(m2); ca[3] = T(m3);
    cb[0] = T(m4); cb[1] = T(m5);
  }
}

// One CTA per 256 outputs of one view: the sinogram segment with a 40-sample halo on
// each side (zero outside the detector) is staged in shared memory and the symmetric
// 81-tap filter is summed from the outermost taps inwards in T.
constexpr int PF_T = 256, PF_H = 40;
// the filter taps q[0..40], formed once on the host (a pow per tap per CTA kept the FP64
// pipe of this part busy for most of the kernel)
struct PfTaps {
  double q[PF_H + 1];
};
static PfTaps pf_taps() {
  PfTaps t;
  const double z1 = 2.0 * 1.4142135623730951 - 3.0;
  for (int i = 0; i <= PF_H; ++i) t.q[i] = 1.4142135623730951 * pow(z1, (double)i);
  return t;
}
template <typename T>
__global__ void __launch_bounds__(PF_T) k_prefilter(const double* __restrict__ ang, const T* __restrict__ g, int na,
                                                    int M, double zeta, T* __restrict__ ct, PfTaps taps) {
  __shared__ T qs[PF_H + 1];
  __shared__ T seg[PF_T + 2 * PF_H];
  __shared__ int deg2;
  const int a = blockIdx.y, m0 = blockIdx.x * PF_T;
  const T* gr = g + (long)a * M;
  if (threadIdx.x == 0) {
    double s_, c_;
    sincospi(ang[a], &s_, &c_);
    deg2 = bp_degree(c_, s_, zeta) == 2;
  }
  if (threadIdx.x <= PF_H) qs[threadIdx.x] = T(taps.q[threadIdx.x]);
  for (int i = threadIdx.x; i < PF_T + 2 * PF_H; i += PF_T) {
    const int mm = m0 - PF_H + i;
    seg[i] = (mm >= 0 && mm < M) ? gr[mm] : T(0);
  }
  __syncthreads();
  const int m = m0 + threadIdx.x;
  if (m >= M) return;
  const T* c = seg + PF_H + threadIdx.x;
  if (!deg2) {
    ct[(long)a * M + m] = c[0];
    return;
  }
  T acc = T(0);
#pragma unroll 8
  for (int j = PF_H; j >= 1; --j) acc = fma(qs[j], c[-j] + c[j], acc);
  ct[(long)a * M + m] = fma(qs[0], c[0], acc);
}

__device__ __forceinline__ void cp_async16_bp(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_bp() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_bp() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T> struct Acc { typedef float part; };
template <> struct Acc<double> { typedef double part; };

// Each warp owns an 8 x 4 pixel sub-tile; its detector coordinate is computed per view in
// FP64 by the warp itself, so the FP32 part of p only spans |offset| <= 7|c| + 3|s| + 1.
// The tables of BP_CH views at a time are staged in shared memory (one float4 copy per
// chunk), so the per-pair piece search and coefficient reads hit shared memory.
constexpr int BP_CH = 8;
// Detector samples one view needs for a 32 x 8 tile.  Over the tile the detector
// coordinate spans at most (31|c| + 7|s|) / lambda <= 31.7805 / lambda bins; a pixel's
// first sample index is floor(p) + J0 with floor(p) in [floor(p_min) - 1, p_max + 1]
// (the -1 / +1 absorb FP32 rounding of p), and it reads nJ <= BP_NJMAX samples from
// there, so the window [floor(p_min) - 1 + J0, ...) needs 31.7805 / lambda + BP_NJMAX + 3
// entries; bp_window() adds one more and rounds up to a multiple of 4.
inline int bp_window(double lambda) {
  const int w = (int)ceil(31.7806 / lambda) + BP_NJMAX + 4;
  return (w + 3) & ~3;
}
template <typename T> size_t bp_gather_smem(int win) { return (size_t)BP_CH * (BP_STRIDE + win) * sizeof(T); }

// the six coefficients of one (piece, offset) from shared memory: one 16-byte and one
// 8-byte read in FP32 (three 16-byte reads in FP64)
__device__ inline void bp_load6(const float* a, const float* b, float c[6]) {
  const float4 x = *reinterpret_cast<const float4*>(a);
  const float2 y = *reinterpret_cast<const float2*>(b);
  c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w; c[4] = y.x; c[5] = y.y;
}
__device__ inline void bp_load6(const double* a, const double* b, double c[6]) {
  const double2 x0 = *reinterpret_cast<const double2*>(a), x1 = *reinterpret_cast<const double2*>(a + 2);
  const double2 y = *reinterpret_cast<const double2*>(b);
  c[0] = x0.x; c[1] = x0.y; c[2] = x1.x; c[3] = x1.y; c[4] = y.x; c[5] = y.y;
}

template <typename T>
__global__ void __launch_bounds__(BP_TX* BP_TY) k_bp_gather(const T* __restrict__ tab, const double2* __restrict__ csl,
                                                          const double* __restrict__ p00, const T* __restrict__ ct,
                                                          int na, int N, int M, int win, T* __restrict__ b) {
  constexpr int WX = 8, WY = 4;
  extern __shared__ __align__(16) unsigned char bp_smraw[];
  T* stab = reinterpret_cast<T*>(bp_smraw);  // [BP_CH][BP_STRIDE] view tables
  T* s_ct = stab + BP_CH * BP_STRIDE;        // [BP_CH][win] detector samples of this tile
  __shared__ int s_mlo[BP_CH];
  __shared__ int s_mb[8][BP_CH];
  __shared__ T s_fb[8][BP_CH];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int TX0 = blockIdx.x * BP_TX, TY0 = blockIdx.y * BP_TY;
  const int X0 = TX0 + (w & 3) * WX, Y0 = TY0 + (w >> 2) * WY;
  const int lx = lane & 7, ly = lane >> 3;
  const int k1 = X0 + lx, k2 = Y0 + ly;
  double total = 0.0;
  typename Acc<T>::part part = 0;
  for (int a0 = 0; a0 < na; a0 += BP_CH) {
    const int nc = min(BP_CH, na - a0);
    __syncthreads();  // previous chunk's tables are no longer read
    {
      constexpr int V = 16 / sizeof(T);  // elements per 16-byte vector
      const int nv = nc * BP_STRIDE / V;
      const float4* src = reinterpret_cast<const float4*>(tab + (long)a0 * BP_STRIDE);
      float4* dst = reinterpret_cast<float4*>(stab);
      for (int i = threadIdx.x; i < nv; i += blockDim.x) dst[i] = src[i];
    }
    if (threadIdx.x < nc) {
      // lowest sample any pixel of the tile touches for this view (tile corners, FP64)
      const int a = a0 + threadIdx.x;
      const double2 u = csl[a];
      const double pa = p00[a] + (double)TX0 * u.x + (double)TY0 * u.y;
      const double ex = (double)(BP_TX - 1) * u.x, ey = (double)(BP_TY - 1) * u.y;
      const double pmin = pa + (ex < 0 ? ex : 0.0) + (ey < 0 ? ey : 0.0);
      const int J0 = (int)tab[(long)a * BP_STRIDE + 3];
      s_mlo[threadIdx.x] = (int)floor(pmin) - 1 + J0;
    }
    if (lane < nc) {
      const double2 u = csl[a0 + lane];
      const double pt = p00[a0 + lane] + (double)X0 * u.x + (double)Y0 * u.y;
      const double mb = floor(pt);
      s_mb[w][lane] = (int)mb;
      s_fb[w][lane] = T(pt - mb);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc * win; i += blockDim.x) {
      const int ai = i / win, k = i - ai * win;
      const int m = s_mlo[ai] + k;
      s_ct[i] = ((unsigned)m < (unsigned)M) ? ct[(long)(a0 + ai) * M + m] : T(0);
    }
    __syncthreads();
    for (int ai = 0; ai < nc; ++ai) {
      const T* h = stab + ai * BP_STRIDE;
      const T cl = h[0], sl = h[1];
      const int J0 = (int)h[3], nJ = (int)h[4];
      const T pl = s_fb[w][ai] + T(lx) * cl + T(ly) * sl;
      const T fl = floor(pl);
      const T f = pl - fl;
      const int moff = s_mb[w][ai] + (int)fl + J0 - s_mlo[ai];  // window index of offset j = 0
      int q = 0;
#pragma unroll
      for (int step = 8; step > 0; step >>= 1)
        if (h[BP_SIG + q + step] <= f) q += step;
      const int Qm1 = (int)h[2] - 1;
      q = q < Qm1 ? q : Qm1;  // f rounded up to 1.0: the last piece's right end
      const T v = (f - h[BP_MI + 2 * q]) * h[BP_MI + 2 * q + 1];
      const T* ca = h + BP_CA + q * BP_QA;
      const T* cb = h + BP_CB + q * BP_QB;
      const T* cw = s_ct + ai * win + moff;
      for (int j = 0; j < nJ; ++j) {
        T c[6];
        bp_load6(ca + j * 4, cb + j * 2, c);
        T wv = c[5];
        wv = fma(wv, v, c[4]);
        wv = fma(wv, v, c[3]);
        wv = fma(wv, v, c[2]);
        wv = fma(wv, v, c[1]);
        wv = fma(wv, v, c[0]);
        part += wv * cw[j];
      }
    }
    if (((a0 / BP_CH) & 3) == 3) { total += (double)part; part = 0; }
  }
  total += (double)part;
  if (k1 < N && k2 < N) b[(long)k2 * N + k1] = T(total);
}

// ------------------------------------------------------------------------------------
// Spline-window gather (FP32, lambda_y >= BS_LAMBDA_MIN).  For one view the pixel sum
//     b_k += sum_j c~[m0 + J0 + j] phi_j(f),  p_k = m0 + f,
// is a function F(p_k) of the detector coordinate alone, and on piece q of bin m0 it is
// one degree-5 polynomial in v = (f - mid_q) / halfwidth_q whose coefficients are
// sum_j c~[m0 + J0 + j] coef_{q,j}.  A CTA owns a 64 x 64 tile; per view it first forms
// those coefficients for every bin slot the tile touches (<= 153 slots, ~0.2 extra FMA
// per pixel-view pair), then every pixel costs one piece lookup and one Horner step.
// The next view's piece table (cp.async) and detector-sample window are fetched while
// the current view is processed.  A warp owns a 16 x 8 BS_KY block of the tile and one read
// of the coefficients by its 32 lanes covers a compact 4 x 8 pixel block, whose (slot,
// piece) records are few and, stored slot-major, mostly on distinct banks; lane (lx, ly)
// takes the pixels (lx + 4 i, ly + 8 k), i < 4, k < BS_KY.  The detector coordinate of a lane's
// first pixel comes from the exact FP32 split of the view's steps, and the offsets 4 i c
// and 8 k s are split the same way into integer and fractional parts, so the FP32 sum
// that decides the piece stays below 3 bins.  Every 32 views the FP32 partial sum acc is
// moved into the FP32 total th by an exact two-sum, th + acc = th' + e, and the rounding
// error e stays in acc: th + acc always holds the running sum without loss (as an FP64
// total would), with no FP64 instruction (GB300 issues FP64 at 1/64 of the FP32 rate).
// ------------------------------------------------------------------------------------
constexpr int BS_TS = 64;                          // tile edge (pixels)
constexpr int BS_KY = 4;                           // rows (8 apart) of a lane's pixels
constexpr int BS_NP = 4 * BS_KY;                   // pixels of a lane
constexpr int BS_NT = BS_TS * BS_TS / BS_NP;       // threads of a tile
constexpr int BS_MINB = BS_KY == 4 ? 3 : 2;        // CTAs per SM (registers)
constexpr double BS_LAMBDA_MIN = 0.6;              // window <= 63 sqrt(2) / lambda + 4 <= 153
constexpr int BS_WMAX = 160;                       // bin slots of the coefficient window
// the record of bin slot s, piece q is entry s Q + q (Q pieces in this view): along a
// pixel block the (slot, piece) pairs met in order of the detector coordinate are
// consecutive entries
constexpr int BS_NREC = BS_WMAX * BP_QMAX;
constexpr int BS_CW = BS_WMAX + BP_NJMAX + 4;      // detector-sample window
struct BsHeader {
  double p00, c, s;   // detector coordinate of pixel (0, 0) and its steps, in bins
  int m0lo, W, J0, nJ, Q;
};
constexpr size_t bs_smem() {
  return (size_t)BS_NREC * (16 + 8) + 2 * (size_t)BP_STRIDE * 4 + 2 * (size_t)BS_CW * 4;
}

// blockIdx.z takes views [z vc, min(na, (z + 1) vc)); with more than one z the sums go to
// the partial image out + z N^2 (summed in order by k_bp_reduce), else to out.
__global__ void __launch_bounds__(BS_NT, BS_MINB) k_bp_spline(const float* __restrict__ tab, const double2* __restrict__ csl,
                                                        const double* __restrict__ p00, const float* __restrict__ ct,
                                                        int na, int vc, int N, int M, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char bs_raw[];
  float4* FcA = reinterpret_cast<float4*>(bs_raw);             // [slot][piece] c0..c3
  float2* FcB = reinterpret_cast<float2*>(FcA + BS_NREC);      // [slot][piece] c4, c5
  float* tb = reinterpret_cast<float*>(FcB + BS_NREC);         // [2][BP_STRIDE]
  float* ctw = tb + 2 * BP_STRIDE;                                  // [2][BS_CW]
  __shared__ BsHeader hdr[2];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int TX0 = blockIdx.x * BS_TS, TY0 = blockIdx.y * BS_TS;
  const int Xb = TX0 + 16 * (w & 3) + (lane & 3), Yb = TY0 + 8 * BS_KY * (w >> 2) + (lane >> 2);

  auto header = [&](int a, BsHeader& h) {
    const double2 u = csl[a];
    h.p00 = p00[a];
    h.c = u.x;
    h.s = u.y;
    const double pa = h.p00 + (double)TX0 * u.x + (double)TY0 * u.y;
    const double ex = (double)(BS_TS - 1) * u.x, ey = (double)(BS_TS - 1) * u.y;
    const double pmin = pa + (ex < 0 ? ex : 0.0) + (ey < 0 ? ey : 0.0);
    const double pmax = pa + (ex > 0 ? ex : 0.0) + (ey > 0 ? ey : 0.0);
    h.m0lo = (int)floor(pmin) - 1;
    const int W = (int)floor(pmax) + 1 - h.m0lo + 1;
    h.W = W < BS_WMAX ? W : BS_WMAX;  // W <= 153 for lambda >= BS_LAMBDA_MIN
    const float* t = tab + (long)a * BP_STRIDE;
    h.Q = (int)t[2];
    h.J0 = (int)t[3];
    h.nJ = (int)t[4];
  };
  auto stage_table = [&](int a, int buf) {
    const char* src = reinterpret_cast<const char*>(tab + (long)a * BP_STRIDE);
    char* dst = reinterpret_cast<char*>(tb + buf * BP_STRIDE);
    for (int q = threadIdx.x; q < BP_STRIDE * 4 / 16; q += BS_NT) cp_async16_bp(dst + q * 16, src + q * 16);
    cp_async_commit_bp();
  };
  auto sample = [&](int a, const BsHeader& h, int t) -> float {
    const int m = h.m0lo + h.J0 + t;
    return (t < h.W + h.nJ - 1 && (unsigned)m < (unsigned)M) ? ct[(long)a * M + m] : 0.f;
  };

  const int a_begin = blockIdx.z * vc, a_end = min(na, a_begin + vc);
  float* b = out + (long)blockIdx.z * N * N;
  // the next view's header (global loads, FP64) is formed by lane 0 of the last warp: the
  // window work items go to the low threads first, so that warp is the least loaded and
  // the loads' latency overlaps the other warps' window work
  constexpr int HDR_T = BS_NT - 32;
  // prologue: first view
  if (threadIdx.x == HDR_T) header(a_begin, hdr[0]);
  stage_table(a_begin, 0);
  __syncthreads();
  if (threadIdx.x < BS_CW) ctw[threadIdx.x] = sample(a_begin, hdr[0], threadIdx.x);
  cp_async_wait_bp();

  float acc[BS_NP];
  float th[BS_NP];  // running sum = th + acc
#pragma unroll
  for (int i = 0; i < BS_NP; ++i) { acc[i] = 0.f; th[i] = 0.f; }

  for (int a = a_begin; a < a_end; ++a) {
    const int buf = (a - a_begin) & 1;
    __syncthreads();  // view a staged; the previous view's pixel phase is done
    if (a + 1 < a_end) {
      if (threadIdx.x == HDR_T) header(a + 1, hdr[buf ^ 1]);
      stage_table(a + 1, buf ^ 1);
    }
    // coefficient window: F on (slot s, piece q) = sum_j c~[m0lo + s + J0 + j] coef_{q,j}.
    // A work item is 2 consecutive slots of one piece: the coefficients are read once per j
    // for both, the samples slide through registers (one shared load per j), and the six
    // sums of a slot are three packed FP32 pairs (fma.rn.f32x2: per element the same
    // rounding and order as scalar FMAs, so the window is bit-identical to one slot an item)
    {
      const BsHeader& h = hdr[buf];
      const float* t = tb + buf * BP_STRIDE;
      const float* cw = ctw + buf * BS_CW;
      const int W = h.W, nJ = h.nJ, Q = h.Q, items = Q * ((W + 1) >> 1);
      for (int it = threadIdx.x; it < items; it += BS_NT) {
        const int g = it / Q, q = it - g * Q, s0 = g << 1;
        const float* ca = t + BP_CA + q * BP_QA;
        const float* cb = t + BP_CB + q * BP_QB;
        float2 a01 = make_float2(0.f, 0.f), a23 = a01, a45 = a01, b01 = a01, b23 = a01, b45 = a01;
        float c0 = cw[s0];
        for (int j = 0; j < nJ; ++j) {
          const float c1 = cw[s0 + j + 1];
          const float4 x = *reinterpret_cast<const float4*>(ca + 4 * j);
          const float2 y = *reinterpret_cast<const float2*>(cb + 2 * j);
          const float2 x01 = make_float2(x.x, x.y), x23 = make_float2(x.z, x.w);
          const float2 p0 = make_float2(c0, c0), p1 = make_float2(c1, c1);
          a01 = __ffma2_rn(p0, x01, a01);
          a23 = __ffma2_rn(p0, x23, a23);
          a45 = __ffma2_rn(p0, y, a45);
          b01 = __ffma2_rn(p1, x01, b01);
          b23 = __ffma2_rn(p1, x23, b23);
          b45 = __ffma2_rn(p1, y, b45);
          c0 = c1;
        }
        FcA[s0 * Q + q] = make_float4(a01.x, a01.y, a23.x, a23.y);
        FcB[s0 * Q + q] = a45;
        if (s0 + 1 < W) {
          FcA[(s0 + 1) * Q + q] = make_float4(b01.x, b01.y, b23.x, b23.y);
          FcB[(s0 + 1) * Q + q] = b45;
        }
      }
    }
    __syncthreads();  // window ready; next header visible
    float cnext = 0.f;
    if (a + 1 < a_end && threadIdx.x < BS_CW) cnext = sample(a + 1, hdr[buf ^ 1], threadIdx.x);
    // pixels
    {
      const BsHeader& h = hdr[buf];
      const float* t = tb + buf * BP_STRIDE;
      // p = floor(p00) + frac(p00) + X c_hi + Y s_hi + (X c_lo + Y s_lo): the two hi
      // products are exact, so their integer and fractional parts separate exactly
      const float X = (float)Xb, Y = (float)Yb;
      const float a1 = X * t[7], a2 = Y * t[9];
      const float n1 = floorf(a1), n2 = floorf(a2);
      const float fr = (t[6] + (a1 - n1)) + ((a2 - n2) + fmaf(Y, t[10], X * t[8]));
      const float n3 = floorf(fr);
      const int mb = (int)t[5] + (int)n1 + (int)n2 + (int)n3 - h.m0lo;
      const float fb = fr - n3;
      const int Q = h.Q, Qm1 = Q - 1;
      const unsigned char* lut = reinterpret_cast<const unsigned char*>(t + BP_LUT);
      // offsets 8 k s of the lane's rows: integer part and fraction (+ the lo part)
      float gy[BS_KY];
      int ny[BS_KY];
#pragma unroll
      for (int k = 0; k < BS_KY; ++k) {
        const float hy = (float)(8 * k) * t[9];  // exact
        const float fy = floorf(hy);
        ny[k] = (int)fy;
        gy[k] = (hy - fy) + (float)(8 * k) * t[10];
      }
      // the piece of f: one lookup and one compare where no cell holds two kinks (E <= 1,
      // the same piece as the search), else a 4-step search; the branch is per view
      const bool by_lut = t[11] <= 1.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float hx = (float)(4 * i) * t[7];  // exact
        const float fx = floorf(hx);
        const int nx = mb + (int)fx;
        const float gx = fb + ((hx - fx) + (float)(4 * i) * t[8]);
#pragma unroll
        for (int k = 0; k < BS_KY; ++k) {
          const float pl = gx + gy[k];
          const float fl = floorf(pl);
          const float f = pl - fl;
          const int slot = nx + ny[k] + (int)fl;
          int q = 0;
          if (by_lut) {
            const int cell = (int)(f * (float)BP_NL);
            q = lut[cell < BP_NL - 1 ? cell : BP_NL - 1];
            q += t[BP_SIG + q + 1] <= f ? 1 : 0;
          } else {
#pragma unroll
            for (int step = 8; step > 0; step >>= 1)
              if (t[BP_SIG + q + step] <= f) q += step;
          }
          q = q < Qm1 ? q : Qm1;  // f rounded up to 1.0: the last piece's right end
          const float2 mi = *reinterpret_cast<const float2*>(t + BP_MI + 2 * q);
          const float v = (f - mi.x) * mi.y;
          const float4 x = FcA[slot * Q + q];
          const float2 y = FcB[slot * Q + q];
          float r = fmaf(y.y, v, y.x);
          r = fmaf(r, v, x.w);
          r = fmaf(r, v, x.z);
          r = fmaf(r, v, x.y);
          r = fmaf(r, v, x.x);
          acc[4 * k + i] += r;
        }
      }
    }
    if (a + 1 < a_end && threadIdx.x < BS_CW) ctw[(buf ^ 1) * BS_CW + threadIdx.x] = cnext;
    if (((a - a_begin) & 31) == 31) {
#pragma unroll
      for (int i = 0; i < BS_NP; ++i) {  // two-sum: th + acc = sum + e exactly
        const float sum = th[i] + acc[i];
        const float bb = sum - th[i];
        const float e = (th[i] - (sum - bb)) + (acc[i] - bb);
        th[i] = sum;
        acc[i] = e;
      }
    }
    cp_async_wait_bp();
  }
#pragma unroll
  for (int k = 0; k < BS_KY; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int X = Xb + 4 * i, Y = Yb + 8 * k;
      if (X < N && Y < N)
        b[(long)Y * N + X] = (float)((double)th[4 * k + i] + (double)acc[4 * k + i]);
    }
}

// b = sum over z of part[z] (fixed order)
__global__ void k_bp_reduce(const float* __restrict__ part, int S, long n, float* __restrict__ b) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int z = 0; z < S; ++z) acc += (double)part[(long)z * n + i];
  b[i] = (float)acc;
}

// View splits of the spline gather: blockIdx.z takes 1 / S of the views, and the S partial
// images are summed in order by k_bp_reduce.  At least enough splits that a small image
// still fills about 1024 CTAs, at most four times that (and >= 16 views per split); within
// that range the split is chosen so that the CTAs fill the resident slots of the current
// GPU (SMs x resident CTAs per SM) in whole waves (the last wave of 1024 tiles on 456 slots
// would otherwise run a quarter full).  The workspace is sized for the largest split of the range, so it does
// not depend on the device.
static void bp_split_range(int N, int na, double lambda, int precision, int* smin, int* smax) {
  *smin = *smax = 1;
  if (precision != BSCT_F32 || lambda < BS_LAMBDA_MIN) return;
  const int t = (N + BS_TS - 1) / BS_TS;
  const int lim = na / 16 > 1 ? na / 16 : 1;
  const int s0 = (1024 + t * t - 1) / (t * t);
  *smin = s0 < lim ? s0 : lim;
  *smax = 4 * s0 < lim ? 4 * s0 : lim;
}
int bp_view_split(int N, int na, double lambda, int precision) {
  int smin, smax;
  bp_split_range(N, na, lambda, precision, &smin, &smax);
  if (smax == smin) return smin;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    return smin;
  }
  int per_sm = 0;
  if (cudaFuncSetAttribute(k_bp_spline, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs_smem()) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bp_spline, BS_NT, bs_smem()) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = BS_MINB;
  }
  const int t = (N + BS_TS - 1) / BS_TS;
  const double slots = (double)per_sm * sms;
  int best = smin;
  double best_score = -1.0;
  for (int S = smin; S <= smax; ++S) {
    const double waves = (double)t * t * S / slots;
    const double score = waves / ceil(waves) - 0.002 * (S - smin);  // fill, then fewer splits
    if (score > best_score + 1e-12) { best_score = score; best = S; }
  }
  return best;
}
size_t bp_partial_bytes(int N, int na, double lambda, int precision) {
  int smin, smax;
  bp_split_range(N, na, lambda, precision, &smin, &smax);
  return smax > 1 ? (size_t)smax * N * N * sizeof(float) : 0;
}
}  // namespace bsct

using namespace bsct;

int bsct_check_geom(const bsct_geom* g);

static size_t bp_workspace(const bsct_geom* g, int precision) {
  double wb[2];
  if (bsct_blur_boxes(g, wb) == 2) return mb_bp_workspace(g, precision);
  const size_t T = precision == BSCT_F32 ? 4 : 8;
  size_t b = 0;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  b += al((size_t)g->n_angles * sizeof(double));             // angles
  b += al((size_t)g->n_angles * sizeof(double));             // p00
  b += al((size_t)g->n_angles * sizeof(double2));            // (c, s) / lambda
  b += al((size_t)g->n_angles * BP_STRIDE * T);               // tables
  b += al((size_t)g->n_angles * g->n_bins * T);               // prefiltered sinogram
  b += al(sizeof(int));                                       // status
  b += al(bp_partial_bytes(g->N, g->n_angles, g->lambda_y, precision));  // partial images
  return b;
}

extern "C" int bsct_backproject_workspace(const bsct_geom* geom, int precision, size_t* bytes) {
  int rc = bsct_check_geom(geom);
  if (rc != BSCT_OK) return rc;
  if (!bytes) { bsct_set_last_message("bytes is NULL"); return BSCT_ERR_INVALID_ARG; }
  if (precision != BSCT_F32 && precision != BSCT_F64) { bsct_set_last_message("precision"); return BSCT_ERR_INVALID_ARG; }
  *bytes = bp_workspace(geom, precision);
  return BSCT_OK;
}

namespace bsct {
// per-geometry part: view tables (device angles in p.ang must already be uploaded)
template <typename T> int bp_make_tables(const BpPlan& p, cudaStream_t st) {
  BSCT_CUDA_TRY(cudaMemsetAsync(p.status, 0, sizeof(int), st));
  const double tol = sizeof(T) == 4 ? 1e-6 : 1e-12;
  k_bp_tables<T><<<p.na, 256, 0, st>>>(p.ang, p.N, p.M, p.lambda, p.zeta, tol, (T*)p.tab, p.p00, p.csl, p.status);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}
// per-sinogram part: prefilter into ct ([na][M] scratch), then gather into b
template <typename T> int bp_apply(const BpPlan& p, const T* sino, T* ct, T* b, cudaStream_t st) {
  dim3 gp((p.M + PF_T - 1) / PF_T, p.na);
  static const PfTaps taps = pf_taps();
  k_prefilter<T><<<gp, PF_T, 0, st>>>(p.ang, sino, p.na, p.M, p.zeta, ct, taps);
  if constexpr (sizeof(T) == 4) {
    if (p.lambda >= BS_LAMBDA_MIN) {
      const int S = bp_view_split(p.N, p.na, p.lambda, BSCT_F32);
      if (S > 1 && !p.part) { bsct_set_last_message("back projection: no partial-image scratch"); return BSCT_ERR_INVALID_ARG; }
      const int vc = (p.na + S - 1) / S;
      dim3 gs((p.N + BS_TS - 1) / BS_TS, (p.N + BS_TS - 1) / BS_TS, (p.na + vc - 1) / vc);
      BSCT_CUDA_TRY(cudaFuncSetAttribute(k_bp_spline, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs_smem()));
      k_bp_spline<<<gs, BS_NT, bs_smem(), st>>>((const float*)p.tab, p.csl, p.p00, (const float*)ct, p.na, vc, p.N,
                                               p.M, gs.z > 1 ? p.part : (float*)b);
      count_launch(2);
      if (gs.z > 1) {
        const long n = (long)p.N * p.N;
        k_bp_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p.part, (int)gs.z, n, (float*)b);
        count_launch();
      }
      BSCT_CUDA_TRY(cudaGetLastError());
      return BSCT_OK;
    }
  }
  dim3 gg((p.N + BP_TX - 1) / BP_TX, (p.N + BP_TY - 1) / BP_TY);
  const int win = bp_window(p.lambda);
  const size_t smem = bp_gather_smem<T>(win);
  BSCT_CUDA_TRY(cudaFuncSetAttribute(k_bp_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_bp_gather<T><<<gg, BP_TX * BP_TY, smem, st>>>((const T*)p.tab, p.csl, p.p00, ct, p.na, p.N, p.M, win, b);
  count_launch(2);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}
template int bp_make_tables<float>(const BpPlan&, cudaStream_t);
template int bp_make_tables<double>(const BpPlan&, cudaStream_t);
template int bp_apply<float>(const BpPlan&, const float*, float*, float*, cudaStream_t);
template int bp_apply<double>(const BpPlan&, const double*, double*, double*, cudaStream_t);

size_t bp_table_bytes(int n_angles, int precision) {
  return (size_t)n_angles * BP_STRIDE * (precision == BSCT_F32 ? 4 : 8);
}
}  // namespace bsct

template <typename T>
static int bp_run(const bsct_geom* g, const T* sino, T* b, char* work, cudaStream_t st) {
  const int na = g->n_angles, M = g->n_bins, N = g->N;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  BpPlan p;
  double wb[2];
  bsct_blur_boxes(g, wb);  // one box (or none) here
  p.N = N; p.na = na; p.M = M; p.lambda = g->lambda_y; p.zeta = wb[0];
  p.ang = (double*)work;
  work += al((size_t)na * sizeof(double));
  p.p00 = (double*)work;
  work += al((size_t)na * sizeof(double));
  p.csl = (double2*)work;
  work += al((size_t)na * sizeof(double2));
  p.tab = work;
  work += al((size_t)na * BP_STRIDE * sizeof(T));
  T* d_ct = (T*)work;
  work += al((size_t)na * M * sizeof(T));
  p.status = (int*)work;
  work += al(sizeof(int));
  p.part = bp_partial_bytes(N, na, g->lambda_y, sizeof(T) == 4 ? BSCT_F32 : BSCT_F64) ? (float*)work : nullptr;
  BSCT_CUDA_TRY(cudaMemcpyAsync(p.ang, g->angles_pi, na * sizeof(double), cudaMemcpyHostToDevice, st));
  int rc = bp_make_tables<T>(p, st);
  if (rc != BSCT_OK) return rc;
  return bp_apply<T>(p, sino, d_ct, b, st);
}

int bsct_check_bp_geom(const bsct_geom* geom) {
  if (geom->N < 1 || geom->N > 16384) { bsct_set_last_message("N out of range"); return BSCT_ERR_UNSUPPORTED_SIZE; }
  double wb[2];
  if (bsct_blur_boxes(geom, wb) == 2) return mb_check_bp(geom);
  // widest kernel: |c| + |s| <= sqrt(2), degree <= 2
  const double W = 1.4142135623730951 + wb[0] + 3.0 * geom->lambda_y;
  int J0, nJ;
  bp_jrange(W, geom->lambda_y, &J0, &nJ);
  if (nJ > BP_NJMAX) { bsct_set_last_message("lambda_y too small: too many samples per pixel"); return BSCT_ERR_UNSUPPORTED_SIZE; }
  if (bp_gather_smem<double>(bp_window(geom->lambda_y)) > 227 * 1024) {
    bsct_set_last_message("lambda_y too small: detector window does not fit in shared memory");
    return BSCT_ERR_UNSUPPORTED_SIZE;
  }
  return BSCT_OK;
}

extern "C" int bsct_backproject(const bsct_geom* geom, const void* d_sino, void* d_b, int precision, void* d_work,
                                size_t work_bytes, void* stream) {
  int rc = bsct_check_geom(geom);
  if (rc != BSCT_OK) return rc;
  if (!d_sino || !d_b || !d_work) { bsct_set_last_message("NULL device pointer"); return BSCT_ERR_INVALID_ARG; }
  if (precision != BSCT_F32 && precision != BSCT_F64) { bsct_set_last_message("precision"); return BSCT_ERR_INVALID_ARG; }
  rc = bsct_check_bp_geom(geom);
  if (rc != BSCT_OK) return rc;
  if (work_bytes < bp_workspace(geom, precision)) { bsct_set_last_message("workspace too small"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const long ns = (long)geom->n_angles * geom->n_bins;  // non-finite samples set the input status
  double wb[2];
  const bool two = bsct_blur_boxes(geom, wb) == 2;
  if (precision == BSCT_F32) {
    rc = check_finite_async<float>((const float*)d_sino, ns, st);
    if (rc != BSCT_OK) return rc;
    return two ? mb_bp_run<float>(geom, (const float*)d_sino, (float*)d_b, (char*)d_work, st)
               : bp_run<float>(geom, (const float*)d_sino, (float*)d_b, (char*)d_work, st);
  }
  rc = check_finite_async<double>((const double*)d_sino, ns, st);
  if (rc != BSCT_OK) return rc;
  return two ? mb_bp_run<double>(geom, (const double*)d_sino, (double*)d_b, (char*)d_work, st)
             : bp_run<double>(geom, (const double*)d_sino, (double*)d_b, (char*)d_work, st);
}
