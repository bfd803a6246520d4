// FP64 evaluation of centred, unit-mass univariate box splines on the GPU (Sec. 3, Eq. 1-2).
//
// A direction list is given as up to 4 groups (value a_g > 0, multiplicity m_g).  Two
// evaluators:
//   box_tp     - the truncated-power expansion of the convolution of Eq. 1,
//                M(x) = sum_k prod_g C(m_g, k_g) (-1)^k_g (x + sum m a / 2 - sum k a)_+^(n-1)
//                       / ((n-1)! prod a_g^m_g),
//                grouped by equal directions (27 terms for the 6-direction Gram kernel).
//                Its terms are ~ (sum a)^(n-1) / prod a while the result is ~ 1 / sum a,
//                so it loses about log10((sum a)^n / prod a) digits when one direction
//                is short (views close to the axes).
//   box_stable - for such lists: one short group S = (s, m_s), m_s in {1, 2}, is split
//                off and M = M_L * M_S is integrated as  int M_L(x - v) M_S(v) dv  over
//                |v| < m_s s / 2 by 3-point Gauss-Legendre on every piece between the
//                kinks of both factors (exact: the integrand is piecewise polynomial of
//                degree <= 5).  M_S is a box (m_s = 1) or a hat (m_s = 2) and M_L has no
//                short direction, so no term cancels.
#pragma once
#include <math.h>

namespace bsct {

struct BoxDirs {
  double a[4];
  int m[4];
  int ng;
};

__host__ __device__ __forceinline__ double ipow(double z, int p) {
  double r = 1.0;
  for (int i = 0; i < p; ++i) r *= z;
  return r;
}

__device__ __forceinline__ int binom4(int m, int k) {
  // C(m, k) for 0 <= k <= m <= 4
  const int tab[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
  return tab[m][k];
}

__device__ inline double box_tp(double x, const BoxDirs& D) {
  int n = 0;
  double tot = 0.0, prod = 1.0;
  for (int g = 0; g < D.ng; ++g) {
    n += D.m[g];
    tot += D.m[g] * D.a[g];
    prod *= ipow(D.a[g], D.m[g]);
  }
  if (n == 0) return 0.0;
  double fact = 1.0;
  for (int i = 2; i < n; ++i) fact *= i;
  const double x0 = x + 0.5 * tot;
  const int m0 = D.ng > 0 ? D.m[0] : 0, m1 = D.ng > 1 ? D.m[1] : 0;
  const int m2 = D.ng > 2 ? D.m[2] : 0, m3 = D.ng > 3 ? D.m[3] : 0;
  double acc = 0.0;
  for (int k0 = 0; k0 <= m0; ++k0)
    for (int k1 = 0; k1 <= m1; ++k1)
      for (int k2 = 0; k2 <= m2; ++k2)
        for (int k3 = 0; k3 <= m3; ++k3) {
          double off = 0.0;
          if (k0) off += k0 * D.a[0];
          if (k1) off += k1 * D.a[1];
          if (k2) off += k2 * D.a[2];
          if (k3) off += k3 * D.a[3];
          const double z = x0 - off;
          if (z <= 0.0) continue;
          const int w = binom4(m0, k0) * binom4(m1, k1) * binom4(m2, k2) * binom4(m3, k3);
          const double term = (n == 1) ? 1.0 : ipow(z, n - 1);
          acc += ((k0 + k1 + k2 + k3) & 1) ? -w * term : w * term;
        }
  return acc / (fact * prod);
}

// kinks (knots) of M_L: -sum/2 + sum_g k_g a_g; at most 3*3*1*5 combinations are used
#define BSCT_MAXKNOTS 48

__device__ inline double box_stable(double x, const BoxDirs& L, double s, int ms) {
  const double half = 0.5 * ms * s;
  // candidate cut points in v: window ends, centre of the hat, x - knot(M_L)
  double cut[BSCT_MAXKNOTS + 3];
  int nc = 0;
  cut[nc++] = -half;
  cut[nc++] = half;
  if (ms == 2) cut[nc++] = 0.0;
  double tot = 0.0;
  for (int g = 0; g < L.ng; ++g) tot += L.m[g] * L.a[g];
  const int m0 = L.ng > 0 ? L.m[0] : 0, m1 = L.ng > 1 ? L.m[1] : 0;
  const int m2 = L.ng > 2 ? L.m[2] : 0, m3 = L.ng > 3 ? L.m[3] : 0;
  for (int k0 = 0; k0 <= m0; ++k0)
    for (int k1 = 0; k1 <= m1; ++k1)
      for (int k2 = 0; k2 <= m2; ++k2)
        for (int k3 = 0; k3 <= m3; ++k3) {
          double knot = -0.5 * tot;
          if (k0) knot += k0 * L.a[0];
          if (k1) knot += k1 * L.a[1];
          if (k2) knot += k2 * L.a[2];
          if (k3) knot += k3 * L.a[3];
          const double v = x - knot;
          if (v > -half && v < half && nc < BSCT_MAXKNOTS + 3) cut[nc++] = v;
        }
  // insertion sort (nc is small)
  for (int i = 1; i < nc; ++i) {
    double t = cut[i];
    int j = i - 1;
    while (j >= 0 && cut[j] > t) { cut[j + 1] = cut[j]; --j; }
    cut[j + 1] = t;
  }
  const double g0 = 0.11270166537925831148, g1 = 0.5, g2 = 0.88729833462074168852;  // (1 -+ sqrt(3/5))/2
  const double w0 = 5.0 / 18.0, w1 = 8.0 / 18.0;
  double acc = 0.0;
  for (int i = 0; i + 1 < nc; ++i) {
    const double lo = cut[i], w = cut[i + 1] - cut[i];
    if (w <= 0.0) continue;
    const double vs[3] = {lo + g0 * w, lo + g1 * w, lo + g2 * w};
    const double ws[3] = {w0, w1, w0};
    double piece = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double v = vs[q];
      const double ms_v = (ms == 1) ? 1.0 / s : (s - fabs(v)) / (s * s);
      piece += ws[q] * ms_v * box_tp(x - v, L);
    }
    acc += piece * w;
  }
  return acc;
}

// Evaluate M_D(x) where group `small` (or -1) is short relative to the others.
__device__ inline double box_eval(double x, const BoxDirs& D, int small) {
  if (small < 0) return box_tp(x, D);
  BoxDirs L;
  L.ng = 0;
  for (int g = 0; g < D.ng; ++g)
    if (g != small) { L.a[L.ng] = D.a[g]; L.m[L.ng] = D.m[g]; ++L.ng; }
  for (int g = L.ng; g < 4; ++g) { L.a[g] = 0.0; L.m[g] = 0; }
  return box_stable(x, L, D.a[small], D.m[small]);
}

// Relative length below which the short direction goes through box_stable.
#define BSCT_SHORT_DIR 0.2

// Kinks of M_D: -sum m a / 2 + sum_g k_g a_g (0 <= k_g <= m_g); returns how many (<= cap).
__device__ inline int box_kinks(const BoxDirs& D, double* out, int cap) {
  double tot = 0.0;
  for (int g = 0; g < D.ng; ++g) tot += D.m[g] * D.a[g];
  const int m0 = D.ng > 0 ? D.m[0] : 0, m1 = D.ng > 1 ? D.m[1] : 0;
  const int m2 = D.ng > 2 ? D.m[2] : 0, m3 = D.ng > 3 ? D.m[3] : 0;
  int n = 0;
  for (int k0 = 0; k0 <= m0; ++k0)
    for (int k1 = 0; k1 <= m1; ++k1)
      for (int k2 = 0; k2 <= m2; ++k2)
        for (int k3 = 0; k3 <= m3; ++k3) {
          double k = -0.5 * tot;
          if (k0) k += k0 * D.a[0];
          if (k1) k += k1 * D.a[1];
          if (k2) k += k2 * D.a[2];
          if (k3) k += k3 * D.a[3];
          if (n < cap) out[n++] = k;
        }
  return n;
}

// Convolution of two box splines, M_[P, Q](x) = int M_P(x - v) M_Q(v) dv, for direction lists
// too long for the truncated-power form (several detector boxes): 4-point Gauss-Legendre on
// every piece between the kinks of both factors inside the overlap of their supports (exact
// for deg M_P + deg M_Q <= 7).  M_P is evaluated with the short-direction split of group
// small_p (or -1), M_Q by truncated powers (its directions - detector boxes and sample
// spacings - are never short).  Both factors are centred and symmetric, so each is evaluated
// at -|argument|, where its truncated powers are smallest.  Every term is non-negative.
#define BSCT_CONV_CUTS 96
__device__ inline double box_conv(double x, const BoxDirs& P, int small_p, const BoxDirs& Q) {
  double cut[BSCT_CONV_CUTS];
  double qt = 0.0, pt = 0.0;
  for (int g = 0; g < Q.ng; ++g) qt += Q.m[g] * Q.a[g];
  for (int g = 0; g < P.ng; ++g) pt += P.m[g] * P.a[g];
  const double lo = fmax(-0.5 * qt, x - 0.5 * pt), hi = fmin(0.5 * qt, x + 0.5 * pt);
  if (!(hi > lo)) return 0.0;
  int nc = 0;
  cut[nc++] = lo;
  cut[nc++] = hi;
  double kq[48], kp[48];
  const int nq = box_kinks(Q, kq, 48), np = box_kinks(P, kp, 48);
  for (int i = 0; i < nq && nc < BSCT_CONV_CUTS; ++i)
    if (kq[i] > lo && kq[i] < hi) cut[nc++] = kq[i];
  for (int i = 0; i < np && nc < BSCT_CONV_CUTS; ++i) {
    const double v = x - kp[i];
    if (v > lo && v < hi) cut[nc++] = v;
  }
  for (int i = 1; i < nc; ++i) {  // insertion sort
    const double t = cut[i];
    int j = i - 1;
    while (j >= 0 && cut[j] > t) { cut[j + 1] = cut[j]; --j; }
    cut[j + 1] = t;
  }
  // Gauss-Legendre, 4 points on [0, 1]
  const double gx[4] = {0.06943184420297371239, 0.33000947820757186760, 0.66999052179242813240,
                        0.93056815579702628761};
  const double gw[4] = {0.17392742256872692869, 0.32607257743127307131, 0.32607257743127307131,
                        0.17392742256872692869};
  double acc = 0.0;
  for (int i = 0; i + 1 < nc; ++i) {
    const double a = cut[i], w = cut[i + 1] - cut[i];
    if (w <= 0.0) continue;
    double piece = 0.0;
    for (int q = 0; q < 4; ++q) {
      const double v = a + gx[q] * w;
      piece += gw[q] * box_eval(-fabs(x - v), P, small_p) * box_tp(-fabs(v), Q);
    }
    acc += piece * w;
  }
  return acc;
}

// cos(pi k (2i + 1) / (2 NC)) for k, i < NC at entry NC k + i: the Chebyshev nodes (k = 1)
// and the cosines of the discrete Chebyshev transform, formed once by the threads of a CTA
// (the caller synchronises before reading them)
template <int NC>
__device__ inline void cheb_cos_fill(double* t) {
  for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) t[e] = cospi((e / NC) * (2.0 * (e % NC) + 1.0) / (2.0 * NC));
}

// Monomial coefficients c[0..7] (in v on [-1, 1]) of the polynomial of degree <= 7 through
// the values fv[i] at the Chebyshev nodes cos(pi (2i + 1) / 16): the discrete Chebyshev
// transform, then T_0..T_7 written out in powers of v.  ck: cheb_cos_fill<8>.
__device__ inline void cheb8_monomials(const double fv[8], double c[8], const double* ck) {
  double ch[8];
  for (int k = 0; k < 8; ++k) {
    double acc = 0.0;
    for (int i = 0; i < 8; ++i) acc += fv[i] * ck[8 * k + i];
    ch[k] = acc * (k == 0 ? 1.0 / 8.0 : 2.0 / 8.0);
  }
  c[0] = ch[0] - ch[2] + ch[4] - ch[6];
  c[1] = ch[1] - 3.0 * ch[3] + 5.0 * ch[5] - 7.0 * ch[7];
  c[2] = 2.0 * ch[2] - 8.0 * ch[4] + 18.0 * ch[6];
  c[3] = 4.0 * ch[3] - 20.0 * ch[5] + 56.0 * ch[7];
  c[4] = 8.0 * ch[4] - 48.0 * ch[6];
  c[5] = 16.0 * ch[5] - 112.0 * ch[7];
  c[6] = 32.0 * ch[6];
  c[7] = 64.0 * ch[7];
}

// ---------------------------------------------------------------------------------------
// Footprint of one view with two detector boxes, h = M_[A, B, w1, w2] (A, B = |cos|, |sin|),
// as exact cubic pieces between its kinks -W/2 + k0 A + k1 B + k2 w1 + k3 w2 (W = A + B +
// w1 + w2; <= 15 pieces).  Each piece is fitted by Chebyshev interpolation at 4 nodes of
// FP64 values of box_conv(M_[A, B], M_[w1, w2]) (short-direction split near the axes), which
// reproduces the cubic exactly up to rounding.  Held in shared memory by one CTA, it turns
// the kernels built on h into single convolutions of piecewise polynomials:
//   back projection  lambda M_[A, B, w1, w2, lambda x (d+1)] = lambda (h * beta_d),
//   Gram kernel      M_[A, A, B, B, w1, w1, w2, w2]          = h * h   (h is even),
// integrated exactly by 4-point Gauss-Legendre between the kinks of both factors
// (degree <= 3 + 3).
struct FootPoly {
  int K;               // pieces
  double hw;           // half support W / 2
  double kn[17];       // piece starts, kn[K] = W / 2
  double mid[16], ihw[16];
  double c[16][4];     // monomials in v = (x - mid) * ihw
  double fv[16][4];    // node values while building
};

__device__ inline double foot_box_conv(double x, double A, double B, double w1, double w2) {
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
  return box_conv(x, P, small, Q);
}

// Built by all threads of a CTA (contains barriers).
__device__ inline void foot_build(FootPoly& F, double A, double B, double w1, double w2, double merge_tol) {
  __shared__ double ck[16];
  cheb_cos_fill<4>(ck);
  if (threadIdx.x == 0) {
    const double W = A + B + w1 + w2;
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
    int m = 1;  // merge kinks closer than merge_tol (the ends -W/2 and W/2 stay)
    for (int i = 1; i < n; ++i)
      if (k[i] - k[m - 1] > merge_tol) k[m++] = k[i];
      else if (i == n - 1) k[m - 1] = k[i];
    for (int i = 0; i < 17; ++i) F.kn[i] = i < m ? k[i] : 1e300;
    F.K = m - 1;
    F.hw = 0.5 * W;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < F.K * 4; it += blockDim.x) {
    const int q = it >> 2, i = it & 3;
    const double mid = 0.5 * (F.kn[q] + F.kn[q + 1]), hw = 0.5 * (F.kn[q + 1] - F.kn[q]);
    F.fv[q][i] = foot_box_conv(mid + hw * ck[4 + i], A, B, w1, w2);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < F.K; q += blockDim.x) {
    double ch[4];
    for (int k = 0; k < 4; ++k) {
      double acc = 0.0;
      for (int i = 0; i < 4; ++i) acc += F.fv[q][i] * ck[4 * k + i];
      ch[k] = acc * (k == 0 ? 0.25 : 0.5);
    }
    // T0 = 1, T1 = v, T2 = 2v^2 - 1, T3 = 4v^3 - 3v
    F.c[q][0] = ch[0] - ch[2];
    F.c[q][1] = ch[1] - 3.0 * ch[3];
    F.c[q][2] = 2.0 * ch[2];
    F.c[q][3] = 4.0 * ch[3];
    F.mid[q] = 0.5 * (F.kn[q] + F.kn[q + 1]);
    F.ihw[q] = 2.0 / (F.kn[q + 1] - F.kn[q]);
  }
  __syncthreads();
}

__device__ inline int foot_piece(const FootPoly& F, double x) {
  int q = 0;
  for (int step = 8; step > 0; step >>= 1)
    if (q + step < F.K && F.kn[q + step] <= x) q += step;
  return q;
}
__device__ inline double foot_piece_eval(const FootPoly& F, int q, double x) {
  const double v = (x - F.mid[q]) * F.ihw[q];
  return fma(fma(fma(F.c[q][3], v, F.c[q][2]), v, F.c[q][1]), v, F.c[q][0]);
}
__device__ inline double foot_eval(const FootPoly& F, double x) {
  if (!(x > -F.hw && x < F.hw)) return 0.0;
  return foot_piece_eval(F, foot_piece(F, x), x);
}

// int h(x - v) g(v) dv for g supported on [glo, ghi] with kinks gk[0..ng) there; g(v) by
// the functor.  Cuts at the kinks of both factors inside the overlap of the supports; on
// every interval h(x - v) is one piece (found at the interval's midpoint) and g one
// polynomial, so 4-point Gauss-Legendre is exact for total degree <= 7.
template <typename G>
__device__ inline double foot_conv(const FootPoly& F, double x, double glo, double ghi, const double* gk, int ng,
                                   G g) {
  const double lo = fmax(glo, x - F.hw), hi = fmin(ghi, x + F.hw);
  if (!(hi > lo)) return 0.0;
  double cut[40];
  int nc = 0;
  cut[nc++] = lo;
  cut[nc++] = hi;
  for (int i = 0; i < ng && nc < 40; ++i)
    if (gk[i] > lo && gk[i] < hi) cut[nc++] = gk[i];
  for (int i = 0; i <= F.K && nc < 40; ++i) {
    const double v = x - F.kn[i];
    if (v > lo && v < hi) cut[nc++] = v;
  }
  for (int i = 1; i < nc; ++i) {  // insertion sort
    const double t = cut[i];
    int j = i - 1;
    while (j >= 0 && cut[j] > t) { cut[j + 1] = cut[j]; --j; }
    cut[j + 1] = t;
  }
  const double gx[4] = {0.06943184420297371239, 0.33000947820757186760, 0.66999052179242813240,
                        0.93056815579702628761};
  const double gw[4] = {0.17392742256872692869, 0.32607257743127307131, 0.32607257743127307131,
                        0.17392742256872692869};
  double acc = 0.0;
  for (int i = 0; i + 1 < nc; ++i) {
    const double a = cut[i], w = cut[i + 1] - cut[i];
    if (w <= 0.0) continue;
    const int q = foot_piece(F, x - (a + 0.5 * w));
    double piece = 0.0;
    for (int k = 0; k < 4; ++k) {
      const double v = a + gx[k] * w;
      piece += gw[k] * foot_piece_eval(F, q, x - v) * g(v);
    }
    acc += piece * w;
  }
  return acc;
}

}  // namespace bsct
