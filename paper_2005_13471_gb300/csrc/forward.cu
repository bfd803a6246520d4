// Forward projection g_s = S H c (Sec. 2, Eq. 3-4): detector samples of the blurred
// X-ray transform of the pixel-basis image,
//
//   g_s[theta, m] = sum_k c_k h_theta(y_m - x_k . u_theta),   h_theta = M_[|cos|, |sin|, zeta],
//
// the footprint of one unit pixel: its projection (the box spline with directions
// |cos theta|, |sin theta|, Eq. 3) averaged over the detector cell (one more direction
// zeta, Eq. 4).
//
// Design.  One thread per (view, detector sample) walks the lines of the image along
// the view's major axis (rows when |cos| >= |sin|, else columns, read from a transposed
// copy so that both cases read along contiguous memory).  On a line the sample's
// footprint covers a few consecutive pixels whose offsets from the sample, in pixel
// units along the line, are delta = f + r: f in [0, 1) is the same for all of them and
// r runs over a handful of integers.  h is piecewise polynomial of degree <= 2, and its
// kinks cut [0, 1) into at most 9 intervals of f; on each interval and for each r,
// h(|major| (f + r)) is ONE polynomial of f.  A per-view table of those polynomials
// (built in FP64 from the footprint's piecewise-linear factor, without cancelling
// terms) leaves per pixel one table read, two FMAs of Horner, the pixel load and the
// accumulate.  Once per line: the interval of f, from a 64-cell lookup whose entries
// carry the interval and its next two starts (one shared load and two comparisons), and
// two comparisons that skip the first and last offsets when they fall outside the
// support.  The table's rows are padded to 36 floats so that lanes in different
// intervals read different banks.
//
// FP32 path: the line coordinate kappa = alpha - k beta (alpha per sample, beta per
// view) reaches ~2N, where an FP32 rounding would move the footprint by ~1e-4 pixel; it
// is kept in 64-bit fixed point instead (40 fractional bits), which makes each line's
// step an exact integer subtraction and leaves f accurate to 2^-23 whatever N.
#include <cmath>

#include "bsct_internal.h"

namespace bsct {

constexpr int FP_IMAX = 9;       // intervals of f per view (<= 8 kinks)
constexpr int FP_RMAX = 8;       // integer offsets r per (sample, line): zeta <= 4
constexpr int FP_FSTART = 16;    // interval starts, padded
constexpr int FP_LUT = 64;       // cells of the interval lookup, 4 T entries each
constexpr int FP_TAB = FP_FSTART + FP_IMAX * FP_RMAX * 4 + FP_LUT * 4;  // T entries per view
constexpr int FP_HDR = 12;       // doubles per view
constexpr int FP_PS = FP_RMAX + 1;  // shared-memory stride of a table row: rows of 36 floats
                                    // put lanes in different intervals on different banks
constexpr int FP_THREADS = 256;
constexpr double FP_ZETA_MAX = 4.0;

enum { FH_ALPHA0 = 0, FH_GAMMA = 1, FH_BETA = 2, FH_MODE = 3, FH_RLO = 4, FH_R = 5, FH_NI = 6, FH_OPEN = 7,
       FH_LUT = 8, FH_IBETA = 9, FH_PHILO = 10, FH_PHIHI = 11 };

// The footprint's factor M_[A, zeta] (zeta > 0: trapezoid; zeta = 0: box of width A) as
// linear pieces a_p + b_p v between sorted kinks e[0..nk).
struct Lin {
  int nk;
  double e[4];
  double a[5], b[5];
  __device__ void init(double A, double zeta) {
    for (int p = 0; p < 5; ++p) { a[p] = 0.0; b[p] = 0.0; }
    if (zeta > 0.0) {
      const double lo = 0.5 * (A + zeta), in = 0.5 * fabs(A - zeta), inv = 1.0 / (A * zeta);
      nk = 4;
      e[0] = -lo; e[1] = -in; e[2] = in; e[3] = lo;
      a[1] = lo * inv;  b[1] = inv;                  // rising: (v + lo) / (A zeta)
      a[2] = 1.0 / fmax(A, zeta);                    // plateau
      a[3] = lo * inv;  b[3] = -inv;                 // falling: (lo - v) / (A zeta)
    } else {
      nk = 2;
      e[0] = -0.5 * A; e[1] = 0.5 * A; e[2] = e[3] = 0.0;
      a[1] = 1.0 / A;
    }
  }
  __device__ int piece(double v) const {
    int p = 0;
    for (int i = 0; i < nk; ++i) p += (e[i] <= v);
    return p;
  }
  __device__ double val(int p, double v) const { return a[p] + b[p] * v; }
  // exact integral over [lo, hi] (linear pieces: length x midpoint value)
  __device__ double integral(double lo, double hi) const {
    double s = 0.0;
    for (int p = 0; p <= nk; ++p) {
      const double pl = p == 0 ? lo : fmax(lo, e[p - 1]);
      const double ph = p == nk ? hi : fmin(hi, e[p]);
      if (ph > pl) s += (ph - pl) * (a[p] + b[p] * 0.5 * (pl + ph));
    }
    return s;
  }
};

__device__ __forceinline__ void cos_sin_pi(double a, double* c, double* s) {
  // exact values on multiples of half a turn / 2 (axis-aligned views), sincospi elsewhere
  a = a - 2.0 * floor(0.5 * a);  // [0, 2)
  const double two = 2.0 * a;
  if (two == rint(two)) {
    const int q = ((int)rint(two)) & 3;
    const double ct[4] = {1.0, 0.0, -1.0, 0.0}, st[4] = {0.0, 1.0, 0.0, -1.0};
    *c = ct[q];
    *s = st[q];
  } else {
    sincospi(a, s, c);
  }
}

// Per-view header and polynomial table (one block per view).
template <typename T>
__global__ void k_fp_tables(const double* __restrict__ ang, int N, int M, double lam, double zeta,
                            double* __restrict__ hdr, T* __restrict__ tab) {
  const int v = blockIdx.x;
  __shared__ double s_f[FP_IMAX];
  __shared__ double s_A, s_B;
  __shared__ int s_ni, s_rlo, s_R;
  if (threadIdx.x == 0) {
    double c, s;
    cos_sin_pi(ang[v], &c, &s);
    const bool rows = fabs(c) >= fabs(s);
    const double major = rows ? c : s, minor = rows ? s : c;
    const double A = fabs(major), B = fabs(minor);
    const double half = 0.5 * (N - 1);
    const double y0 = -0.5 * (M - 1) * lam;
    double* h = hdr + (long)v * FP_HDR;
    h[FH_ALPHA0] = (y0 + half * minor) / major + half;
    h[FH_GAMMA] = lam / major;
    h[FH_BETA] = minor / major;
    h[FH_IBETA] = minor != 0.0 ? major / minor : 0.0;
    h[FH_MODE] = rows ? 0.0 : 1.0;
    // kinks of h = M_[A, zeta] * box_B, in units of A, reduced to [0, 1)
    Lin L;
    L.init(A, zeta);
    double fr[8];
    int n = 0;
    for (int i = 0; i < L.nk; ++i) {
      if (B > 0.0) {
        fr[n++] = (L.e[i] - 0.5 * B) / A;
        fr[n++] = (L.e[i] + 0.5 * B) / A;
      } else {
        fr[n++] = L.e[i] / A;
      }
    }
    for (int i = 0; i < n; ++i) fr[i] -= floor(fr[i]);
    for (int i = 1; i < n; ++i)  // insertion sort
      for (int j = i; j > 0 && fr[j - 1] > fr[j]; --j) { const double t = fr[j]; fr[j] = fr[j - 1]; fr[j - 1] = t; }
    int ni = 1;
    s_f[0] = 0.0;
    for (int i = 0; i < n; ++i)
      if (fr[i] > s_f[ni - 1]) s_f[ni++] = fr[i];
    const double D = (A + B + zeta) / (2.0 * A);  // |delta| < D on the support
    const int rlo = (int)floor(-D), rhi = (int)floor(D);
    int R = rhi - rlo + 1;
    if (R > FP_RMAX) R = FP_RMAX;  // excluded on the host (zeta <= 4)
    s_ni = ni;
    s_rlo = rlo;
    s_R = R;
    s_A = A;
    s_B = B;
    h[FH_RLO] = rlo;
    // the first offset (r = rlo) is inside the support only for f > -D - rlo, the last
    // (r = rhi) only for f < D - rhi; the ones between always are
    h[FH_PHILO] = -D - rlo;
    h[FH_PHIHI] = D - rhi;
    h[FH_R] = R;
    h[FH_NI] = ni;
    h[FH_OPEN] = (B == 0.0 && zeta == 0.0) ? 1.0 : 0.0;
    // interval lookup on the starts as the gather kernel sees them (rounded to T):
    // cell c of [0, 1) holds (I, s_I, s_I+1, s_I+2) for the interval I holding c / FP_LUT
    // and the next two starts (2 past the last), so one load and two comparisons find
    // the interval of any f in the cell - unless some cell holds more than two starts,
    // when the gather searches them all.  For FP32, I is stored as the bit pattern of
    // the integer I * FP_PS (the interval's row in the shared table)
    T* lut = tab + (long)v * FP_TAB + FP_FSTART + FP_IMAX * FP_RMAX * 4;
    auto start = [&](int i) { return i < ni ? T(s_f[i]) : T(2); };
    bool ok = true;
    for (int c = 0; c < FP_LUT; ++c) {
      const double lo = (double)c / FP_LUT, hi = (double)(c + 1) / FP_LUT;
      int I = 0, inside = 0;
      for (int i = 1; i < ni; ++i) {
        const double st = (double)T(s_f[i]);
        I += st <= lo;
        inside += (st > lo && st < hi);
      }
      if constexpr (sizeof(T) == 4) lut[4 * c] = __int_as_float(I * FP_PS);
      else lut[4 * c] = T(I);
      lut[4 * c + 1] = start(I);
      lut[4 * c + 2] = start(I + 1);
      lut[4 * c + 3] = start(I + 2);
      ok = ok && inside <= 2;
    }
    h[FH_LUT] = ok ? 1.0 : 0.0;
  }
  __syncthreads();
  T* tv = tab + (long)v * FP_TAB;
  for (int i = threadIdx.x; i < FP_FSTART; i += blockDim.x) tv[i] = i < s_ni ? T(s_f[i]) : T(2);
  const double A = s_A, B = s_B;
  Lin L;
  L.init(A, zeta);
  for (int i = threadIdx.x; i < FP_IMAX * FP_RMAX; i += blockDim.x) {
    const int I = i / FP_RMAX, rr = i % FP_RMAX;
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    if (I < s_ni && rr < s_R) {
      const double r = (double)(s_rlo + rr);
      const double f0 = s_f[I], f1 = I + 1 < s_ni ? s_f[I + 1] : 1.0;
      const double u0 = A * (f0 + r), um = A * (0.5 * (f0 + f1) + r);
      if (B == 0.0) {
        const int p = L.piece(um);
        c0 = L.val(p, u0);
        c1 = L.b[p];
      } else {
        // h(u) = (1/B) int_{u - B/2}^{u + B/2} M(v) dv; on this interval the window's
        // ends stay inside fixed pieces pL, pR of M
        const int pL = L.piece(um - 0.5 * B), pR = L.piece(um + 0.5 * B);
        c0 = L.integral(u0 - 0.5 * B, u0 + 0.5 * B) / B;
        if (pL == pR) {
          c1 = L.b[pL];
        } else {
          c1 = (L.val(pR, u0 + 0.5 * B) - L.val(pL, u0 - 0.5 * B)) / B;
          c2 = (L.b[pR] - L.b[pL]) / (2.0 * B);
        }
      }
      c1 *= A;  // polynomial in t = f - f0 (u - u0 = A t)
      c2 *= A * A;
    }
    T* p = tv + FP_FSTART + 4 * i;
    p[0] = T(c0);
    p[1] = T(c1);
    p[2] = T(c2);
    p[3] = T(0);
  }
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 t; };
template <> struct Vec4<double> { typedef double4_32a t; };

// one thread per (sample m, view blockIdx.y); lines of the image along the major axis
template <typename T>
__global__ void __launch_bounds__(FP_THREADS) k_fp_gather(const T* __restrict__ img, const T* __restrict__ imgT,
                                                          const double* __restrict__ hdr, const T* __restrict__ tab,
                                                          int N, int M, T* __restrict__ sino) {
  typedef typename Vec4<T>::t V4;
  const int v = blockIdx.y;
  __shared__ T s_f[FP_FSTART];
  __shared__ V4 s_p[FP_IMAX * FP_PS];
  __shared__ V4 s_lut[FP_LUT];
  const T* tv = tab + (long)v * FP_TAB;
  if (threadIdx.x < FP_FSTART) s_f[threadIdx.x] = tv[threadIdx.x];
  if (threadIdx.x < FP_IMAX * FP_RMAX)
    s_p[(threadIdx.x / FP_RMAX) * FP_PS + threadIdx.x % FP_RMAX] = reinterpret_cast<const V4*>(tv + FP_FSTART)[threadIdx.x];
  if (threadIdx.x < FP_LUT) s_lut[threadIdx.x] = reinterpret_cast<const V4*>(tv + FP_FSTART + FP_IMAX * FP_RMAX * 4)[threadIdx.x];
  const double* h = hdr + (long)v * FP_HDR;
  const double alpha0 = h[FH_ALPHA0], gamma = h[FH_GAMMA], beta = h[FH_BETA], ibeta = h[FH_IBETA];
  const int rlo = (int)h[FH_RLO], R = (int)h[FH_R];
  const bool open_box = h[FH_OPEN] != 0.0, lut_ok = h[FH_LUT] != 0.0;
  const T phi_lo = (T)h[FH_PHILO], phi_hi = (T)h[FH_PHIHI];
  const T* src = h[FH_MODE] == 0.0 ? img : imgT;
  __syncthreads();
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const double alpha = alpha0 + (double)m * gamma;
  // lines whose kappa = alpha - k beta lies in [rlo, N + rlo + R): the others touch no pixel
  const double klo = (double)rlo, khi = (double)(N + rlo + R);
  // (bounds widened by one line: 1 / beta is rounded)
  double lo = 0.0, hi = (double)(N - 1);
  if (beta > 0.0) {
    lo = fmax(lo, floor((alpha - khi) * ibeta) - 1.0);
    hi = fmin(hi, ceil((alpha - klo) * ibeta) + 1.0);
  } else if (beta < 0.0) {
    lo = fmax(lo, floor((alpha - klo) * ibeta) - 1.0);
    hi = fmin(hi, ceil((alpha - khi) * ibeta) + 1.0);
  } else if (!(alpha >= klo && alpha < khi)) {
    hi = -1.0;
  }
  const int k0 = (int)lo, k1 = hi < lo ? -1 : (int)hi;  // both clamped to [0, N - 1] first
  T acc = T(0);
  if constexpr (sizeof(T) == 4) {
    // kappa in fixed point with 40 fractional bits (alpha and beta are doubles whose last
    // bit is worth at most 2^-40 here, so the conversion is exact): the per-line step is
    // one 64-bit subtraction, the pixel index is the integer part, and f (its top 23
    // fraction bits) and the lookup cell come from the fraction bits with no conversion
    const double two40 = 1099511627776.0;
    const long long bfx = llrint(beta * two40);
    long long kfx = llrint(alpha * two40) - (long long)k0 * bfx;
    const long long half = 1LL << 39, fmask = (1LL << 40) - 1;
#pragma unroll 2
    for (int k = k0; k <= k1; ++k, kfx -= bfx) {
      if (open_box && (kfx & fmask) == half) continue;  // a sample exactly on a pixel edge of the box
      const int K = (int)(kfx >> 40);
      const unsigned fr = (unsigned)(kfx >> 8);  // fraction bits 2^-1 .. 2^-32
      const float f = __int_as_float(0x3f800000u | (fr >> 9)) - 1.0f;
      int Ir;    // the interval's row offset in s_p
      float t;   // f - (start of the interval)
      if (lut_ok) {
        const float4 L = s_lut[fr >> 26];  // cell floor(64 f)
        const bool g1 = L.z <= f, g2 = L.w <= f;
        Ir = __float_as_int(L.x) + (g1 ? FP_PS : 0) + (g2 ? FP_PS : 0);
        t = f - (g2 ? L.w : (g1 ? L.z : L.y));
      } else {
        int I = 0;
#pragma unroll
        for (int i = 1; i < FP_IMAX; ++i) I += (s_f[i] <= f);
        Ir = I * FP_PS;
        t = f - s_f[I];
      }
      const int kb = K - rlo;
      const float* lp = src + (k * N + kb);  // pixel kb - rr of the line at lp[-rr] (N^2 < 2^31)
      const float4* pr = s_p + Ir;
      // offsets outside the footprint's support are skipped (their table rows are zero)
      const bool first = f > phi_lo, last = f < phi_hi;
      if (kb >= R - 1 && kb < N) {  // all R pixels inside the line
        if (first) {
          const float4 p = pr[0];
          acc = fmaf(__ldg(lp), fmaf(fmaf(p.z, t, p.y), t, p.x), acc);
        }
#pragma unroll
        for (int rr = 1; rr < FP_RMAX - 1; ++rr) {
          if (rr >= R - 1) break;
          const float4 p = pr[rr];
          acc = fmaf(__ldg(lp - rr), fmaf(fmaf(p.z, t, p.y), t, p.x), acc);
        }
        if (last) {
          const float4 p = pr[R - 1];
          acc = fmaf(__ldg(lp - (R - 1)), fmaf(fmaf(p.z, t, p.y), t, p.x), acc);
        }
      } else {
#pragma unroll
        for (int rr = 0; rr < FP_RMAX; ++rr) {
          if (rr >= R) break;
          if ((unsigned)(kb - rr) < (unsigned)N && (rr > 0 || first) && (rr < R - 1 || last)) {
            const float4 p = pr[rr];
            acc = fmaf(__ldg(lp - rr), fmaf(fmaf(p.z, t, p.y), t, p.x), acc);
          }
        }
      }
    }
  } else {
    for (int k = k0; k <= k1; ++k) {
      const double kap = fma(-(double)k, beta, alpha);
      double K = floor(kap);
      double f = kap - K;
      if (open_box && f == 0.5) continue;
      int I;
      if (lut_ok) {
        const double4_32a L = s_lut[min((int)(f * (double)FP_LUT), FP_LUT - 1)];
        I = (int)L.x + (L.z <= f) + (L.w <= f);
      } else {
        I = 0;
#pragma unroll
        for (int i = 1; i < FP_IMAX; ++i) I += (s_f[i] <= f);
      }
      const double t = f - s_f[I];
      const double* line = src + (long)k * N;
      const int kb = (int)K - rlo;
#pragma unroll
      for (int rr = 0; rr < FP_RMAX; ++rr) {
        if (rr >= R) break;
        const int j = kb - rr;
        if ((unsigned)j < (unsigned)N) {
          const double4_32a p = s_p[I * FP_PS + rr];
          acc = fma(line[j], fma(fma(p.z, t, p.y), t, p.x), acc);
        }
      }
    }
  }
  sino[(long)v * M + m] = acc;
}

template <typename T>
__global__ void k_fp_transpose(const T* __restrict__ a, int N, T* __restrict__ at) {
  __shared__ T tile[32][33];
  const int x = blockIdx.x * 32 + threadIdx.x;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int y = blockIdx.y * 32 + j;
    if (x < N && y < N) tile[j][threadIdx.x] = a[(long)y * N + x];
  }
  __syncthreads();
  const int xo = blockIdx.y * 32 + threadIdx.x;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int yo = blockIdx.x * 32 + j;
    if (xo < N && yo < N) at[(long)yo * N + xo] = tile[threadIdx.x][j];
  }
}

}  // namespace bsct

using namespace bsct;

int bsct_check_geom(const bsct_geom* g);

static size_t fp_al(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t fp_workspace(const bsct_geom* g, int precision) {
  double wb[2];
  if (bsct_blur_boxes(g, wb) == 2) return mb_fp_workspace(g, precision);
  const size_t T = precision == BSCT_F32 ? 4 : 8;
  return fp_al((size_t)g->n_angles * sizeof(double)) + fp_al((size_t)g->n_angles * FP_HDR * sizeof(double)) +
         fp_al((size_t)g->n_angles * FP_TAB * T) + fp_al((size_t)g->N * g->N * T);
}

static int fp_check(const bsct_geom* geom, int precision) {
  int rc = bsct_check_geom(geom);
  if (rc != BSCT_OK) return rc;
  if (precision != BSCT_F32 && precision != BSCT_F64) { bsct_set_last_message("precision"); return BSCT_ERR_INVALID_ARG; }
  if (geom->N < 1 || geom->N > 16384) { bsct_set_last_message("forward projection: N outside [1, 16384]"); return BSCT_ERR_UNSUPPORTED_SIZE; }
  if ((long long)geom->n_angles * geom->n_bins > (1LL << 31) - 1) {
    bsct_set_last_message("forward projection: n_angles x n_bins >= 2^31");
    return BSCT_ERR_UNSUPPORTED_SIZE;
  }
  if (geom->zeta_blur > FP_ZETA_MAX) {
    bsct_set_last_message("forward projection: zeta_blur > 4 is not supported");
    return BSCT_ERR_UNSUPPORTED_SIZE;
  }
  return BSCT_OK;
}

extern "C" int bsct_forward_project_workspace(const bsct_geom* geom, int precision, size_t* bytes) {
  int rc = fp_check(geom, precision);
  if (rc != BSCT_OK) return rc;
  if (!bytes) { bsct_set_last_message("bytes is NULL"); return BSCT_ERR_INVALID_ARG; }
  *bytes = fp_workspace(geom, precision);
  return BSCT_OK;
}

template <typename T>
static int fp_run(const bsct_geom* geom, const T* c, T* sino, char* w, cudaStream_t st) {
  const int N = geom->N, M = geom->n_bins, na = geom->n_angles;
  double* ang = (double*)w;
  w += fp_al((size_t)na * sizeof(double));
  double* hdr = (double*)w;
  w += fp_al((size_t)na * FP_HDR * sizeof(double));
  T* tab = (T*)w;
  w += fp_al((size_t)na * FP_TAB * sizeof(T));
  T* ct = (T*)w;
  BSCT_CUDA_TRY(cudaMemcpyAsync(ang, geom->angles_pi, (size_t)na * sizeof(double), cudaMemcpyHostToDevice, st));
  double wb[2];
  bsct_blur_boxes(geom, wb);  // one box (or none) here
  k_fp_tables<T><<<na, 128, 0, st>>>(ang, N, M, geom->lambda_y, wb[0], hdr, tab);
  dim3 tb(32, 8), tg((N + 31) / 32, (N + 31) / 32);
  k_fp_transpose<T><<<tg, tb, 0, st>>>(c, N, ct);
  dim3 gg((M + FP_THREADS - 1) / FP_THREADS, na);
  k_fp_gather<T><<<gg, FP_THREADS, 0, st>>>(c, ct, hdr, tab, N, M, sino);
  count_launch(3);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

extern "C" int bsct_forward_project(const bsct_geom* geom, const void* d_coeffs, void* d_sino, int precision,
                                    void* d_work, size_t work_bytes, void* stream) {
  int rc = fp_check(geom, precision);
  if (rc != BSCT_OK) return rc;
  if (!d_coeffs || !d_sino || !d_work) { bsct_set_last_message("NULL device pointer"); return BSCT_ERR_INVALID_ARG; }
  if (work_bytes < fp_workspace(geom, precision)) { bsct_set_last_message("workspace too small"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const long nc = (long)geom->N * geom->N;  // non-finite coefficients set the input status
  double wb[2];
  const bool two = bsct_blur_boxes(geom, wb) == 2;
  if (precision == BSCT_F32) {
    rc = check_finite_async<float>((const float*)d_coeffs, nc, st);
    if (rc != BSCT_OK) return rc;
    return two ? mb_fp_run<float>(geom, (const float*)d_coeffs, (float*)d_sino, (char*)d_work, st)
               : fp_run<float>(geom, (const float*)d_coeffs, (float*)d_sino, (char*)d_work, st);
  }
  rc = check_finite_async<double>((const double*)d_coeffs, nc, st);
  if (rc != BSCT_OK) return rc;
  return two ? mb_fp_run<double>(geom, (const double*)d_coeffs, (double*)d_sino, (char*)d_work, st)
             : fp_run<double>(geom, (const double*)d_coeffs, (double*)d_sino, (char*)d_work, st);
}
