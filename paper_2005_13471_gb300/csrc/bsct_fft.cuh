// Block-level Stockham FFT for the Gram-filter convolution (sm_103a).
//
// One FFT of length L is computed by L/E threads, each holding E complex values in
// registers.  A stage of radix R makes every thread run E/R radix-R butterflies on
// its registers; between stages the values are exchanged once through shared
// memory (padded index i + i/16 to spread the stride-R writes over the banks).
// The first stage takes its inputs from registers that the caller filled from HBM
// and the last stage leaves its outputs in registers for the caller to store, so a
// 3-stage 4096-point FFT costs two shared-memory round trips.
//
// Register layout (Stockham autosort, natural order in and out):
//   stage input : v[b*R + r] = x[j + r*L/R],            j = tid + b*(L/E)
//   stage output: y[(j/Ns)*Ns*R + (j%Ns) + r*Ns]          (Ns = product of earlier radices)
//   last output : v[b*R + r] = y[j + r*L/R]
// so running the inverse with the radix order reversed starts from exactly the
// registers the forward transform ended with (no exchange between them).
//
// Twiddles: stage s (Ns = product of earlier radices, radix R) multiplies element r of
// butterfly j by exp(-2 pi i r (j mod Ns) / (Ns R)).  They come from a per-plan table
// laid out [stage][r-1][j mod Ns] (Ns - 1 + (r-1) Ns + j mod Ns; the stages add up to
// L - 1 entries), so consecutive threads read consecutive entries; FP32 radix-8/16
// stages read the powers 1, 2, 4, 8 and multiply out the rest (see stage_compute).
#pragma once
#include "bsct_common.cuh"

namespace bsct {

// ----------------------------------------------------------------------------------
// Radix plans.  E values per thread must be a multiple of every radix used.
// ----------------------------------------------------------------------------------
template <int L> struct Plan;
#define BSCT_PLAN(LEN, EPT, ...)                                                     \
  template <> struct Plan<LEN> {                                                     \
    static constexpr int E = EPT;                                                    \
    static constexpr int R[] = {__VA_ARGS__};                                        \
    static constexpr int NS = sizeof(R) / sizeof(int);                               \
  };
BSCT_PLAN(16, 16, 16)
BSCT_PLAN(32, 16, 16, 2)
BSCT_PLAN(64, 16, 16, 4)
BSCT_PLAN(128, 16, 16, 8)
BSCT_PLAN(256, 16, 16, 16)
BSCT_PLAN(384, 24, 8, 4, 4, 3)
BSCT_PLAN(512, 16, 16, 2, 16)
BSCT_PLAN(768, 24, 8, 8, 4, 3)
BSCT_PLAN(1024, 16, 16, 4, 16)
BSCT_PLAN(1536, 24, 8, 8, 8, 3)
BSCT_PLAN(2048, 16, 16, 8, 16)
BSCT_PLAN(4096, 16, 16, 16, 16)
#undef BSCT_PLAN

// Plans of 512, 1024, 2048 and 4096 points read the same forwards and backwards, so the
// inverse transforms (run with the plan reversed) share the forward stage twiddle table:
// one table per length stays resident in L1 next to the large shared-memory buffers.
template <int L> __host__ __device__ constexpr bool plan_palindrome() {
  for (int i = 0; i < Plan<L>::NS; ++i)
    if (Plan<L>::R[i] != Plan<L>::R[Plan<L>::NS - 1 - i]) return false;
  return true;
}

// radix of stage s (REV = run the plan's radices in reverse order)
template <int L, bool REV> __host__ __device__ constexpr int radix_of(int s) {
  return REV ? Plan<L>::R[Plan<L>::NS - 1 - s] : Plan<L>::R[s];
}
template <int L, bool REV> __host__ __device__ constexpr int ns_of(int s) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= radix_of<L, REV>(i);
  return p;
}

__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }
template <int L> __host__ __device__ constexpr int smem_elems() { return L + L / 16; }

// ----------------------------------------------------------------------------------
// Small DFTs in registers: X[k] = sum_r v[r] w^(rk), w = exp(-+2 pi i / R)
// ----------------------------------------------------------------------------------
template <typename T, bool INV>
__device__ __forceinline__ void dft2(cpx<T>& a, cpx<T>& b) {
  cpx<T> t = a - b;
  a = a + b;
  b = t;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(cpx<T>& v0, cpx<T>& v1, cpx<T>& v2, cpx<T>& v3) {
  cpx<T> a0 = v0 + v2, a1 = v0 - v2, a2 = v1 + v3, a3 = mul_mi<T, INV>(v1 - v3);
  v0 = a0 + a2;
  v2 = a0 - a2;
  v1 = a1 + a3;
  v3 = a1 - a3;
}

// dft4 of (v0, v1, 0, 0): the upper half of the inputs is known to be zero
template <typename T, bool INV>
__device__ __forceinline__ void dft4h(cpx<T>& v0, cpx<T>& v1, cpx<T>& v2, cpx<T>& v3) {
  const cpx<T> a = v0, b = v1, bi = mul_mi<T, INV>(v1);
  v0 = a + b;
  v2 = a - b;
  v1 = a + bi;
  v3 = a - bi;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft3(cpx<T>& a, cpx<T>& b, cpx<T>& c) {
  const T h3 = T(0.86602540378443864676);  // sqrt(3)/2
  cpx<T> t1 = b + c;
  cpx<T> t2 = mk(fma(T(-0.5), t1.x, a.x), fma(T(-0.5), t1.y, a.y));
  cpx<T> t3 = mul_mi<T, INV>(scale(b - c, h3));
  a = a + t1;
  b = t2 + t3;
  c = t2 - t3;
}

// exp(-+2 pi i k / 16) as constants
template <typename T, bool INV> __device__ __forceinline__ cpx<T> w16(int k) {
  const T C1 = T(0.92387953251128675613), S1 = T(0.38268343236508977173), H = T(0.70710678118654752440);
  T c, s;
  switch (k) {
    case 1: c = C1; s = S1; break;
    case 2: c = H; s = H; break;
    case 3: c = S1; s = C1; break;
    case 6: c = -H; s = H; break;
    case 9: c = -C1; s = -S1; break;
    default: c = T(1); s = T(0); break;
  }
  return mk(c, INV ? s : -s);
}

template <typename T, bool INV, bool HALF = false>
__device__ __forceinline__ void dft8(cpx<T>* v) {
  if constexpr (HALF) {
    dft4h<T, INV>(v[0], v[2], v[4], v[6]);
    dft4h<T, INV>(v[1], v[3], v[5], v[7]);
  } else {
    dft4<T, INV>(v[0], v[2], v[4], v[6]);
    dft4<T, INV>(v[1], v[3], v[5], v[7]);
  }
  const T H = T(0.70710678118654752440);
  cpx<T> o0 = v[1];
  cpx<T> o1 = cmul(v[3], mk(H, INV ? H : -H));
  cpx<T> o2 = mul_mi<T, INV>(v[5]);
  cpx<T> o3 = cmul(v[7], mk(-H, INV ? H : -H));
  cpx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  v[0] = e0 + o0; v[4] = e0 - o0;
  v[1] = e1 + o1; v[5] = e1 - o1;
  v[2] = e2 + o2; v[6] = e2 - o2;
  v[3] = e3 + o3; v[7] = e3 - o3;
}

// 16 = 4 x 4: r = r1 + 4 r2, k = k1 + 4 k2
template <typename T, bool INV, bool HALF = false>
__device__ __forceinline__ void dft16(cpx<T>* v) {
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) {
    if constexpr (HALF) dft4h<T, INV>(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
    else dft4<T, INV>(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
  }
  // now v[r1 + 4 k1] = A[r1][k1]; twiddle by w16^(r1 k1)
  v[5] = cmul(v[5], w16<T, INV>(1));
  v[9] = cmul(v[9], w16<T, INV>(2));
  v[13] = cmul(v[13], w16<T, INV>(3));
  v[6] = cmul(v[6], w16<T, INV>(2));
  v[10] = mul_mi<T, INV>(v[10]);
  v[14] = cmul(v[14], w16<T, INV>(6));
  v[7] = cmul(v[7], w16<T, INV>(3));
  v[11] = cmul(v[11], w16<T, INV>(6));
  v[15] = cmul(v[15], w16<T, INV>(9));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<T, INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4 k1 + k2] = X[k1 + 4 k2]: transpose into natural order
  cpx<T> t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}

// HALF: inputs r >= R/2 are zero (zero-padded first stage); needs an even radix
template <int R, typename T, bool INV, bool HALF = false> __device__ __forceinline__ void dft(cpx<T>* v) {
  static_assert(!HALF || R % 2 == 0, "half-zero stage needs an even radix");
  if constexpr (R == 2) { if constexpr (HALF) v[1] = v[0]; else dft2<T, INV>(v[0], v[1]); }
  else if constexpr (R == 3) dft3<T, INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) { if constexpr (HALF) dft4h<T, INV>(v[0], v[1], v[2], v[3]); else dft4<T, INV>(v[0], v[1], v[2], v[3]); }
  else if constexpr (R == 8) dft8<T, INV, HALF>(v);
  else if constexpr (R == 16) dft16<T, INV, HALF>(v);
  else static_assert(R == 2, "unsupported radix");
}

// ----------------------------------------------------------------------------------
// Stages
// ----------------------------------------------------------------------------------
// tws: stage twiddle table of this plan (and radix order), see the top of the file
// Per-thread cache of the base twiddle powers (w^1, w^2, w^4, w^8) of every radix-8/16
// stage of a plan, for persistent kernels that run many FFTs of one length with one
// thread layout: loaded once into registers, their latency leaves the stages.
template <typename T, int L> struct TwCache {
  static constexpr int NB = Plan<L>::E / 8;  // butterflies per thread of a radix-8 stage
  cpx<T> w[Plan<L>::NS][NB][4];
};
template <typename T, int L, bool REV, int S>
__device__ __forceinline__ void tw_cache_stages(TwCache<T, L>& c, int tid, const cpx<T>* __restrict__ tws) {
  constexpr int R = radix_of<L, REV>(S), NSV = ns_of<L, REV>(S), E = Plan<L>::E, TT = L / E;
  if constexpr (NSV > 1 && (R == 8 || R == 16)) {
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const cpx<T>* t = tws + (NSV - 1) + ((tid + b * TT) % NSV);
      c.w[S][b][0] = ld_cpx(t);
      c.w[S][b][1] = ld_cpx(t + NSV);
      c.w[S][b][2] = ld_cpx(t + 3 * NSV);
      if constexpr (R == 16) c.w[S][b][3] = ld_cpx(t + 7 * NSV);
    }
  }
  if constexpr (S + 1 < Plan<L>::NS) tw_cache_stages<T, L, REV, S + 1>(c, tid, tws);
}
template <typename T, int L, bool REV>
__device__ __forceinline__ void tw_cache_load(TwCache<T, L>& c, int tid, const cpx<T>* __restrict__ tws) {
  tw_cache_stages<T, L, REV, 0>(c, tid, tws);
}

// FP32 radix-8 and radix-16 stages load only w^1, w^2, w^4 (and w^8) of their butterfly
// from the table and form the other powers by at most three complex products (a few
// ulps): the table loads compete with the exchanges for the L1 / shared-memory pipe, and
// measured, fewer loads and more FMAs win.  FP64 (the reference-precision path) loads
// every twiddle.
template <typename T, int L, int R, int NSV, bool INV, bool HALF, int S = 0, bool CACHED = false>
__device__ __forceinline__ void stage_compute(cpx<T> (&v)[Plan<L>::E], int tid, const cpx<T>* __restrict__ tws,
                                              const TwCache<T, L>* cache = nullptr) {
  constexpr int E = Plan<L>::E;
  constexpr int TT = L / E;
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    if constexpr (NSV > 1 && (R == 8 || R == 16) && sizeof(T) == 4) {
      const int j = tid + b * TT;
      cpx<T> w[R];
      if constexpr (CACHED) {
        w[1] = cache->w[S][b][0];
        w[2] = cache->w[S][b][1];
        w[4] = cache->w[S][b][2];
        if constexpr (R == 16) w[8] = cache->w[S][b][3];
      } else {
        const cpx<T>* t = tws + (NSV - 1) + (j % NSV);
        w[1] = ld_cpx(t);
        w[2] = ld_cpx(t + NSV);
        w[4] = ld_cpx(t + 3 * NSV);
        if constexpr (R == 16) w[8] = ld_cpx(t + 7 * NSV);
      }
      w[3] = cmul(w[2], w[1]);
      w[5] = cmul(w[4], w[1]);
      w[6] = cmul(w[4], w[2]);
      w[7] = cmul(w[4], w[3]);
      if constexpr (R == 16) {
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) v[b * R + r] = INV ? cmulc(v[b * R + r], w[r]) : cmul(v[b * R + r], w[r]);
    } else if constexpr (NSV > 1) {
      const int j = tid + b * TT;
      const cpx<T>* t = tws + (NSV - 1) + (j % NSV);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const cpx<T> w = ld_cpx(t + (r - 1) * NSV);
        v[b * R + r] = INV ? cmulc(v[b * R + r], w) : cmul(v[b * R + r], w);
      }
    }
    dft<R, T, INV, HALF>(&v[b * R]);
  }
}

template <typename T, int L, int R, int NSV, int R2>
__device__ __forceinline__ void stage_exchange(cpx<T> (&v)[Plan<L>::E], cpx<T>* sm, int tid) {
  constexpr int E = Plan<L>::E;
  constexpr int TT = L / E;
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    const int j = tid + b * TT;
    const int base = (j / NSV) * NSV * R + (j % NSV);
    if constexpr (NSV % 16 == 0) {
      // (base + r NSV) / 16 = base / 16 + r NSV / 16
      const int pb = spad(base);
#pragma unroll
      for (int r = 0; r < R; ++r) sm[pb + r * (NSV + NSV / 16)] = v[b * R + r];
    } else if constexpr (NSV == 1 && 16 % R == 0) {
      // base = j R and r < R <= 16 never crosses a 16-element boundary
      const int pb = spad(base);
#pragma unroll
      for (int r = 0; r < R; ++r) sm[pb + r] = v[b * R + r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) sm[spad(base + r * NSV)] = v[b * R + r];
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < E / R2; ++b) {
    const int j = tid + b * TT;
    if constexpr ((L / R2) % 16 == 0) {
      const int pj = spad(j);
#pragma unroll
      for (int r = 0; r < R2; ++r) v[b * R2 + r] = sm[pj + r * ((L / R2) + (L / R2) / 16)];
    } else {
#pragma unroll
      for (int r = 0; r < R2; ++r) v[b * R2 + r] = sm[spad(j + r * (L / R2))];
    }
  }
  __syncthreads();
}

template <typename T, int L, bool INV, bool REV, bool HALF, int S, bool CACHED>
__device__ __forceinline__ void fft_stages(cpx<T> (&v)[Plan<L>::E], cpx<T>* sm, int tid, const cpx<T>* __restrict__ tws,
                                           const TwCache<T, L>* cache) {
  constexpr int R = radix_of<L, REV>(S);
  constexpr int NSV = ns_of<L, REV>(S);
  stage_compute<T, L, R, NSV, INV, HALF && S == 0, S, CACHED>(v, tid, tws, cache);
  if constexpr (S + 1 < Plan<L>::NS) {
    stage_exchange<T, L, R, NSV, radix_of<L, REV>(S + 1)>(v, sm, tid);
    fft_stages<T, L, INV, REV, HALF, S + 1, CACHED>(v, sm, tid, tws, cache);
  }
}

// Full FFT of one length-L sequence by L/E threads.  On entry v holds the inputs in
// the first-stage layout, on exit the outputs in the last-stage layout (see top).
// sm: this FFT's shared buffer of smem_elems<L>() values; tws: the stage twiddle table
// of (L, REV).  HALF: the upper half of the input sequence is zero (its registers are
// not read).  Unnormalised both ways.
template <typename T, int L, bool INV, bool REV, bool HALF = false>
__device__ __forceinline__ void fft(cpx<T> (&v)[Plan<L>::E], cpx<T>* sm, int tid, const cpx<T>* __restrict__ tws) {
  fft_stages<T, L, INV, REV, HALF, 0, false>(v, sm, tid, tws, nullptr);
}
// Same with the radix-8/16 stage twiddles taken from a register cache filled by
// tw_cache_load for the same plan order (for a palindromic plan the forward cache serves
// the reversed order); stages of other radices still read tws.
template <typename T, int L, bool INV, bool REV, bool HALF = false>
__device__ __forceinline__ void fft_cached(cpx<T> (&v)[Plan<L>::E], cpx<T>* sm, int tid, const cpx<T>* __restrict__ tws,
                                           const TwCache<T, L>& cache) {
  fft_stages<T, L, INV, REV, HALF, 0, true>(v, sm, tid, tws, &cache);
}

// Host-side copy of a plan (for building the stage twiddle tables).
struct PlanInfo {
  int L, ns, R[8];
};
inline bool plan_info(int L, bool rev, PlanInfo* p) {
  auto fill = [&](const int* R, int ns) {
    p->L = L;
    p->ns = ns;
    for (int i = 0; i < ns; ++i) p->R[i] = rev ? R[ns - 1 - i] : R[i];
  };
  switch (L) {
#define BSCT_PI(LEN) case LEN: fill(Plan<LEN>::R, Plan<LEN>::NS); return true;
    BSCT_PI(16) BSCT_PI(32) BSCT_PI(64) BSCT_PI(128) BSCT_PI(256) BSCT_PI(384) BSCT_PI(512)
    BSCT_PI(768) BSCT_PI(1024) BSCT_PI(1536) BSCT_PI(2048) BSCT_PI(4096)
#undef BSCT_PI
    default: return false;
  }
}

}  // namespace bsct
