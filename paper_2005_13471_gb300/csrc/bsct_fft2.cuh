// Paired FP32 Stockham FFT: two independent sequences transformed side by side with the
// packed FP32 instructions of sm_100+ (add / mul / fma on float2 register pairs).
//
// A value c2 holds element k of sequence 0 in the .x lanes and element k of sequence 1 in
// the .y lanes of its real and imaginary parts (structure of arrays), so every complex
// add, subtraction and product of a butterfly is one packed instruction for both
// sequences; negated operands and a scalar twiddle broadcast to both lanes are operand
// modifiers of those instructions, not extra instructions.  The two sequences share one
// plan and one set of twiddles (Plan, radix order, thread layout and stage tables of
// bsct_fft.cuh), so the twiddles stay scalar and are computed once for both.
//
// Shared-memory exchanges move 16-byte values (both sequences at once) with the padding of
// bsct_fft.cuh (index i + i / 16), which keeps a quarter warp on distinct banks for every
// stage pattern of the plans.
#pragma once
#include "bsct_fft.cuh"

namespace bsct {

struct c2 {
  float2 re, im;
};

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ c2 operator+(c2 a, c2 b) { return c2{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ c2 operator-(c2 a, c2 b) { return c2{sub2(a.re, b.re), sub2(a.im, b.im)}; }
__device__ __forceinline__ c2 c2zero() { return c2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
// (a0, a1), (b0, b1) as the two sequences' values
__device__ __forceinline__ c2 c2pack(cpx<float> a, cpx<float> b) {
  return c2{make_float2(a.x, b.x), make_float2(a.y, b.y)};
}
__device__ __forceinline__ cpx<float> c2lane0(c2 v) { return mk(v.re.x, v.im.x); }
__device__ __forceinline__ cpx<float> c2lane1(c2 v) { return mk(v.re.y, v.im.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ c2 mul_mi2(c2 a) {
  return INV ? c2{neg2(a.im), a.re} : c2{a.im, neg2(a.re)};
}
// a * w and a * conj(w) for a scalar twiddle w used by both sequences
__device__ __forceinline__ c2 cmul2(c2 a, cpx<float> w) {
  return c2{fma2(a.re, bc2(w.x), mul2(a.im, bc2(-w.y))), fma2(a.im, bc2(w.x), mul2(a.re, bc2(w.y)))};
}
__device__ __forceinline__ c2 cmulc2(c2 a, cpx<float> w) {
  return c2{fma2(a.re, bc2(w.x), mul2(a.im, bc2(w.y))), fma2(a.im, bc2(w.x), mul2(a.re, bc2(-w.y)))};
}
template <bool INV> __device__ __forceinline__ c2 tw2(c2 a, cpx<float> w) { return INV ? cmulc2(a, w) : cmul2(a, w); }
__device__ __forceinline__ c2 scale2(c2 a, float s) { return c2{mul2(a.re, bc2(s)), mul2(a.im, bc2(s))}; }

__device__ __forceinline__ void st_c2(c2* p, c2 v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
}
__device__ __forceinline__ c2 ld_c2(const c2* p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  return c2{make_float2(t.x, t.y), make_float2(t.z, t.w)};
}

// ----------------------------------------------------------------------------------
// Small DFTs on paired values (same algebra as the scalar ones in bsct_fft.cuh)
// ----------------------------------------------------------------------------------
template <bool INV> __device__ __forceinline__ void dft2p(c2& a, c2& b) {
  const c2 t = a - b;
  a = a + b;
  b = t;
}
template <bool INV> __device__ __forceinline__ void dft4p(c2& v0, c2& v1, c2& v2, c2& v3) {
  const c2 a0 = v0 + v2, a1 = v0 - v2, a2 = v1 + v3, a3 = mul_mi2<INV>(v1 - v3);
  v0 = a0 + a2;
  v2 = a0 - a2;
  v1 = a1 + a3;
  v3 = a1 - a3;
}
// inputs v2, v3 known to be zero
template <bool INV> __device__ __forceinline__ void dft4hp(c2& v0, c2& v1, c2& v2, c2& v3) {
  const c2 a = v0, b = v1, bi = mul_mi2<INV>(v1);
  v0 = a + b;
  v2 = a - b;
  v1 = a + bi;
  v3 = a - bi;
}
template <bool INV> __device__ __forceinline__ void dft3p(c2& a, c2& b, c2& c) {
  const float h3 = 0.86602540378443864676f;  // sqrt(3)/2
  const c2 t1 = b + c;
  const c2 t2 = c2{fma2(bc2(-0.5f), t1.re, a.re), fma2(bc2(-0.5f), t1.im, a.im)};
  const c2 t3 = mul_mi2<INV>(scale2(b - c, h3));
  a = a + t1;
  b = t2 + t3;
  c = t2 - t3;
}
// a * w^k for the constant 16th roots used inside dft16 (k in {1, 2, 3, 6, 9})
template <bool INV> __device__ __forceinline__ c2 w16mul(c2 a, int k) {
  const float C1 = 0.92387953251128675613f, S1 = 0.38268343236508977173f, H = 0.70710678118654752440f;
  float c, s;
  switch (k) {
    case 1: c = C1; s = S1; break;
    case 2: c = H; s = H; break;
    case 3: c = S1; s = C1; break;
    case 6: c = -H; s = H; break;
    case 9: c = -C1; s = -S1; break;
    default: c = 1.f; s = 0.f; break;
  }
  return cmul2(a, mk(c, INV ? s : -s));
}
template <bool INV, bool HALF = false> __device__ __forceinline__ void dft8p(c2* v) {
  if constexpr (HALF) {
    dft4hp<INV>(v[0], v[2], v[4], v[6]);
    dft4hp<INV>(v[1], v[3], v[5], v[7]);
  } else {
    dft4p<INV>(v[0], v[2], v[4], v[6]);
    dft4p<INV>(v[1], v[3], v[5], v[7]);
  }
  const float H = 0.70710678118654752440f;
  const c2 o0 = v[1];
  const c2 o1 = cmul2(v[3], mk(H, INV ? H : -H));
  const c2 o2 = mul_mi2<INV>(v[5]);
  const c2 o3 = cmul2(v[7], mk(-H, INV ? H : -H));
  const c2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  v[0] = e0 + o0; v[4] = e0 - o0;
  v[1] = e1 + o1; v[5] = e1 - o1;
  v[2] = e2 + o2; v[6] = e2 - o2;
  v[3] = e3 + o3; v[7] = e3 - o3;
}
// 16 = 4 x 4: r = r1 + 4 r2, k = k1 + 4 k2
template <bool INV, bool HALF = false> __device__ __forceinline__ void dft16p(c2* v) {
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) {
    if constexpr (HALF) dft4hp<INV>(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
    else dft4p<INV>(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
  }
  v[5] = w16mul<INV>(v[5], 1);
  v[9] = w16mul<INV>(v[9], 2);
  v[13] = w16mul<INV>(v[13], 3);
  v[6] = w16mul<INV>(v[6], 2);
  v[10] = mul_mi2<INV>(v[10]);
  v[14] = w16mul<INV>(v[14], 6);
  v[7] = w16mul<INV>(v[7], 3);
  v[11] = w16mul<INV>(v[11], 6);
  v[15] = w16mul<INV>(v[15], 9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4p<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  c2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}
template <int R, bool INV, bool HALF = false> __device__ __forceinline__ void dftp(c2* v) {
  static_assert(!HALF || R % 2 == 0, "half-zero stage needs an even radix");
  if constexpr (R == 2) { if constexpr (HALF) v[1] = v[0]; else dft2p<INV>(v[0], v[1]); }
  else if constexpr (R == 3) dft3p<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) { if constexpr (HALF) dft4hp<INV>(v[0], v[1], v[2], v[3]); else dft4p<INV>(v[0], v[1], v[2], v[3]); }
  else if constexpr (R == 8) dft8p<INV, HALF>(v);
  else if constexpr (R == 16) dft16p<INV, HALF>(v);
  else static_assert(R == 2, "unsupported radix");
}

// ----------------------------------------------------------------------------------
// Stages (thread layout, twiddle tables and register cache as in bsct_fft.cuh)
// ----------------------------------------------------------------------------------
template <int L, int R, int NSV, bool INV, bool HALF, int S, bool CACHED>
__device__ __forceinline__ void stage_compute2(c2 (&v)[Plan<L>::E], int tid, const cpx<float>* __restrict__ tws,
                                               const TwCache<float, L>* cache) {
  constexpr int E = Plan<L>::E;
  constexpr int TT = L / E;
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    if constexpr (NSV > 1 && (R == 8 || R == 16)) {
      const int j = tid + b * TT;
      cpx<float> w[R];
      if constexpr (CACHED) {
        w[1] = cache->w[S][b][0];
        w[2] = cache->w[S][b][1];
        w[4] = cache->w[S][b][2];
        if constexpr (R == 16) w[8] = cache->w[S][b][3];
      } else {
        const cpx<float>* t = tws + (NSV - 1) + (j % NSV);
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
      for (int r = 1; r < R; ++r) v[b * R + r] = tw2<INV>(v[b * R + r], w[r]);
    } else if constexpr (NSV > 1) {
      const int j = tid + b * TT;
      const cpx<float>* t = tws + (NSV - 1) + (j % NSV);
#pragma unroll
      for (int r = 1; r < R; ++r) v[b * R + r] = tw2<INV>(v[b * R + r], ld_cpx(t + (r - 1) * NSV));
    }
    dftp<R, INV, HALF>(&v[b * R]);
  }
}

template <int L, int R, int NSV, int R2>
__device__ __forceinline__ void stage_exchange2(c2 (&v)[Plan<L>::E], c2* sm, int tid) {
  constexpr int E = Plan<L>::E;
  constexpr int TT = L / E;
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    const int j = tid + b * TT;
    const int base = (j / NSV) * NSV * R + (j % NSV);
    if constexpr (NSV % 16 == 0) {
      const int pb = spad(base);
#pragma unroll
      for (int r = 0; r < R; ++r) st_c2(sm + pb + r * (NSV + NSV / 16), v[b * R + r]);
    } else if constexpr (NSV == 1 && 16 % R == 0) {
      const int pb = spad(base);
#pragma unroll
      for (int r = 0; r < R; ++r) st_c2(sm + pb + r, v[b * R + r]);
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) st_c2(sm + spad(base + r * NSV), v[b * R + r]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < E / R2; ++b) {
    const int j = tid + b * TT;
    if constexpr ((L / R2) % 16 == 0) {
      const int pj = spad(j);
#pragma unroll
      for (int r = 0; r < R2; ++r) v[b * R2 + r] = ld_c2(sm + pj + r * ((L / R2) + (L / R2) / 16));
    } else {
#pragma unroll
      for (int r = 0; r < R2; ++r) v[b * R2 + r] = ld_c2(sm + spad(j + r * (L / R2)));
    }
  }
  __syncthreads();
}

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// hook(): called by every thread once the shared buffer is free for good (after the last
// exchange), before the last stage's arithmetic - e.g. to start copies into the buffer
template <int L, bool INV, bool REV, bool HALF, int S, bool CACHED, typename F>
__device__ __forceinline__ void fft2_stages(c2 (&v)[Plan<L>::E], c2* sm, int tid, const cpx<float>* __restrict__ tws,
                                            const TwCache<float, L>* cache, const F& hook) {
  constexpr int R = radix_of<L, REV>(S);
  constexpr int NSV = ns_of<L, REV>(S);
  if constexpr (S + 1 == Plan<L>::NS) hook();
  stage_compute2<L, R, NSV, INV, HALF && S == 0, S, CACHED>(v, tid, tws, cache);
  if constexpr (S + 1 < Plan<L>::NS) {
    stage_exchange2<L, R, NSV, radix_of<L, REV>(S + 1)>(v, sm, tid);
    fft2_stages<L, INV, REV, HALF, S + 1, CACHED>(v, sm, tid, tws, cache, hook);
  }
}

// Paired FFT of length L by L/E threads: register layouts as fft() in bsct_fft.cuh; sm is
// this pair's shared buffer of smem_elems<L>() c2 values.
template <int L, bool INV, bool REV, bool HALF = false, typename F = NoHook>
__device__ __forceinline__ void fft2(c2 (&v)[Plan<L>::E], c2* sm, int tid, const cpx<float>* __restrict__ tws,
                                     const F& hook = F()) {
  fft2_stages<L, INV, REV, HALF, 0, false>(v, sm, tid, tws, nullptr, hook);
}
template <int L, bool INV, bool REV, bool HALF = false, typename F = NoHook>
__device__ __forceinline__ void fft2_cached(c2 (&v)[Plan<L>::E], c2* sm, int tid, const cpx<float>* __restrict__ tws,
                                            const TwCache<float, L>& cache, const F& hook = F()) {
  fft2_stages<L, INV, REV, HALF, 0, true>(v, sm, tid, tws, &cache, hook);
}

}  // namespace bsct
