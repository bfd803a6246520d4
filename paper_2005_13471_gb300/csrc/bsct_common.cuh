// Common device/host helpers for libbsct (pixel-basis Gram filtering, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bsct.h"

namespace bsct {

template <typename T> struct cpx { T x, y; };

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> w) {
  return mk(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
template <typename T> __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> w) {  // a * conj(w)
  return mk(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y));
}
template <typename T> __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ cpx<T> mul_mi(cpx<T> a) {
  return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

// vector-width aliases for coalesced complex loads / stores
template <typename T> struct vec2;
template <> struct vec2<float> { typedef float2 type; };
template <> struct vec2<double> { typedef double2 type; };

template <typename T> __device__ __forceinline__ cpx<T> ld_cpx(const cpx<T>* p) {
  typename vec2<T>::type v = *reinterpret_cast<const typename vec2<T>::type*>(p);
  return mk(v.x, v.y);
}
// Load through L2 only (ld.global.cg).  Kernels launched with programmatic dependent
// launch start before their predecessor has finished, so the L1 invalidation that
// separates dependent grids can come before the predecessor's stores; L1 may then still
// hold an older copy of the line.  Every load of data another kernel writes goes through
// this in those kernels (constant tables may use ld_cpx).
template <typename T> __device__ __forceinline__ cpx<T> ld_cpx_cg(const cpx<T>* p) {
  typename vec2<T>::type v = __ldcg(reinterpret_cast<const typename vec2<T>::type*>(p));
  return mk(v.x, v.y);
}
template <typename T> __device__ __forceinline__ void st_cpx(cpx<T>* p, cpx<T> a) {
  typename vec2<T>::type v; v.x = a.x; v.y = a.y;
  *reinterpret_cast<typename vec2<T>::type*>(p) = v;
}

}  // namespace bsct

#define BSCT_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) { bsct_set_last_cuda_error(_e); return BSCT_ERR_CUDA; } \
  } while (0)

// records the CUDA error of the last failing call (readable via bsct_last_error_string)
void bsct_set_last_cuda_error(cudaError_t e);
void bsct_set_last_message(const char* msg);
