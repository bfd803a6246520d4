// Launch-shape selection for the FFT Gram apply (the autotuner).  Each supported size N
// has its own current shape per device and precision (rows per CTA of the two row
// passes, CTAs per SM of the column pass; see gram_fft.cu).  bsct_fft_autotune times
// every valid shape on scratch data of that size and keeps the fastest.
#include "bsct_internal.h"

using namespace bsct;

namespace {
template <typename T> int ops_for(int N, FftOps<T>* o) {
  if (!fft_ops_for<T>(N, o)) {
    bsct_set_last_message("unsupported N (see bsct_supported_size)");
    return BSCT_ERR_UNSUPPORTED_SIZE;
  }
  return BSCT_OK;
}

template <typename T> int get_shape(int N, bsct_fft_shape* out) {
  FftOps<T> o;
  int rc = ops_for<T>(N, &o);
  if (rc != BSCT_OK) return rc;
  int fwd[3], inv[3], idx[3];
  o.shape_cands(fwd, inv);
  o.shape_index(idx, 0);
  out->rows_fwd = fwd[idx[0]];
  out->rows_inv = inv[idx[1]];
  out->cols_one_per_sm = idx[2];
  out->reserved = 0;
  return BSCT_OK;
}

template <typename T> int set_shape(int N, const bsct_fft_shape* s) {
  FftOps<T> o;
  int rc = ops_for<T>(N, &o);
  if (rc != BSCT_OK) return rc;
  int fwd[3], inv[3], idx[3] = {-1, -1, s->cols_one_per_sm ? 1 : 0};
  o.shape_cands(fwd, inv);
  for (int i = 0; i < 3; ++i) {
    if (fwd[i] && fwd[i] == s->rows_fwd) idx[0] = i;
    if (inv[i] && inv[i] == s->rows_inv) idx[1] = i;
  }
  return o.shape_index(idx, 1);
}

template <typename T> __global__ void k_fill(T* a, long n, T v) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) a[i] = v;
}

// flush_bytes > 0: before every timed apply, a write of that many bytes evicts the data of
// the previous one from L2 (the applies are then timed one by one, the writes excluded)
template <typename T>
int autotune(int N, int reps, bsct_fft_shape* best, double* best_us, double* all_us, cudaStream_t st,
             long flush_bytes = 0) {
  FftOps<T> o;
  int rc = ops_for<T>(N, &o);
  if (rc != BSCT_OK) return rc;
  const long n = (long)N * N, ng = (long)(N + 1) * 2 * N;
  T *x = nullptr, *y = nullptr, *Gt = nullptr;
  cpx<T>*S = nullptr, *tw = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  unsigned char* fl = nullptr;
  auto cleanup = [&]() {
    cudaFree(x); cudaFree(y); cudaFree(Gt); cudaFree(S); cudaFree(tw); cudaFree(fl);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
#define TTRY(expr)                                                    \
  do {                                                                \
    cudaError_t _e = (expr);                                          \
    if (_e != cudaSuccess) { bsct_set_last_cuda_error(_e); cleanup(); return BSCT_ERR_CUDA; } \
  } while (0)
  TTRY(cudaMalloc(&x, n * sizeof(T)));
  TTRY(cudaMalloc(&y, n * sizeof(T)));
  TTRY(cudaMalloc(&Gt, ng * sizeof(T)));
  TTRY(cudaMalloc(&S, n * sizeof(cpx<T>)));
  TTRY(cudaMalloc(&tw, fft_table_elems(N) * sizeof(cpx<T>)));
  TTRY(cudaEventCreate(&e0));
  TTRY(cudaEventCreate(&e1));
  if (flush_bytes > 0) TTRY(cudaMalloc(&fl, (size_t)flush_bytes));
  k_fill<T><<<256, 256, 0, st>>>(x, n, T(1));
  k_fill<T><<<256, 256, 0, st>>>(Gt, ng, T(1e-6));
  count_launch(2);
  rc = build_fft_tables<T>(tw, N, st);
  if (rc != BSCT_OK) { cleanup(); return rc; }
  int fwd[3], inv[3], keep[3];
  o.shape_cands(fwd, inv);
  o.shape_index(keep, 0);
  double best_t = 1e30;
  int best_idx[3] = {keep[0], keep[1], keep[2]};
  for (int i = 0; i < 18; ++i) {
    int idx[3] = {i / 6, (i / 2) % 3, i % 2};
    if (all_us) all_us[i] = -1.0;
    if (!fwd[idx[0]] || !inv[idx[1]]) continue;
    o.shape_index(idx, 1);
    for (int w = 0; w < 3; ++w) {
      rc = o.apply(x, y, S, Gt, tw, st);
      if (rc != BSCT_OK) { o.shape_index(keep, 1); cleanup(); return rc; }
    }
    double tot_ms = 0.0;
    if (!fl) {
      TTRY(cudaEventRecord(e0, st));
      for (int r = 0; r < reps; ++r) o.apply(x, y, S, Gt, tw, st);
      TTRY(cudaEventRecord(e1, st));
      TTRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      TTRY(cudaEventElapsedTime(&ms, e0, e1));
      tot_ms = ms;
    } else {
      for (int r = 0; r < reps; ++r) {
        k_fill<unsigned char><<<1024, 256, 0, st>>>(fl, flush_bytes, (unsigned char)r);
        count_launch();
        TTRY(cudaEventRecord(e0, st));
        o.apply(x, y, S, Gt, tw, st);
        TTRY(cudaEventRecord(e1, st));
        TTRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        TTRY(cudaEventElapsedTime(&ms, e0, e1));
        tot_ms += ms;
      }
    }
    const double us = 1e3 * tot_ms / reps;
    if (all_us) all_us[i] = us;
    if (us < best_t) {
      best_t = us;
      best_idx[0] = idx[0];
      best_idx[1] = idx[1];
      best_idx[2] = idx[2];
    }
  }
#undef TTRY
  o.shape_index(best_idx, 1);
  cleanup();
  if (best) get_shape<T>(N, best);
  if (best_us) *best_us = best_t;
  return BSCT_OK;
}
}  // namespace

extern "C" int bsct_fft_get_shape(int32_t N, int precision, bsct_fft_shape* out) {
  if (!out || (precision != BSCT_F32 && precision != BSCT_F64)) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  return precision == BSCT_F32 ? get_shape<float>(N, out) : get_shape<double>(N, out);
}

extern "C" int bsct_fft_set_shape(int32_t N, int precision, const bsct_fft_shape* shape) {
  if (!shape || (precision != BSCT_F32 && precision != BSCT_F64)) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  return precision == BSCT_F32 ? set_shape<float>(N, shape) : set_shape<double>(N, shape);
}

extern "C" int bsct_fft_shape_candidates(int32_t N, int precision, int32_t* rows_fwd, int32_t* rows_inv) {
  if (!rows_fwd || !rows_inv || (precision != BSCT_F32 && precision != BSCT_F64)) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  int f[3], v[3];
  if (precision == BSCT_F32) {
    FftOps<float> o;
    int rc = ops_for<float>(N, &o);
    if (rc != BSCT_OK) return rc;
    o.shape_cands(f, v);
  } else {
    FftOps<double> o;
    int rc = ops_for<double>(N, &o);
    if (rc != BSCT_OK) return rc;
    o.shape_cands(f, v);
  }
  for (int i = 0; i < 3; ++i) { rows_fwd[i] = f[i]; rows_inv[i] = v[i]; }
  return BSCT_OK;
}

extern "C" int bsct_fft_autotune_flushed(int32_t N, int precision, int reps, int64_t flush_bytes,
                                         bsct_fft_shape* best, double* best_us, double* all_us, void* stream) {
  if (reps < 1 || flush_bytes < 0 || (precision != BSCT_F32 && precision != BSCT_F64)) {
    bsct_set_last_message("invalid argument");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return precision == BSCT_F32 ? autotune<float>(N, reps, best, best_us, all_us, st, (long)flush_bytes)
                               : autotune<double>(N, reps, best, best_us, all_us, st, (long)flush_bytes);
}

extern "C" int bsct_fft_autotune(int32_t N, int precision, int reps, bsct_fft_shape* best, double* best_us,
                                 double* all_us, void* stream) {
  if (reps < 1 || (precision != BSCT_F32 && precision != BSCT_F64)) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  return precision == BSCT_F32 ? autotune<float>(N, reps, best, best_us, all_us, st)
                               : autotune<double>(N, reps, best, best_us, all_us, st);
}
