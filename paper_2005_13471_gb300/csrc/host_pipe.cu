// Gram apply of many images held in host memory, with the transfers overlapped.
//
// Image k goes through three stages, each on its own library stream:
//   copy in  (host x_k -> device dx[k % 2]),
//   apply    (dy[k % 2] = G dx[k % 2], the handle's FFT apply),
//   copy out (dy[k % 2] -> host y_k),
// so that while image k is transformed, image k + 1 is copied in and image k - 1 out.
// Two device images per direction (double buffering); events order the reuse of a
// buffer after the stage that last read it.  In steady state one image takes as long as
// the slowest stage (the copies over the host link for the FP32 apply at N = 2048).
#include "bsct_internal.h"

using namespace bsct;

struct bsct_host_pipe {
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};  // copy in, apply, copy out
  cudaEvent_t in_done[2] = {}, comp_done[2] = {}, out_done[2] = {}, start = nullptr, done = nullptr;
  void* dx[2] = {nullptr, nullptr};
  void* dy[2] = {nullptr, nullptr};
};

void bsct_host_pipe_free(bsct_host_pipe* p) {
  if (!p) return;
  for (int i = 0; i < 3; ++i)
    if (p->s[i]) cudaStreamDestroy(p->s[i]);
  for (int b = 0; b < 2; ++b) {
    if (p->in_done[b]) cudaEventDestroy(p->in_done[b]);
    if (p->comp_done[b]) cudaEventDestroy(p->comp_done[b]);
    if (p->out_done[b]) cudaEventDestroy(p->out_done[b]);
    cudaFree(p->dx[b]);
    cudaFree(p->dy[b]);
  }
  if (p->start) cudaEventDestroy(p->start);
  if (p->done) cudaEventDestroy(p->done);
  delete p;
}

static int pipe_create(bsct_gram* g, size_t bytes) {
  bsct_host_pipe* p = new bsct_host_pipe();
  auto fail = [&](cudaError_t e) {
    bsct_set_last_cuda_error(e);
    bsct_host_pipe_free(p);
    return BSCT_ERR_CUDA;
  };
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&p->s[i], cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&p->in_done[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->comp_done[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->out_done[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&p->dx[b], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->dy[b], bytes);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail(e);
  g->pipe = p;
  return BSCT_OK;
}

extern "C" int bsct_gram_apply_host(bsct_gram* g, const void* h_x, void* h_y, int32_t n, void* stream) {
  if (!g || n < 0) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  if (n == 0) return BSCT_OK;  // the image pointers may then be NULL
  if (!h_x || !h_y) { bsct_set_last_message("NULL image pointer"); return BSCT_ERR_INVALID_ARG; }
  const size_t bytes = (size_t)g->N * g->N * (g->precision == BSCT_F32 ? sizeof(float) : sizeof(double));
  if (!g->pipe) {
    int rc = pipe_create(g, bytes);
    if (rc != BSCT_OK) return rc;
  }
  bsct_host_pipe* p = g->pipe;
  cudaStream_t st = (cudaStream_t)stream, si = p->s[0], sa = p->s[1], so = p->s[2];
  const int mode = g->precision == BSCT_F32 ? BSCT_APPLY_FFT32 : BSCT_APPLY_F64;
  // everything below runs after the work already queued on the caller's stream
  BSCT_CUDA_TRY(cudaEventRecord(p->start, st));
  for (int i = 0; i < 3; ++i) BSCT_CUDA_TRY(cudaStreamWaitEvent(p->s[i], p->start, 0));
  const char* hx = (const char*)h_x;
  char* hy = (char*)h_y;
  for (int k = 0; k < n; ++k) {
    const int b = k & 1;
    if (k >= 2) BSCT_CUDA_TRY(cudaStreamWaitEvent(si, p->comp_done[b], 0));  // dx[b] read by apply k - 2
    BSCT_CUDA_TRY(cudaMemcpyAsync(p->dx[b], hx + (size_t)k * bytes, bytes, cudaMemcpyHostToDevice, si));
    BSCT_CUDA_TRY(cudaEventRecord(p->in_done[b], si));
    BSCT_CUDA_TRY(cudaStreamWaitEvent(sa, p->in_done[b], 0));
    if (k >= 2) BSCT_CUDA_TRY(cudaStreamWaitEvent(sa, p->out_done[b], 0));  // dy[b] copied out (k - 2)
    int rc = bsct_gram_apply(g, p->dx[b], p->dy[b], mode, sa);
    if (rc != BSCT_OK) return rc;
    BSCT_CUDA_TRY(cudaEventRecord(p->comp_done[b], sa));
    BSCT_CUDA_TRY(cudaStreamWaitEvent(so, p->comp_done[b], 0));
    BSCT_CUDA_TRY(cudaMemcpyAsync(hy + (size_t)k * bytes, p->dy[b], bytes, cudaMemcpyDeviceToHost, so));
    BSCT_CUDA_TRY(cudaEventRecord(p->out_done[b], so));
  }
  // the caller's stream continues once the last image is back (which orders after all)
  BSCT_CUDA_TRY(cudaEventRecord(p->done, so));
  BSCT_CUDA_TRY(cudaStreamWaitEvent(st, p->done, 0));
  return BSCT_OK;
}
