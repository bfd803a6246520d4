// Gram apply of many images held in host memory, with the transfers overlapped.
//
// Image k goes through three stages on library streams:
//   copy in  (host x_k -> device dx[k % 2]),
//   apply    (dy[k % 2] = G dx[k % 2], the handle's FFT apply),
//   copy out (dy[k % 2] -> host y_k),
// so that while image k is transformed, image k + 1 is copied in and image k - 1 out.
// Two device images per direction (double buffering); events order the reuse of a
// buffer after the stage that last read it.  In steady state one image takes as long as
// the slowest stage (the copies over the host link for the FP32 apply at N = 2048).
#include "bsct_internal.h"

using namespace bsct;

// copy streams per direction (each image is copied in HP_LANES parts): at N = 2048 one
// lane gave 9 133 images/s end to end and two lanes 8 135, so one
constexpr int HP_LANES = 1;

struct bsct_host_pipe {
  cudaStream_t s[1 + 2 * HP_LANES] = {};  // apply, copy-in lanes, copy-out lanes
  cudaEvent_t in_done[2][HP_LANES] = {}, out_done[2][HP_LANES] = {}, comp_done[2] = {};
  cudaEvent_t start = nullptr, done[HP_LANES] = {};
  void* dx[2] = {nullptr, nullptr};
  void* dy[2] = {nullptr, nullptr};
};

void bsct_host_pipe_free(bsct_host_pipe* p) {
  if (!p) return;
  for (cudaStream_t& st : p->s)
    if (st) cudaStreamDestroy(st);
  for (int b = 0; b < 2; ++b) {
    for (int l = 0; l < HP_LANES; ++l) {
      if (p->in_done[b][l]) cudaEventDestroy(p->in_done[b][l]);
      if (p->out_done[b][l]) cudaEventDestroy(p->out_done[b][l]);
    }
    if (p->comp_done[b]) cudaEventDestroy(p->comp_done[b]);
    cudaFree(p->dx[b]);
    cudaFree(p->dy[b]);
  }
  if (p->start) cudaEventDestroy(p->start);
  for (cudaEvent_t& e : p->done)
    if (e) cudaEventDestroy(e);
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
  for (cudaStream_t& st : p->s)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    for (int l = 0; l < HP_LANES && e == cudaSuccess; ++l) {
      e = cudaEventCreateWithFlags(&p->in_done[b][l], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->out_done[b][l], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->comp_done[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&p->dx[b], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->dy[b], bytes);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  for (cudaEvent_t& ev : p->done)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
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
  cudaStream_t st = (cudaStream_t)stream, sa = p->s[0];
  const cudaStream_t* si = p->s + 1;             // copy-in lanes
  const cudaStream_t* so = p->s + 1 + HP_LANES;  // copy-out lanes
  const int mode = g->precision == BSCT_F32 ? BSCT_APPLY_FFT32 : BSCT_APPLY_F64;
  // an image is copied as HP_LANES contiguous parts (16-byte multiples but the last)
  size_t part = (bytes / HP_LANES + 15) & ~(size_t)15;
  // everything below runs after the work already queued on the caller's stream
  BSCT_CUDA_TRY(cudaEventRecord(p->start, st));
  for (cudaStream_t s : p->s) BSCT_CUDA_TRY(cudaStreamWaitEvent(s, p->start, 0));
  const char* hx = (const char*)h_x;
  char* hy = (char*)h_y;
  for (int k = 0; k < n; ++k) {
    const int b = k & 1;
    for (int l = 0; l < HP_LANES; ++l) {
      const size_t off = (size_t)l * part, len = off >= bytes ? 0 : (bytes - off < part ? bytes - off : part);
      if (k >= 2) BSCT_CUDA_TRY(cudaStreamWaitEvent(si[l], p->comp_done[b], 0));  // dx[b] read by apply k - 2
      if (len) BSCT_CUDA_TRY(cudaMemcpyAsync((char*)p->dx[b] + off, hx + (size_t)k * bytes + off, len,
                                             cudaMemcpyHostToDevice, si[l]));
      BSCT_CUDA_TRY(cudaEventRecord(p->in_done[b][l], si[l]));
      BSCT_CUDA_TRY(cudaStreamWaitEvent(sa, p->in_done[b][l], 0));
      if (k >= 2) BSCT_CUDA_TRY(cudaStreamWaitEvent(sa, p->out_done[b][l], 0));  // dy[b] copied out (k - 2)
    }
    int rc = bsct_gram_apply(g, p->dx[b], p->dy[b], mode, sa);
    if (rc != BSCT_OK) return rc;
    BSCT_CUDA_TRY(cudaEventRecord(p->comp_done[b], sa));
    for (int l = 0; l < HP_LANES; ++l) {
      const size_t off = (size_t)l * part, len = off >= bytes ? 0 : (bytes - off < part ? bytes - off : part);
      BSCT_CUDA_TRY(cudaStreamWaitEvent(so[l], p->comp_done[b], 0));
      if (len) BSCT_CUDA_TRY(cudaMemcpyAsync(hy + (size_t)k * bytes + off, (char*)p->dy[b] + off, len,
                                             cudaMemcpyDeviceToHost, so[l]));
      BSCT_CUDA_TRY(cudaEventRecord(p->out_done[b][l], so[l]));
    }
  }
  // the caller's stream continues once the last image is back on every lane (which
  // orders after all the other work)
  for (int l = 0; l < HP_LANES; ++l) {
    BSCT_CUDA_TRY(cudaEventRecord(p->done[l], so[l]));
    BSCT_CUDA_TRY(cudaStreamWaitEvent(st, p->done[l], 0));
  }
  return BSCT_OK;
}
