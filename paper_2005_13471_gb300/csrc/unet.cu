// Learned warm start for CG: a 4-level encoder-decoder CNN (U-Net) with BF16 tensor-core
// convolutions and FP32 accumulation, trained on (back projection, converged
// reconstruction) pairs that the method itself produces.  Not part of the paper.
//
// Architecture (channels-first, activations stored [C][n][H][W] in FP32):
//   level 0: conv3x3(1->32)+ReLU, conv3x3(32->32)+ReLU -> e0 ; maxpool 2x2
//   level 1: 32->64, 64->64 -> e1 ; pool      level 2: 64->128, 128->128 -> e2 ; pool
//   level 3: 128->256, 256->256
//   up 3: convT2x2(256->128) ++ e2 -> conv(256->128), conv(128->128)
//   up 2: convT2x2(128->64)  ++ e1 -> conv(128->64),  conv(64->64)
//   up 1: convT2x2(64->32)   ++ e0 -> conv(64->32),   conv(32->32) ; head conv1x1(32->1)
// 3x3 convolutions run as im2col (BF16) x weights (BF16) GEMMs on the tensor cores;
// backward: weight gradient = dpre x col^T, data gradient = W^T x dpre then a col2im
// gather; the transposed convolutions are GEMMs followed by a 2x2 scatter (gather in
// the backward pass).  Master weights, gradients and Adam moments are FP32; a BF16 copy
// of the weights feeds the GEMMs.
#include <cuda_bf16.h>
#include <math.h>

#include <vector>

#include "bsct_internal.h"

namespace {

using bsct::count_launch;
typedef __nv_bfloat16 bf16;

constexpr int TPB = 256;
inline unsigned nblk(long n) { return (unsigned)((n + TPB - 1) / TPB); }

// ---------------------------------------------------------------------------- kernels
__device__ __forceinline__ unsigned long long splitmix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
// He-normal weights by Box-Muller on a counter-based generator; valid < cols of each row
__global__ void k_init_weights(float* w, long n, int cols, int valid, float stdv, unsigned long long seed) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if ((int)(i % cols) >= valid) { w[i] = 0.f; return; }
  const unsigned long long a = splitmix(seed * 0x100000001B3ull + 2 * (unsigned long long)i);
  const unsigned long long b = splitmix(seed * 0x100000001B3ull + 2 * (unsigned long long)i + 1);
  const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
  w[i] = (float)(stdv * sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
}

__global__ void k_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// col[(ci*9 + ky*3 + kx)][(n, y, x)] = in[ci][n][y+ky-1][x+kx-1] (zero outside), rows >= 9*C zero.
// Grid (NB*H, C + 1): block (image row, input channel) stages the three input rows y-1..y+1
// (with a zero halo) in shared memory and writes the nine col rows of that channel, two x
// per thread as one BF16 pair (W even); blocks with blockIdx.y == C write the zero rows
__global__ void k_im2col3(const float* __restrict__ in, int C, int NB, int H, int W, int Kpad,
                          bf16* __restrict__ col) {
  extern __shared__ float srow[];  // 3 (W + 2)
  const int row = blockIdx.x, ci = blockIdx.y;  // row = n H + y
  const long P = (long)NB * H * W;
  const int W2 = W >> 1;
  if (ci == C) {
    for (int k = 9 * C; k < Kpad; ++k) {
      __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(col + (long)k * P + (long)row * W);
      for (int x2 = threadIdx.x; x2 < W2; x2 += blockDim.x) dst[x2] = __floats2bfloat162_rn(0.f, 0.f);
    }
    return;
  }
  const int nb = row / H, y = row - nb * H;
  const float* src = in + ((long)ci * NB + nb) * H * W;
  const int WS = W + 2;
  for (int t = threadIdx.x; t < 3 * WS; t += blockDim.x) {
    const int r = t / WS, xx = t - r * WS - 1, yy = y - 1 + r;
    srow[t] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? src[(long)yy * W + xx] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int ky = tap / 3, kx = tap - 3 * ky;
    __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(col + (long)(ci * 9 + tap) * P + (long)row * W);
    const float* s2 = srow + ky * WS + kx;  // s2[x] = in[y + ky - 1][x + kx - 1]
    for (int x2 = threadIdx.x; x2 < W2; x2 += blockDim.x) dst[x2] = __floats2bfloat162_rn(s2[2 * x2], s2[2 * x2 + 1]);
  }
}
inline int row_threads(int n) { return n >= 256 ? 256 : ((n + 31) / 32) * 32; }
inline void launch_im2col3(const float* in, int C, int NB, int H, int W, int Kpad, bf16* col, cudaStream_t st) {
  const unsigned gy = (unsigned)(C + (Kpad > 9 * C ? 1 : 0));
  k_im2col3<<<dim3((unsigned)(NB * H), gy), row_threads(W / 2), (size_t)3 * (W + 2) * sizeof(float), st>>>(
      in, C, NB, H, W, Kpad, col);
}

// gin[ci][n][y][x] = sum_{ky,kx} dcol[(ci,ky,kx)][n][y-ky+1][x-kx+1]; grid (NB*H, C), one image
// row per block
__global__ void k_col2im3(const float* __restrict__ dcol, int C, int NB, int H, int W, float* __restrict__ gin) {
  const int ci = blockIdx.y, row = blockIdx.x;
  const int nb = row / H, y = row - nb * H;
  const long P = (long)NB * H * W;
  const long base = (long)nb * H * W;
  float* out = gin + (long)ci * P + (long)row * W;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    float acc = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
      const int yy = y - ky + 1;
      if (yy < 0 || yy >= H) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int xx = x - kx + 1;
        if (xx < 0 || xx >= W) continue;
        acc += dcol[(long)(ci * 9 + ky * 3 + kx) * P + base + (long)yy * W + xx];
      }
    }
    out[x] = acc;
  }
}
inline void launch_col2im3(const float* dcol, int C, int NB, int H, int W, float* gin, cudaStream_t st) {
  k_col2im3<<<dim3((unsigned)(NB * H), (unsigned)C), row_threads(W), 0, st>>>(dcol, C, NB, H, W, gin);
}

// a[c][p] = act(a[c][p] + b[c]); grid (chunks, C), four values per thread (P % 4 == 0)
__global__ void k_bias_relu(float* __restrict__ a, const float* __restrict__ b, int C, long P, int relu) {
  const int c = blockIdx.y;
  const float bc = b[c];
  float4* row = reinterpret_cast<float4*>(a + (long)c * P);
  const long P4 = P >> 2;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < P4; i += (long)gridDim.x * blockDim.x) {
    float4 v = row[i];
    v.x += bc; v.y += bc; v.z += bc; v.w += bc;
    if (relu) { v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f); }
    row[i] = v;
  }
}
inline void launch_bias_relu(float* a, const float* b, int C, long P, int relu, cudaStream_t st) {
  long bx = (P / 4 + TPB - 1) / TPB;
  if (bx > 1024) bx = 1024;
  k_bias_relu<<<dim3((unsigned)bx, (unsigned)C), TPB, 0, st>>>(a, b, C, P, relu);
}

// dpre = g * (out > 0) (BF16 for the GEMMs); the channel sums go to per-block partials
// part[c][chunk] (grid: x = chunks of the channel, y = channel), added to db[c] in chunk
// order by k_chan_finish, so every run gives the same bits
__device__ __forceinline__ float block_reduce(float v) {
  __shared__ float red[TPB / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < 32) {
    t = threadIdx.x < TPB / 32 ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}
constexpr int CHUNK = 8192;
// relu = 0: no mask (a layer without its ReLU)
__global__ void k_relu_bwd(const float* __restrict__ g, const float* __restrict__ out, long P, bf16* __restrict__ dpre,
                           float* __restrict__ part, int relu = 1) {
  const int c = blockIdx.y;
  const long p0 = (long)blockIdx.x * CHUNK, p1 = p0 + CHUNK < P ? p0 + CHUNK : P;
  float acc = 0.f;
  for (long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const long i = (long)c * P + p;
    const float d = (!relu || out[i] > 0.f) ? g[i] : 0.f;
    dpre[i] = __float2bfloat16_rn(d);
    acc += d;
  }
  acc = block_reduce(acc);
  if (threadIdx.x == 0) part[(long)c * gridDim.x + blockIdx.x] = acc;
}

// part[c][chunk] = sum over the chunk of g[c][p]
__global__ void k_chan_sum(const float* __restrict__ g, long P, float* __restrict__ part) {
  const int c = blockIdx.y;
  const long p0 = (long)blockIdx.x * CHUNK, p1 = p0 + CHUNK < P ? p0 + CHUNK : P;
  float acc = 0.f;
  for (long p = p0 + threadIdx.x; p < p1; p += blockDim.x) acc += g[(long)c * P + p];
  acc = block_reduce(acc);
  if (threadIdx.x == 0) part[(long)c * gridDim.x + blockIdx.x] = acc;
}
// db[c] += sum over chunks of part[c][chunk] (one warp per channel: each lane sums a
// strided subset in order, then a fixed shuffle tree); with db_last, channel C goes to
// db_last[0] instead
__global__ void k_chan_finish(const float* __restrict__ part, int nchunks, float* __restrict__ db,
                              float* __restrict__ db_last = nullptr, int C = 0) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (int k = threadIdx.x; k < nchunks; k += 32) acc += part[(long)c * nchunks + k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) {
    if (db_last && c == C) db_last[0] += acc;
    else db[c] += acc;
  }
}
inline dim3 chan_grid(long P, int C) { return dim3((unsigned)((P + CHUNK - 1) / CHUNK), (unsigned)C); }
inline long chan_parts(long P, int C) { return (long)C * ((P + CHUNK - 1) / CHUNK); }

__global__ void k_maxpool2(const float* __restrict__ in, int C, int NB, int H, int W, float* __restrict__ out) {
  const int Ho = H / 2, Wo = W / 2;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)C * NB * Ho * Wo) return;
  const int x = (int)(i % Wo), y = (int)((i / Wo) % Ho);
  const long cn = i / ((long)Ho * Wo);
  const float* s = in + cn * H * W + (long)(2 * y) * W + 2 * x;
  out[i] = fmaxf(fmaxf(s[0], s[1]), fmaxf(s[W], s[W + 1]));
}
// routes g_out to the first maximum of each 2x2 window, adding into gin
__global__ void k_maxpool2_bwd(const float* __restrict__ in, const float* __restrict__ gout, int C, int NB, int H, int W,
                               float* __restrict__ gin) {
  const int Ho = H / 2, Wo = W / 2;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)C * NB * Ho * Wo) return;
  const int x = (int)(i % Wo), y = (int)((i / Wo) % Ho);
  const long cn = i / ((long)Ho * Wo);
  const long o = cn * H * W + (long)(2 * y) * W + 2 * x;
  const float v[4] = {in[o], in[o + 1], in[o + W], in[o + W + 1]};
  int a = 0;
  for (int k = 1; k < 4; ++k)
    if (v[k] > v[a]) a = k;
  const long t = o + (a >> 1) * W + (a & 1);
  gin[t] += gout[i];
}

// tmp[(co,dy,dx)][(n,y,x)] (+ b[co]) -> out[co][n][2y+dy][2x+dx]; grid (NB*2H, Co), one output
// row per block
__global__ void k_tconv_scatter(const float* __restrict__ tmp, const float* __restrict__ b, int Co, int NB, int H,
                                int W, float* __restrict__ out) {
  const int co = blockIdx.y, orow = blockIdx.x;  // orow = n 2H + Y
  const int nb = orow / (2 * H), Y = orow - nb * 2 * H, y = Y >> 1, dy = Y & 1;
  const long P = (long)NB * H * W;
  const float bc = b[co];
  const float* t0 = tmp + (long)(co * 4 + dy * 2) * P + (long)nb * H * W + (long)y * W;  // dx = 1: + P
  float* o = out + (long)co * 4 * P + (long)orow * 2 * W;
  for (int X = threadIdx.x; X < 2 * W; X += blockDim.x) o[X] = t0[(long)(X & 1) * P + (X >> 1)] + bc;
}
inline void launch_tconv_scatter(const float* tmp, const float* b, int Co, int NB, int H, int W, float* out,
                                 cudaStream_t st) {
  k_tconv_scatter<<<dim3((unsigned)(NB * 2 * H), (unsigned)Co), row_threads(2 * W), 0, st>>>(tmp, b, Co, NB, H, W, out);
}
// gathered[(co,dy,dx)][(n,y,x)] = bf16(gout[co][n][2y+dy][2x+dx]); grid (NB*H, Co*4)
__global__ void k_tconv_gather(const float* __restrict__ gout, int Co, int NB, int H, int W, bf16* __restrict__ g) {
  const int r = blockIdx.y, row = blockIdx.x;  // row = n H + y
  const int co = r >> 2, dy = (r >> 1) & 1, dx = r & 1;
  const int nb = row / H, y = row - nb * H;
  const long P = (long)NB * H * W;
  const float* src = gout + (long)co * 4 * P + ((long)nb * 2 * H + 2 * y + dy) * 2 * W + dx;
  bf16* d = g + (long)r * P + (long)row * W;
  for (int x = threadIdx.x; x < W; x += blockDim.x) d[x] = __float2bfloat16_rn(src[2 * x]);
}
inline void launch_tconv_gather(const float* gout, int Co, int NB, int H, int W, bf16* g, cudaStream_t st) {
  k_tconv_gather<<<dim3((unsigned)(NB * H), (unsigned)(Co * 4)), row_threads(W), 0, st>>>(gout, Co, NB, H, W, g);
}

// head: out[p] = sum_c w[c] a[c][p] + b
__global__ void k_head_fwd(const float* __restrict__ a, const float* __restrict__ w, const float* __restrict__ b, int C,
                           long P, float* __restrict__ out) {
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float acc = b[0];
  for (int c = 0; c < C; ++c) acc = fmaf(w[c], a[(long)c * P + p], acc);
  out[p] = acc;
}
__global__ void k_head_bwd_data(const float* __restrict__ gout, const float* __restrict__ w, int C, long P,
                                float* __restrict__ ga) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)C * P) return;
  ga[i] = w[i / P] * gout[i % P];
}
// part[c][chunk] = sum over the chunk of a[c][p] g[p] (grid y = channel; y == C: of g[p],
// for db); k_chan_finish then adds them to dw[c] / db
__global__ void k_head_bwd_w(const float* __restrict__ a, const float* __restrict__ g, int C, long P,
                             float* __restrict__ part) {
  const int c = blockIdx.y;
  const long p0 = (long)blockIdx.x * CHUNK, p1 = p0 + CHUNK < P ? p0 + CHUNK : P;
  float acc = 0.f;
  for (long p = p0 + threadIdx.x; p < p1; p += blockDim.x) acc += (c < C ? a[(long)c * P + p] : 1.f) * g[p];
  acc = block_reduce(acc);
  if (threadIdx.x == 0) part[(long)c * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_adam(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ wb, long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
  g[i] = 0.f;
}

// stream-ordered scratch of one call (freed at scope exit), and the layer shape checks
struct LayerScratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  bool ok = true;
  template <typename T> T* get(long n) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, (size_t)(n > 0 ? n : 1) * sizeof(T), st) != cudaSuccess) { ok = false; return nullptr; }
    ptrs.push_back(p);
    return (T*)p;
  }
  ~LayerScratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
};
bool layer_dims_ok(int n, int cin, int cout, int H, int W) {
  return n >= 1 && cin >= 1 && cout >= 1 && H >= 1 && W >= 2 && W % 2 == 0 && cout % 8 == 0 && (long)n * H * W % 8 == 0 &&
         (long)n * H * W * 9 * cin < (1L << 31);
}

// ---------------------------------------------------------------------------- network
struct Conv3 {
  int cin, cout, kpad;
  long w, b;  // offsets into the parameter arrays (w: cout x kpad)
};
struct TConv {
  int cin, cout;
  long w, b;  // w: (cout*4) x cin
};

}  // namespace

struct bsct_unet {
  int base = 32;
  long n_params = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16* wb = nullptr;
  Conv3 c0a, c0b, c1a, c1b, c2a, c2b, c3a, c3b, d2a, d2b, d1a, d1b, d0a, d0b;
  TConv t3, t2, t1;
  long hw, hb;  // head
  // activations for the cached shape
  int NB = 0, H = 0, W = 0;
  std::vector<void*> bufs;
  float *x = nullptr, *a00, *cat0, *p0, *a10, *cat1, *p1, *a20, *cat2, *p2, *a30, *a31, *u2a, *u2b, *u1a, *u1b, *u0a, *u0b;
  float *tmp, *dcol;
  float *g00, *gcat0, *gp0, *g10, *gcat1, *gp1, *g20, *gcat2, *gp2, *g30, *g31, *gu2a, *gu2b, *gu1a, *gu1b, *gu0a,
      *gu0b;
  bf16 *col, *dpre;
  float* red = nullptr;  // per-block partials of the channel sums (bias and head gradients)
  float* out = nullptr;
};

namespace {

long add_conv(bsct_unet* u, Conv3& c, int cin, int cout, long off) {
  c.cin = cin;
  c.cout = cout;
  c.kpad = ((9 * cin + 7) / 8) * 8;
  c.w = off;
  off += (long)cout * c.kpad;
  c.b = off;
  off += cout;
  return off;
}
long add_tconv(TConv& t, int cin, int cout, long off) {
  t.cin = cin;
  t.cout = cout;
  t.w = off;
  off += (long)cout * 4 * cin;
  t.b = off;
  off += cout;
  return off;
}

void free_acts(bsct_unet* u) {
  for (void* p : u->bufs) cudaFree(p);
  u->bufs.clear();
  u->NB = u->H = u->W = 0;
}

int alloc_acts(bsct_unet* u, int NB, int H, int W) {
  if (u->NB == NB && u->H == H && u->W == W) return BSCT_OK;
  free_acts(u);
  const int B = u->base;
  const long P0 = (long)NB * H * W, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  auto mk = [&](long n, size_t es = 4) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)n * es) != cudaSuccess) return nullptr;
    u->bufs.push_back(p);
    return p;
  };
  bool ok = true;
  auto f = [&](long n) {
    float* p = (float*)mk(n);
    ok = ok && p;
    return p;
  };
  u->x = f(P0);
  u->a00 = f(B * P0); u->cat0 = f(2 * B * P0); u->p0 = f(B * P1);
  u->a10 = f(2 * B * P1); u->cat1 = f(4 * B * P1); u->p1 = f(2 * B * P2);
  u->a20 = f(4 * B * P2); u->cat2 = f(8 * B * P2); u->p2 = f(4 * B * P3);
  u->a30 = f(8 * B * P3); u->a31 = f(8 * B * P3);
  u->u2a = f(4 * B * P2); u->u2b = f(4 * B * P2);
  u->u1a = f(2 * B * P1); u->u1b = f(2 * B * P1);
  u->u0a = f(B * P0); u->u0b = f(B * P0);
  u->out = f(P0);
  u->g00 = f(B * P0); u->gcat0 = f(2 * B * P0); u->gp0 = f(B * P1);
  u->g10 = f(2 * B * P1); u->gcat1 = f(4 * B * P1); u->gp1 = f(2 * B * P2);
  u->g20 = f(4 * B * P2); u->gcat2 = f(8 * B * P2); u->gp2 = f(4 * B * P3);
  u->g30 = f(8 * B * P3); u->g31 = f(8 * B * P3);
  u->gu2a = f(4 * B * P2); u->gu2b = f(4 * B * P2);
  u->gu1a = f(2 * B * P1); u->gu1b = f(2 * B * P1);
  u->gu0a = f(B * P0); u->gu0b = f(B * P0);
  // scratch: the largest im2col (K x P) over all layers, transposed-conv products
  long colmax = 0;
  const Conv3* cs[] = {&u->c0a, &u->c0b, &u->c1a, &u->c1b, &u->c2a, &u->c2b, &u->c3a,
                       &u->c3b, &u->d2a, &u->d2b, &u->d1a, &u->d1b, &u->d0a, &u->d0b};
  const long Ps[] = {P0, P0, P1, P1, P2, P2, P3, P3, P2, P2, P1, P1, P0, P0};
  for (int i = 0; i < 14; ++i) colmax = colmax > cs[i]->kpad * Ps[i] ? colmax : cs[i]->kpad * Ps[i];
  long tmpmax = 4L * B * 4 * P1;  // (cout*4) x P_in of the largest transposed conv
  if (8L * B * P3 * 4 > tmpmax) tmpmax = 8L * B * P3 * 4;
  if (2L * B * P2 * 4 > tmpmax) tmpmax = 2L * B * P2 * 4;
  u->col = (bf16*)mk(colmax, 2);
  u->dcol = f(colmax);
  {
    long redmax = chan_parts(P0, B + 1);  // head
    for (int i = 0; i < 14; ++i) redmax = redmax > chan_parts(Ps[i], cs[i]->cout) ? redmax : chan_parts(Ps[i], cs[i]->cout);
    const TConv* ts[] = {&u->t3, &u->t2, &u->t1};
    const long Pt[] = {P3, P2, P1};  // input pixels of the transposed convolutions
    for (int i = 0; i < 3; ++i) redmax = redmax > chan_parts(4 * Pt[i], ts[i]->cout) ? redmax : chan_parts(4 * Pt[i], ts[i]->cout);
    u->red = f(redmax);
  }
  u->tmp = f(tmpmax > 8L * B * P0 ? tmpmax : 8L * B * P0);
  u->dpre = (bf16*)mk(tmpmax > 8L * B * P0 ? tmpmax : 8L * B * P0, 2);
  ok = ok && u->col && u->dpre;
  if (!ok) {
    free_acts(u);
    bsct_set_last_message("out of device memory for U-Net activations");
    return BSCT_ERR_CUDA;
  }
  u->NB = NB;
  u->H = H;
  u->W = W;
  return BSCT_OK;
}

#define UTRY(expr)                            \
  do {                                        \
    int _rc = (expr);                         \
    if (_rc != BSCT_OK) return _rc;           \
  } while (0)

int conv_fwd(bsct_unet* u, const Conv3& c, const float* in, int NB, int H, int W, float* out, cudaStream_t st) {
  const long P = (long)NB * H * W;
  launch_im2col3(in, c.cin, NB, H, W, c.kpad, u->col, st);
  count_launch();
  UTRY(bsct::gemm_bf16(false, false, c.cout, (int)P, c.kpad, 1.f, u->wb + c.w, c.kpad, 0, u->col, P, 0, 0.f, out, P,
                       0, 1, st));
  launch_bias_relu(out, u->w + c.b, c.cout, P, 1, st);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

// gout: gradient of the post-ReLU output; gin (optional): gradient of the input (overwritten)
int conv_bwd(bsct_unet* u, const Conv3& c, const float* in, const float* out, const float* gout, int NB, int H, int W,
             float* gin, cudaStream_t st) {
  const long P = (long)NB * H * W;
  const dim3 cg = chan_grid(P, c.cout);
  k_relu_bwd<<<cg, TPB, 0, st>>>(gout, out, P, u->dpre, u->red);
  k_chan_finish<<<c.cout, 32, 0, st>>>(u->red, (int)cg.x, u->g + c.b);
  launch_im2col3(in, c.cin, NB, H, W, c.kpad, u->col, st);
  count_launch(3);
  // dW[cout][kpad] += dpre[cout][P] col[kpad][P]^T
  UTRY(bsct::gemm_bf16(false, true, c.cout, c.kpad, (int)P, 1.f, u->dpre, P, 0, u->col, P, 0, 1.f, u->g + c.w, c.kpad,
                       0, 1, st));
  if (gin) {
    // dcol[kpad][P] = W^T dpre
    UTRY(bsct::gemm_bf16(true, false, c.kpad, (int)P, c.cout, 1.f, u->wb + c.w, c.kpad, 0, u->dpre, P, 0, 0.f, u->dcol,
                         P, 0, 1, st));
    launch_col2im3(u->dcol, c.cin, NB, H, W, gin, st);
    count_launch();
  }
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

// transposed 2x2 stride-2 convolution from [cin][n][H][W] to [cout][n][2H][2W]
int tconv_fwd(bsct_unet* u, const TConv& t, const float* in, int NB, int H, int W, float* out, cudaStream_t st) {
  const long P = (long)NB * H * W;
  k_to_bf16<<<nblk((long)t.cin * P), TPB, 0, st>>>(in, u->dpre, (long)t.cin * P);
  count_launch();
  UTRY(bsct::gemm_bf16(false, false, t.cout * 4, (int)P, t.cin, 1.f, u->wb + t.w, t.cin, 0, u->dpre, P, 0, 0.f, u->tmp,
                       P, 0, 1, st));
  launch_tconv_scatter(u->tmp, u->w + t.b, t.cout, NB, H, W, out, st);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

int tconv_bwd(bsct_unet* u, const TConv& t, const float* in, const float* gout, int NB, int H, int W, float* gin,
              cudaStream_t st) {
  const long P = (long)NB * H * W;
  bf16* gg = u->dpre;                          // gathered gradient [(cout*4)][P]
  bf16* inb = u->col;                          // BF16 copy of the input [cin][P]
  launch_tconv_gather(gout, t.cout, NB, H, W, gg, st);
  k_to_bf16<<<nblk((long)t.cin * P), TPB, 0, st>>>(in, inb, (long)t.cin * P);
  const dim3 cg = chan_grid(4 * P, t.cout);
  k_chan_sum<<<cg, TPB, 0, st>>>(gout, 4 * P, u->red);
  k_chan_finish<<<t.cout, 32, 0, st>>>(u->red, (int)cg.x, u->g + t.b);
  count_launch(4);
  // dW[(cout*4)][cin] += gg[(cout*4)][P] in[cin][P]^T
  UTRY(bsct::gemm_bf16(false, true, t.cout * 4, t.cin, (int)P, 1.f, gg, P, 0, inb, P, 0, 1.f, u->g + t.w, t.cin, 0, 1,
                       st));
  // gin[cin][P] = W^T gg
  UTRY(bsct::gemm_bf16(true, false, t.cin, (int)P, t.cout * 4, 1.f, u->wb + t.w, t.cin, 0, gg, P, 0, 0.f, gin, P, 0, 1,
                       st));
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

}  // namespace

extern "C" int bsct_unet_create(int32_t base_channels, uint64_t seed, bsct_unet** out, void* stream) {
  if (!out || base_channels < 8 || base_channels % 8) {
    bsct_set_last_message("base_channels must be a positive multiple of 8");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  bsct_unet* u = new bsct_unet();
  const int B = base_channels;
  u->base = B;
  long o = 0;
  o = add_conv(u, u->c0a, 1, B, o);
  o = add_conv(u, u->c0b, B, B, o);
  o = add_conv(u, u->c1a, B, 2 * B, o);
  o = add_conv(u, u->c1b, 2 * B, 2 * B, o);
  o = add_conv(u, u->c2a, 2 * B, 4 * B, o);
  o = add_conv(u, u->c2b, 4 * B, 4 * B, o);
  o = add_conv(u, u->c3a, 4 * B, 8 * B, o);
  o = add_conv(u, u->c3b, 8 * B, 8 * B, o);
  o = add_tconv(u->t3, 8 * B, 4 * B, o);
  o = add_conv(u, u->d2a, 8 * B, 4 * B, o);
  o = add_conv(u, u->d2b, 4 * B, 4 * B, o);
  o = add_tconv(u->t2, 4 * B, 2 * B, o);
  o = add_conv(u, u->d1a, 4 * B, 2 * B, o);
  o = add_conv(u, u->d1b, 2 * B, 2 * B, o);
  o = add_tconv(u->t1, 2 * B, B, o);
  o = add_conv(u, u->d0a, 2 * B, B, o);
  o = add_conv(u, u->d0b, B, B, o);
  u->hw = o;
  o += B;
  u->hb = o;
  o += 1;
  o = ((o + 7) / 8) * 8;
  u->n_params = o;
  auto fail = [&](cudaError_t e) {
    bsct_set_last_cuda_error(e);
    cudaFree(u->w); cudaFree(u->g); cudaFree(u->m); cudaFree(u->v); cudaFree(u->wb);
    delete u;
    return BSCT_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&u->w, o * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&u->g, o * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&u->m, o * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&u->v, o * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&u->wb, o * 2)) != cudaSuccess) return fail(e);
  cudaMemsetAsync(u->w, 0, o * 4, st);
  cudaMemsetAsync(u->g, 0, o * 4, st);
  cudaMemsetAsync(u->m, 0, o * 4, st);
  cudaMemsetAsync(u->v, 0, o * 4, st);
  unsigned long long s = seed;
  auto init_conv = [&](const Conv3& c) {
    const long n = (long)c.cout * c.kpad;
    k_init_weights<<<nblk(n), TPB, 0, st>>>(u->w + c.w, n, c.kpad, 9 * c.cin, sqrtf(2.f / (9.f * c.cin)), ++s);
  };
  auto init_t = [&](const TConv& t) {
    const long n = (long)t.cout * 4 * t.cin;
    k_init_weights<<<nblk(n), TPB, 0, st>>>(u->w + t.w, n, t.cin, t.cin, sqrtf(1.f / t.cin), ++s);
  };
  for (const Conv3* c : {&u->c0a, &u->c0b, &u->c1a, &u->c1b, &u->c2a, &u->c2b, &u->c3a, &u->c3b, &u->d2a, &u->d2b,
                         &u->d1a, &u->d1b, &u->d0a, &u->d0b})
    init_conv(*c);
  init_t(u->t3);
  init_t(u->t2);
  init_t(u->t1);
  k_init_weights<<<1, TPB, 0, st>>>(u->w + u->hw, B, B, B, sqrtf(1.f / B), ++s);
  k_to_bf16<<<nblk(o), TPB, 0, st>>>(u->w, u->wb, o);
  count_launch(20);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  *out = u;
  return BSCT_OK;
}

extern "C" void bsct_unet_free(bsct_unet* u) {
  if (!u) return;
  cudaDeviceSynchronize();
  free_acts(u);
  cudaFree(u->w); cudaFree(u->g); cudaFree(u->m); cudaFree(u->v); cudaFree(u->wb);
  delete u;
}

extern "C" int bsct_unet_params(bsct_unet* u, float** d_params, float** d_grads, int64_t* n_params) {
  if (!u) { bsct_set_last_message("NULL net"); return BSCT_ERR_INVALID_ARG; }
  if (d_params) *d_params = u->w;
  if (d_grads) *d_grads = u->g;
  if (n_params) *n_params = u->n_params;
  return BSCT_OK;
}

extern "C" int bsct_unet_sync_weights(bsct_unet* u, void* stream) {
  if (!u) { bsct_set_last_message("NULL net"); return BSCT_ERR_INVALID_ARG; }
  k_to_bf16<<<nblk(u->n_params), TPB, 0, (cudaStream_t)stream>>>(u->w, u->wb, u->n_params);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

extern "C" int bsct_unet_forward(bsct_unet* u, const float* d_in, float* d_out, int32_t NB, int32_t H, int32_t W,
                                 void* stream) {
  if (!u || !d_in || !d_out || NB < 1 || H < 64 || W < 64 || H % 64 || W % 64) {
    bsct_set_last_message("U-Net input must be n x H x W with H, W multiples of 64");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  UTRY(alloc_acts(u, NB, H, W));
  const int B = u->base;
  const long P0 = (long)NB * H * W, P1 = P0 / 4, P2 = P0 / 16;
  BSCT_CUDA_TRY(cudaMemcpyAsync(u->x, d_in, P0 * 4, cudaMemcpyDeviceToDevice, st));
  // encoder (skip tensors written straight into the upper halves of the concat buffers)
  UTRY(conv_fwd(u, u->c0a, u->x, NB, H, W, u->a00, st));
  UTRY(conv_fwd(u, u->c0b, u->a00, NB, H, W, u->cat0 + B * P0, st));
  k_maxpool2<<<nblk(B * P1), TPB, 0, st>>>(u->cat0 + B * P0, B, NB, H, W, u->p0);
  UTRY(conv_fwd(u, u->c1a, u->p0, NB, H / 2, W / 2, u->a10, st));
  UTRY(conv_fwd(u, u->c1b, u->a10, NB, H / 2, W / 2, u->cat1 + 2 * B * P1, st));
  k_maxpool2<<<nblk(2 * B * P2), TPB, 0, st>>>(u->cat1 + 2 * B * P1, 2 * B, NB, H / 2, W / 2, u->p1);
  UTRY(conv_fwd(u, u->c2a, u->p1, NB, H / 4, W / 4, u->a20, st));
  UTRY(conv_fwd(u, u->c2b, u->a20, NB, H / 4, W / 4, u->cat2 + 4 * B * P2, st));
  k_maxpool2<<<nblk(4 * B * P2 / 4), TPB, 0, st>>>(u->cat2 + 4 * B * P2, 4 * B, NB, H / 4, W / 4, u->p2);
  count_launch(3);
  UTRY(conv_fwd(u, u->c3a, u->p2, NB, H / 8, W / 8, u->a30, st));
  UTRY(conv_fwd(u, u->c3b, u->a30, NB, H / 8, W / 8, u->a31, st));
  // decoder
  UTRY(tconv_fwd(u, u->t3, u->a31, NB, H / 8, W / 8, u->cat2, st));
  UTRY(conv_fwd(u, u->d2a, u->cat2, NB, H / 4, W / 4, u->u2a, st));
  UTRY(conv_fwd(u, u->d2b, u->u2a, NB, H / 4, W / 4, u->u2b, st));
  UTRY(tconv_fwd(u, u->t2, u->u2b, NB, H / 4, W / 4, u->cat1, st));
  UTRY(conv_fwd(u, u->d1a, u->cat1, NB, H / 2, W / 2, u->u1a, st));
  UTRY(conv_fwd(u, u->d1b, u->u1a, NB, H / 2, W / 2, u->u1b, st));
  UTRY(tconv_fwd(u, u->t1, u->u1b, NB, H / 2, W / 2, u->cat0, st));
  UTRY(conv_fwd(u, u->d0a, u->cat0, NB, H, W, u->u0a, st));
  UTRY(conv_fwd(u, u->d0b, u->u0a, NB, H, W, u->u0b, st));
  k_head_fwd<<<nblk(P0), TPB, 0, st>>>(u->u0b, u->w + u->hw, u->w + u->hb, B, P0, u->out);
  count_launch();
  BSCT_CUDA_TRY(cudaMemcpyAsync(d_out, u->out, P0 * 4, cudaMemcpyDeviceToDevice, st));
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

// gradient of the loss w.r.t. the last forward's output; accumulates parameter gradients
extern "C" int bsct_unet_backward(bsct_unet* u, const float* d_gout, void* stream) {
  if (!u || !d_gout || !u->NB) {
    bsct_set_last_message("backward needs a preceding forward");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int B = u->base, NB = u->NB, H = u->H, W = u->W;
  const long P0 = (long)NB * H * W, P1 = P0 / 4, P2 = P0 / 16;
  const dim3 hg = chan_grid(P0, B + 1);
  k_head_bwd_w<<<hg, TPB, 0, st>>>(u->u0b, d_gout, B, P0, u->red);
  k_chan_finish<<<B + 1, 32, 0, st>>>(u->red, (int)hg.x, u->g + u->hw, u->g + u->hb, B);
  k_head_bwd_data<<<nblk(B * P0), TPB, 0, st>>>(d_gout, u->w + u->hw, B, P0, u->gu0b);
  count_launch(3);
  UTRY(conv_bwd(u, u->d0b, u->u0a, u->u0b, u->gu0b, NB, H, W, u->gu0a, st));
  UTRY(conv_bwd(u, u->d0a, u->cat0, u->u0a, u->gu0a, NB, H, W, u->gcat0, st));
  UTRY(tconv_bwd(u, u->t1, u->u1b, u->gcat0, NB, H / 2, W / 2, u->gu1b, st));
  UTRY(conv_bwd(u, u->d1b, u->u1a, u->u1b, u->gu1b, NB, H / 2, W / 2, u->gu1a, st));
  UTRY(conv_bwd(u, u->d1a, u->cat1, u->u1a, u->gu1a, NB, H / 2, W / 2, u->gcat1, st));
  UTRY(tconv_bwd(u, u->t2, u->u2b, u->gcat1, NB, H / 4, W / 4, u->gu2b, st));
  UTRY(conv_bwd(u, u->d2b, u->u2a, u->u2b, u->gu2b, NB, H / 4, W / 4, u->gu2a, st));
  UTRY(conv_bwd(u, u->d2a, u->cat2, u->u2a, u->gu2a, NB, H / 4, W / 4, u->gcat2, st));
  UTRY(tconv_bwd(u, u->t3, u->a31, u->gcat2, NB, H / 8, W / 8, u->g31, st));
  UTRY(conv_bwd(u, u->c3b, u->a30, u->a31, u->g31, NB, H / 8, W / 8, u->g30, st));
  UTRY(conv_bwd(u, u->c3a, u->p2, u->a30, u->g30, NB, H / 8, W / 8, u->gp2, st));
  // e2 receives the skip gradient (upper half of gcat2) plus the pooled path
  k_maxpool2_bwd<<<nblk(4 * B * P2 / 4), TPB, 0, st>>>(u->cat2 + 4 * B * P2, u->gp2, 4 * B, NB, H / 4, W / 4,
                                                     u->gcat2 + 4 * B * P2);
  count_launch();
  UTRY(conv_bwd(u, u->c2b, u->a20, u->cat2 + 4 * B * P2, u->gcat2 + 4 * B * P2, NB, H / 4, W / 4, u->g20, st));
  UTRY(conv_bwd(u, u->c2a, u->p1, u->a20, u->g20, NB, H / 4, W / 4, u->gp1, st));
  k_maxpool2_bwd<<<nblk(2 * B * P2), TPB, 0, st>>>(u->cat1 + 2 * B * P1, u->gp1, 2 * B, NB, H / 2, W / 2,
                                                  u->gcat1 + 2 * B * P1);
  count_launch();
  UTRY(conv_bwd(u, u->c1b, u->a10, u->cat1 + 2 * B * P1, u->gcat1 + 2 * B * P1, NB, H / 2, W / 2, u->g10, st));
  UTRY(conv_bwd(u, u->c1a, u->p0, u->a10, u->g10, NB, H / 2, W / 2, u->gp0, st));
  k_maxpool2_bwd<<<nblk(B * P1), TPB, 0, st>>>(u->cat0 + B * P0, u->gp0, B, NB, H, W, u->gcat0 + B * P0);
  count_launch();
  UTRY(conv_bwd(u, u->c0b, u->a00, u->cat0 + B * P0, u->gcat0 + B * P0, NB, H, W, u->g00, st));
  UTRY(conv_bwd(u, u->c0a, u->x, u->a00, u->g00, NB, H, W, nullptr, st));
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

extern "C" int bsct_unet_adam_step(bsct_unet* u, float lr, float beta1, float beta2, float eps, int32_t step,
                                   void* stream) {
  if (!u || step < 1) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<nblk(u->n_params), TPB, 0, (cudaStream_t)stream>>>(u->w, u->g, u->m, u->v, u->wb, u->n_params, lr, beta1,
                                                              beta2, eps, c1, c2);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

// ---------------------------------------------------------------------------- warm start
namespace {
__global__ void k_scale_copy(const float* __restrict__ a, float s, float* __restrict__ b, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = s * a[i];
}
// Reproducible FP64 sums: every block reduces its values in a fixed order and writes one
// partial per sum, part[k * gridDim.x + block]; k_sum_parts then adds the partials of each
// sum in block order (the results do not depend on scheduling).
__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double red_d[TPB / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // red_d may still be read from a previous call
  if ((threadIdx.x & 31) == 0) red_d[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < TPB / 32; ++w) t += red_d[w];
  return t;
}
// out[k] = (accumulate ? out[k] : 0) + scale * sum_b part[k * nb + b], k < nsum (one warp each)
__global__ void k_sum_parts(const double* __restrict__ part, int nb, int nsum, double scale, int accumulate,
                            double* __restrict__ out) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= nsum) return;
  double acc = 0.0;
  for (int b = lane; b < nb; b += 32) acc += part[(long)k * nb + b];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[k] = (accumulate ? out[k] : 0.0) + scale * acc;
}
constexpr int DOT_BLOCKS = 512;

// part: [2][gridDim.x]; sums <a, b> and <a, c>
__global__ void __launch_bounds__(TPB) k_dot2(const float* __restrict__ a, const float* __restrict__ b,
                                              const float* __restrict__ c, long n, double* __restrict__ part) {
  double s0 = 0.0, s1 = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    s0 += (double)a[i] * b[i];
    s1 += (double)a[i] * c[i];
  }
  s0 = block_sum_d(s0);
  s1 = block_sum_d(s1);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
  }
}
}  // namespace

// x0 = alpha net(in_scale b) into d_x; *x0_zero = 1 when alpha is unusable (x0 = 0 then)
static int learned_warm_start(bsct_gram* g, bsct_unet* net, const void* d_b, void* d_x, float in_scale,
                              double* alpha_out, int* x0_zero, void* stream) {
  if (!g || !net || !d_b || !d_x) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  if (g->precision != BSCT_F32) { bsct_set_last_message("learned warm start needs an F32 handle"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const int N = g->N;
  const long n = (long)N * N;
  float* xin = (float*)g->q;   // CG scratch is free before the solve
  float* xhat = (float*)d_x;
  k_scale_copy<<<nblk(n), TPB, 0, st>>>((const float*)d_b, in_scale, xin, n);
  count_launch();
  UTRY(bsct_unet_forward(net, xin, xhat, 1, N, N, stream));
  float* Gx = (float*)g->r;
  UTRY(bsct_gram_apply(g, xhat, Gx, BSCT_APPLY_FFT32, stream));
  double* acc = g->partials;            // two doubles
  double* part = g->partials + 8;       // 2 x DOT_BLOCKS partials (g->partials holds 2048)
  k_dot2<<<DOT_BLOCKS, TPB, 0, st>>>(xhat, (const float*)d_b, Gx, n, part);
  k_sum_parts<<<1, 64, 0, st>>>(part, DOT_BLOCKS, 2, 1.0, 0, acc);
  count_launch(2);
  double h[2];
  BSCT_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
  BSCT_CUDA_TRY(cudaStreamSynchronize(st));
  // x0 = alpha xhat minimises the G-norm error along xhat; plain CG (x0 = 0) if it is unusable
  const double alpha = (h[1] > 0.0 && isfinite(h[0]) && isfinite(h[1])) ? h[0] / h[1] : 0.0;
  if (alpha_out) *alpha_out = alpha;
  *x0_zero = 1;
  if (alpha > 0.0 && isfinite(alpha)) {
    k_scale_copy<<<nblk(n), TPB, 0, st>>>(xhat, (float)alpha, xhat, n);
    count_launch();
    *x0_zero = 0;
  }
  return BSCT_OK;
}

extern "C" int bsct_cg_solve_learned(bsct_gram* g, bsct_unet* net, const void* d_b, void* d_x, float in_scale,
                                     int max_iter, double rel_tol, int check_every, bsct_cg_report* report,
                                     double* alpha_out, void* stream) {
  int x0_zero = 1;
  UTRY(learned_warm_start(g, net, d_b, d_x, in_scale, alpha_out, &x0_zero, stream));
  return bsct_cg_solve(g, d_b, d_x, x0_zero, max_iter, rel_tol, check_every, report, stream);
}

extern "C" int bsct_pcg_solve_learned(bsct_gram* g, bsct_unet* net, double eps, const void* d_b, void* d_x,
                                      float in_scale, int max_iter, double rel_tol, int check_every,
                                      bsct_cg_report* report, double* alpha_out, void* stream) {
  int x0_zero = 1;
  UTRY(learned_warm_start(g, net, d_b, d_x, in_scale, alpha_out, &x0_zero, stream));
  return bsct_pcg_solve(g, eps, d_b, d_x, x0_zero, max_iter, rel_tol, check_every, report, stream);
}

namespace {
// part[k][block] = block partial of <a_k, b_k> for k < 3 (0 for a null a_k)
__global__ void __launch_bounds__(TPB) k_dots3(const float* __restrict__ a0, const float* __restrict__ b0,
                                               const float* __restrict__ a1, const float* __restrict__ b1,
                                               const float* __restrict__ a2, const float* __restrict__ b2, long n,
                                               double* __restrict__ part) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    if (a0) s0 += (double)a0[i] * b0[i];
    if (a1) s1 += (double)a1[i] * b1[i];
    if (a2) s2 += (double)a2[i] * b2[i];
  }
  s0 = block_sum_d(s0);
  s1 = block_sum_d(s1);
  s2 = block_sum_d(s2);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
    part[2 * gridDim.x + blockIdx.x] = s2;
  }
}
// x += alpha p; r -= alpha q
__global__ void k_fcg_update(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                             const float* __restrict__ q, float alpha, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    x[i] = fmaf(alpha, p[i], x[i]);
    r[i] = fmaf(-alpha, q[i], r[i]);
  }
}
// p = z + beta p
__global__ void k_fcg_dir(float* __restrict__ p, const float* __restrict__ z, float beta, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[i] = fmaf(beta, p[i], z[i]);
}
// part[block] = block partial of sum (b - y)^2
__global__ void __launch_bounds__(TPB) k_resid2(const float* __restrict__ b, const float* __restrict__ y, long n,
                                                double* __restrict__ part) {
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double d = (double)b[i] - y[i];
    s += d * d;
  }
  s = block_sum_d(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
}  // namespace

// Flexible CG with the network as preconditioner (see bsct.h).  Host-driven: every dot
// product is read back, so the loop can branch on the fallback and the tolerance.
extern "C" int bsct_fcg_solve_learned(bsct_gram* g, bsct_unet* net, const void* d_b, void* d_x, float in_scale,
                                      int max_iter, double rel_tol, int precond_every, bsct_cg_report* report,
                                      int32_t* n_precond, int32_t* n_fallback, void* stream) {
  if (!g || !net || !d_b || !d_x || max_iter < 0 || precond_every < 1) {
    bsct_set_last_message("invalid argument");
    return BSCT_ERR_INVALID_ARG;
  }
  if (g->precision != BSCT_F32) { bsct_set_last_message("learned preconditioner needs an F32 handle"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const int N = g->N;
  const long n = (long)N * N;
  const unsigned nb = DOT_BLOCKS;
  const float* b = (const float*)d_b;
  float* x = (float*)d_x;
  float* r = (float*)g->r;
  float* p = (float*)g->p;
  float* q = (float*)g->q;
  float *z = nullptr, *xin = nullptr;
  double* acc = g->partials;             // 3 doubles
  double* part = g->partials + 8;        // 3 x DOT_BLOCKS block partials (g->partials holds 2048)
  int rc = BSCT_OK, npre = 0, nfb = 0, it = 0, conv = 0;
  double h[3], bb = 0.0, rr = 0.0;
  auto dots = [&](const float* a0, const float* b0, const float* a1, const float* b1, const float* a2,
                  const float* b2) -> int {
    k_dots3<<<nb, TPB, 0, st>>>(a0, b0, a1, b1, a2, b2, n, part);
    k_sum_parts<<<1, 96, 0, st>>>(part, (int)nb, 3, 1.0, 0, acc);
    count_launch(2);
    BSCT_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    BSCT_CUDA_TRY(cudaStreamSynchronize(st));
    return BSCT_OK;
  };
  // z = M(r) (network every precond_every iterations, else identity), with the fallback
  // z = r when <r, z> <= 0; returns <r, z> in *rz
  auto precondition = [&](int k, double* rz) -> int {
    if (k % precond_every == 0 && rr > 0.0) {
      const double s = sqrt(bb / rr);
      k_scale_copy<<<nblk(n), TPB, 0, st>>>(r, (float)(in_scale * s), xin, n);
      count_launch();
      int e = bsct_unet_forward(net, xin, z, 1, N, N, stream);
      if (e != BSCT_OK) return e;
      k_scale_copy<<<nblk(n), TPB, 0, st>>>(z, (float)(1.0 / s), z, n);
      count_launch();
      ++npre;
      e = dots(r, z, nullptr, nullptr, nullptr, nullptr);
      if (e != BSCT_OK) return e;
      if (h[0] > 0.0 && isfinite(h[0])) { *rz = h[0]; return BSCT_OK; }
      ++nfb;
    }
    BSCT_CUDA_TRY(cudaMemcpyAsync(z, r, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    *rz = rr;
    return BSCT_OK;
  };
  do {
    if (cudaMalloc(&z, n * sizeof(float)) != cudaSuccess || cudaMalloc(&xin, n * sizeof(float)) != cudaSuccess) {
      bsct_set_last_message("out of device memory");
      rc = BSCT_ERR_CUDA;
      break;
    }
    if ((rc = dots(b, b, nullptr, nullptr, nullptr, nullptr)) != BSCT_OK) break;
    bb = h[0];
    rr = bb;
    if (cudaMemsetAsync(x, 0, n * sizeof(float), st) != cudaSuccess ||
        cudaMemcpyAsync(r, b, n * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      rc = BSCT_ERR_CUDA;
      break;
    }
    if (bb == 0.0) { conv = 1; break; }
    double rz = 0.0;
    if ((rc = precondition(0, &rz)) != BSCT_OK) break;
    if (cudaMemcpyAsync(p, z, n * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess) { rc = BSCT_ERR_CUDA; break; }
    while (it < max_iter) {
      if ((rc = bsct_gram_apply(g, p, q, BSCT_APPLY_FFT32, stream)) != BSCT_OK) break;
      if ((rc = dots(p, q, p, r, nullptr, nullptr)) != BSCT_OK) break;
      const double pq = h[0], pr = h[1];
      if (!(pq > 0.0) || !isfinite(pq)) break;  // breakdown: p is (numerically) in G's null space
      const double alpha = pr / pq;
      k_fcg_update<<<nb, TPB, 0, st>>>(x, r, p, q, (float)alpha, n);
      count_launch();
      ++it;
      if ((rc = dots(r, r, nullptr, nullptr, nullptr, nullptr)) != BSCT_OK) break;
      rr = h[0];
      if (sqrt(rr / bb) <= rel_tol) { conv = 1; break; }
      if (it >= max_iter) break;
      if ((rc = precondition(it, &rz)) != BSCT_OK) break;
      if ((rc = dots(z, q, nullptr, nullptr, nullptr, nullptr)) != BSCT_OK) break;
      const double beta = -h[0] / pq;
      k_fcg_dir<<<nb, TPB, 0, st>>>(p, z, (float)beta, n);
      count_launch();
    }
  } while (0);
  if (rc == BSCT_OK && report) {
    report->iterations = it;
    report->converged = conv;
    report->rel_residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    report->true_rel_residual = -1.0;
    // true residual ||b - G x|| / ||b||
    if ((rc = bsct_gram_apply(g, x, q, BSCT_APPLY_FFT32, stream)) == BSCT_OK) {
      k_resid2<<<nb, TPB, 0, st>>>(b, q, n, part);
      k_sum_parts<<<1, 32, 0, st>>>(part, (int)nb, 1, 1.0, 0, acc);
      count_launch(2);
      if (cudaMemcpyAsync(h, acc, sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
          cudaStreamSynchronize(st) == cudaSuccess)
        report->true_rel_residual = bb > 0.0 ? sqrt(h[0] / bb) : 0.0;
    }
  }
  if (n_precond) *n_precond = npre;
  if (n_fallback) *n_fallback = nfb;
  cudaStreamSynchronize(st);
  if (z) cudaFree(z);
  if (xin) cudaFree(xin);
  return rc;
}

namespace {
// grad = 2 (pred - target) / n; part[block] = block partial of sum (pred - target)^2
// (k_sum_parts adds them, times 1/n, to the loss)
__global__ void __launch_bounds__(TPB) k_mse(const float* __restrict__ pred, const float* __restrict__ target, long n,
                                             float* __restrict__ grad, double* __restrict__ part) {
  double acc = 0.0;
  const float inv = 1.f / (float)n;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float d = pred[i] - target[i];
    grad[i] = 2.f * d * inv;
    acc += (double)d * d;
  }
  acc = block_sum_d(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
}  // namespace

extern "C" int bsct_mse_loss_grad(const float* d_pred, const float* d_target, int64_t n, float* d_grad, double* d_loss,
                                  void* stream) {
  if (!d_pred || !d_target || !d_grad || !d_loss || n < 1) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  LayerScratch sc{st};
  double* part = sc.get<double>(DOT_BLOCKS);
  if (!sc.ok) { bsct_set_last_message("out of device memory"); return BSCT_ERR_CUDA; }
  k_mse<<<DOT_BLOCKS, TPB, 0, st>>>(d_pred, d_target, n, d_grad, part);
  k_sum_parts<<<1, 32, 0, st>>>(part, DOT_BLOCKS, 1, 1.0 / (double)n, 1, d_loss);
  count_launch(2);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

// G-norm loss of a batch of images (a training loss matched to what CG needs):
//   loss += (1/n) sum_i w_i <e_i, G e_i>,  grad_i = (2 w_i / n) G e_i,  e_i = pred_i - target_i
namespace {
constexpr int GN_BLOCKS = 64;
__global__ void k_sub(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ c, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) c[i] = a[i] - b[i];
}
// part[img][blk] = partial <e_img, ge_img> (grid: GN_BLOCKS x n_img)
__global__ void k_gn_dot(const float* __restrict__ e, const float* __restrict__ ge, long m, double* __restrict__ part) {
  const long off = (long)blockIdx.y * m;
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long)gridDim.x * blockDim.x)
    acc += (double)e[off + i] * (double)ge[off + i];
  __shared__ double red[TPB / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < TPB / 32; ++w) t += red[w];
    part[blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}
// one thread: loss += (1/n) sum_i w_i sum_b part[i][b] (fixed order: reproducible)
__global__ void k_gn_fin(const double* __restrict__ part, const double* __restrict__ w, int n, double* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double tot = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int b = 0; b < GN_BLOCKS; ++b) s += part[i * GN_BLOCKS + b];
    tot += (w ? w[i] : 1.0) * s;
  }
  *loss += tot / n;
}
__global__ void k_gn_scale(float* __restrict__ g, const double* __restrict__ w, long m, int n) {
  const long total = m * n;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
    g[i] *= (float)(2.0 * (w ? w[i / m] : 1.0) / n);
}
}  // namespace

extern "C" int bsct_gnorm_loss_grad(const bsct_gram* g, const float* d_pred, const float* d_target, int32_t n,
                                    const double* d_weight, float* d_grad, double* d_loss, void* stream) {
  if (!g || !d_pred || !d_target || !d_grad || !d_loss || n < 1 || g->precision != BSCT_F32) {
    bsct_set_last_message("invalid argument (F32 handle, n >= 1, non-NULL buffers)");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long m = (long)g->N * g->N;
  LayerScratch sc{st};
  float* e = sc.get<float>(m * n);
  double* part = sc.get<double>((long)GN_BLOCKS * n);
  if (!sc.ok) { bsct_set_last_message("out of device memory"); return BSCT_ERR_CUDA; }
  k_sub<<<nblk(m * n) < 4096 ? nblk(m * n) : 4096, TPB, 0, st>>>(d_pred, d_target, e, m * n);
  count_launch();
  for (int i = 0; i < n; ++i) {
    const int rc = bsct_gram_apply(g, e + (long)i * m, d_grad + (long)i * m, BSCT_APPLY_FFT32, stream);
    if (rc != BSCT_OK) return rc;
  }
  k_gn_dot<<<dim3(GN_BLOCKS, n), TPB, 0, st>>>(e, d_grad, m, part);
  k_gn_fin<<<1, 32, 0, st>>>(part, d_weight, n, d_loss);
  k_gn_scale<<<nblk(m * n) < 4096 ? nblk(m * n) : 4096, TPB, 0, st>>>(d_grad, d_weight, m, n);
  count_launch(3);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

// copy the FP32 parameters (which = 0) or gradients (which = 1) to / from caller memory
extern "C" int bsct_unet_copy(bsct_unet* u, int which, int to_net, float* d_buf, void* stream) {
  if (!u || !d_buf || which < 0 || which > 1) { bsct_set_last_message("invalid argument"); return BSCT_ERR_INVALID_ARG; }
  float* net = which == 0 ? u->w : u->g;
  cudaStream_t st = (cudaStream_t)stream;
  if (to_net) {
    BSCT_CUDA_TRY(cudaMemcpyAsync(net, d_buf, u->n_params * 4, cudaMemcpyDeviceToDevice, st));
    if (which == 0) return bsct_unet_sync_weights(u, stream);
  } else {
    BSCT_CUDA_TRY(cudaMemcpyAsync(d_buf, net, u->n_params * 4, cudaMemcpyDeviceToDevice, st));
  }
  return BSCT_OK;
}

// ---------------------------------------------------------------------------- single layers
// The network's layers on their own (for checking them one by one against the oracle):
// the same kernels and GEMMs, with scratch from the stream-ordered allocator.

extern "C" int bsct_conv3x3_forward(int32_t n, int32_t cin, int32_t cout, int32_t H, int32_t W, const float* d_in,
                                    const float* d_w, const float* d_b, int relu, float* d_out, void* stream) {
  if (!d_in || !d_w || !d_b || !d_out || !layer_dims_ok(n, cin, cout, H, W)) {
    bsct_set_last_message("invalid layer arguments (cout and n H W must be multiples of 8)");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int kpad = ((9 * cin + 7) / 8) * 8;
  const long P = (long)n * H * W;
  LayerScratch sc{st};
  bf16* wb = sc.get<bf16>((long)cout * kpad);
  bf16* col = sc.get<bf16>((long)kpad * P);
  if (!sc.ok) { bsct_set_last_message("out of device memory"); return BSCT_ERR_CUDA; }
  k_to_bf16<<<nblk((long)cout * kpad), TPB, 0, st>>>(d_w, wb, (long)cout * kpad);
  launch_im2col3(d_in, cin, n, H, W, kpad, col, st);
  count_launch(2);
  UTRY(bsct::gemm_bf16(false, false, cout, (int)P, kpad, 1.f, wb, kpad, 0, col, P, 0, 0.f, d_out, P, 0, 1, st));
  launch_bias_relu(d_out, d_b, cout, P, relu ? 1 : 0, st);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

extern "C" int bsct_conv3x3_backward(int32_t n, int32_t cin, int32_t cout, int32_t H, int32_t W, const float* d_in,
                                     const float* d_w, const float* d_out, const float* d_gout, int relu, float* d_gin,
                                     float* d_gw, float* d_gb, void* stream) {
  if (!d_in || !d_w || !d_gout || !d_gw || !d_gb || (relu && !d_out) || !layer_dims_ok(n, cin, cout, H, W)) {
    bsct_set_last_message("invalid layer arguments (cout and n H W must be multiples of 8)");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int kpad = ((9 * cin + 7) / 8) * 8;
  const long P = (long)n * H * W;
  LayerScratch sc{st};
  bf16* wb = sc.get<bf16>((long)cout * kpad);
  bf16* col = sc.get<bf16>((long)kpad * P);
  bf16* dpre = sc.get<bf16>((long)cout * P);
  float* dcol = d_gin ? sc.get<float>((long)kpad * P) : nullptr;
  float* red = sc.get<float>(chan_parts(P, cout));
  if (!sc.ok) { bsct_set_last_message("out of device memory"); return BSCT_ERR_CUDA; }
  BSCT_CUDA_TRY(cudaMemsetAsync(d_gb, 0, (size_t)cout * sizeof(float), st));
  k_to_bf16<<<nblk((long)cout * kpad), TPB, 0, st>>>(d_w, wb, (long)cout * kpad);
  const dim3 cg = chan_grid(P, cout);
  k_relu_bwd<<<cg, TPB, 0, st>>>(d_gout, relu ? d_out : d_gout, P, dpre, red, relu ? 1 : 0);
  k_chan_finish<<<cout, 32, 0, st>>>(red, (int)cg.x, d_gb);
  launch_im2col3(d_in, cin, n, H, W, kpad, col, st);
  count_launch(4);
  UTRY(bsct::gemm_bf16(false, true, cout, kpad, (int)P, 1.f, dpre, P, 0, col, P, 0, 0.f, d_gw, kpad, 0, 1, st));
  if (d_gin) {
    UTRY(bsct::gemm_bf16(true, false, kpad, (int)P, cout, 1.f, wb, kpad, 0, dpre, P, 0, 0.f, dcol, P, 0, 1, st));
    launch_col2im3(dcol, cin, n, H, W, d_gin, st);
    count_launch();
  }
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

extern "C" int bsct_tconv2x2_forward(int32_t n, int32_t cin, int32_t cout, int32_t H, int32_t W, const float* d_in,
                                     const float* d_w, const float* d_b, float* d_out, void* stream) {
  if (!d_in || !d_w || !d_b || !d_out || !layer_dims_ok(n, cin, cout, H, W) || cin % 8) {
    bsct_set_last_message("invalid layer arguments (cin, cout and n H W must be multiples of 8)");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long P = (long)n * H * W;
  LayerScratch sc{st};
  bf16* wb = sc.get<bf16>((long)cout * 4 * cin);
  bf16* inb = sc.get<bf16>((long)cin * P);
  float* tmp = sc.get<float>((long)cout * 4 * P);
  if (!sc.ok) { bsct_set_last_message("out of device memory"); return BSCT_ERR_CUDA; }
  k_to_bf16<<<nblk((long)cout * 4 * cin), TPB, 0, st>>>(d_w, wb, (long)cout * 4 * cin);
  k_to_bf16<<<nblk((long)cin * P), TPB, 0, st>>>(d_in, inb, (long)cin * P);
  count_launch(2);
  UTRY(bsct::gemm_bf16(false, false, cout * 4, (int)P, cin, 1.f, wb, cin, 0, inb, P, 0, 0.f, tmp, P, 0, 1, st));
  launch_tconv_scatter(tmp, d_b, cout, n, H, W, d_out, st);
  count_launch();
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

extern "C" int bsct_tconv2x2_backward(int32_t n, int32_t cin, int32_t cout, int32_t H, int32_t W, const float* d_in,
                                      const float* d_w, const float* d_gout, float* d_gin, float* d_gw, float* d_gb,
                                      void* stream) {
  if (!d_in || !d_w || !d_gout || !d_gw || !d_gb || !layer_dims_ok(n, cin, cout, H, W) || cin % 8) {
    bsct_set_last_message("invalid layer arguments (cin, cout and n H W must be multiples of 8)");
    return BSCT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long P = (long)n * H * W;
  LayerScratch sc{st};
  bf16* wb = sc.get<bf16>((long)cout * 4 * cin);
  bf16* gg = sc.get<bf16>((long)cout * 4 * P);
  bf16* inb = sc.get<bf16>((long)cin * P);
  float* red = sc.get<float>(chan_parts(4 * P, cout));
  if (!sc.ok) { bsct_set_last_message("out of device memory"); return BSCT_ERR_CUDA; }
  BSCT_CUDA_TRY(cudaMemsetAsync(d_gb, 0, (size_t)cout * sizeof(float), st));
  k_to_bf16<<<nblk((long)cout * 4 * cin), TPB, 0, st>>>(d_w, wb, (long)cout * 4 * cin);
  launch_tconv_gather(d_gout, cout, n, H, W, gg, st);
  k_to_bf16<<<nblk((long)cin * P), TPB, 0, st>>>(d_in, inb, (long)cin * P);
  const dim3 cg = chan_grid(4 * P, cout);
  k_chan_sum<<<cg, TPB, 0, st>>>(d_gout, 4 * P, red);
  k_chan_finish<<<cout, 32, 0, st>>>(red, (int)cg.x, d_gb);
  count_launch(5);
  UTRY(bsct::gemm_bf16(false, true, cout * 4, cin, (int)P, 1.f, gg, P, 0, inb, P, 0, 0.f, d_gw, cin, 0, 1, st));
  if (d_gin)
    UTRY(bsct::gemm_bf16(true, false, cin, (int)P, cout * 4, 1.f, wb, cin, 0, gg, P, 0, 0.f, d_gin, P, 0, 1, st));
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}
