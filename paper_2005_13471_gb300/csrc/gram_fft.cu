// Gram apply as a zero-padded 2N x 2N FFT convolution (Sec. 4: G is Toeplitz-block-
// Toeplitz, so G x is a linear convolution with the (2N-1)^2 filter, computed exactly by
// a circular convolution on the doubled grid).  Compiled once per image size with
// -DBSCT_FFT_N=<N>.
//
// Three HBM passes per apply:
//   K5 rows_r2c   : each image row (N reals, zero-padded to 2N) -> N packed complex
//                   half-spectrum values (Nyquist real part stored in the imaginary
//                   slot of the DC bin), via one N-point complex FFT of the even/odd
//                   interleaved row.
//   K6 cols_conv  : each of the N packed columns: 2N-point FFT of the N non-zero rows,
//                   times the real spectrum of G, inverse 2N-point FFT, keep N rows.
//                   Column 0 carries the (DC, Nyquist) pair and is separated and
//                   recombined with the two spectrum columns in the frequency domain.
//   K7 rows_c2r   : inverse of K5, keeping the first N outputs of each row.
// The half spectra live in a row-block interleaved layout, element (row, v) at
// ((row/4) * N + v) * 4 + row%4, so K5/K7 stream whole 4-row blocks and K6 reads
// 32-byte row segments per column.
#include "bsct_fft.cuh"
#include "bsct_fft2.cuh"
#include "bsct_internal.h"

#ifndef BSCT_FFT_N
#error "compile with -DBSCT_FFT_N=<N>"
#endif

namespace bsct {

__host__ __device__ constexpr int threads_per_fft(int L, int E) { return L / E; }

// rows handled per CTA of the forward row kernel: at least 4 (one row block, so its
// stores fill whole 32-byte sectors of the interleaved spectra) and at least ~128 threads
template <int LR> __host__ __device__ constexpr int rows_per_cta() {
  return (LR / Plan<LR>::E) >= 32 ? 4 : ((128 / (LR / Plan<LR>::E)) > LR ? LR : (128 / (LR / Plan<LR>::E)));
}
// rows per CTA of the inverse row kernel: long rows go two per CTA (half of a row block;
// its reads hit spectra the column kernel has just left in L2), so the rows spread
// evenly over the SMs instead of leaving a partial second wave of 4-row CTAs
template <int LR> __host__ __device__ constexpr int rows_per_cta_inv() {
  return (LR / Plan<LR>::E) >= 64 ? 2 : rows_per_cta<LR>();
}
// rows of one 4-row block that a CTA of RPC rows touches (2 or 4)
template <int RPC> __host__ __device__ constexpr int rows_per_group() { return RPC < 4 ? 2 : 4; }

// columns per CTA
template <typename T, int LC> __host__ __device__ constexpr int cols_per_cta() {
  return (LC / Plan<LC>::E) >= 256 ? (sizeof(T) == 4 ? 2 : 1)
                                   : ((256 / (LC / Plan<LC>::E)) > 8 ? 8 : (256 / (LC / Plan<LC>::E)));
}

// per-row shared region of the row kernels: the FFT buffer plus 32/RB words (RB = rows of
// a 4-row block in the CTA), so that those rows start on different banks (the untangle
// phase touches the same index of all of them in one warp)
template <typename T, int LR, int RPC> __host__ __device__ constexpr int row_region() {
  return smem_elems<LR>() + (32 / rows_per_group<RPC>()) / (int)(sizeof(cpx<T>) / 4);
}

__device__ __forceinline__ long blk_index(int row, int col, int ncols) {
  return ((long)(row >> 2) * ncols + col) * 4 + (row & 3);
}

// ------------------------------------------------------------------------------------
// K5: real rows -> packed half spectra.  PADDED: the row holds LR reals (zero-padded to
// 2 LR); otherwise it holds 2 LR reals.  Row r of x starts at x + r * ld_x.
// ------------------------------------------------------------------------------------
// CG: the row is p_new = x + beta * p_old (x = the CG residual r), written to p_new
// and transformed (the CG direction update fused into the first FFT pass)
// status (may be null): a non-finite input value sets *status = 1 (the input check of
// the public apply; one FMA per loaded value and a warp vote)
template <typename T, int LR, bool PADDED, int RPC, bool CG = false>
__global__ void __launch_bounds__(RPC * (LR / Plan<LR>::E))
k_rows_r2c(const T* __restrict__ x, long ld_x, cpx<T>* __restrict__ S,
           const cpx<T>* __restrict__ tsf, const cpx<T>* __restrict__ twc, const T* p_old = nullptr,
           T* p_new = nullptr, const double* __restrict__ cg_beta = nullptr, unsigned int* status = nullptr) {
  constexpr int E = Plan<LR>::E, TT = LR / E, R1 = Plan<LR>::R[0], RL = Plan<LR>::R[Plan<LR>::NS - 1];
  constexpr int SME = row_region<T, LR, RPC>();
  static_assert(R1 % 2 == 0, "zero-padding / crop split needs an even first radix");
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* sm_all = reinterpret_cast<cpx<T>*>(smraw);
  const int f = threadIdx.x / TT, tid = threadIdx.x % TT;
  const int row0 = blockIdx.x * RPC;
  cpx<T>* sm = sm_all + f * SME;
  const cpx<T>* z = reinterpret_cast<const cpx<T>*>(x + (long)(row0 + f) * ld_x);
  const cpx<T>* zp = CG ? reinterpret_cast<const cpx<T>*>(p_old + (long)(row0 + f) * ld_x) : nullptr;
  cpx<T>* zn = CG ? reinterpret_cast<cpx<T>*>(p_new + (long)(row0 + f) * ld_x) : nullptr;
  pdl_trigger();
  pdl_wait();
  const T beta = CG ? T(__ldcg(cg_beta)) : T(0);

  cpx<T> v[E];
  T chk = T(0);  // stays 0 unless an input value is infinite or NaN (x * 0 = NaN)
#pragma unroll
  for (int b = 0; b < E / R1; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      if (PADDED && r >= R1 / 2) {
        v[b * R1 + r] = mk(T(0), T(0));  // z[n] = 0 for n >= LR/2 (never read)
      } else if constexpr (CG) {
        const int n = j + r * (LR / R1);
        const cpx<T> a = ld_cpx_cg(z + n), pp = ld_cpx_cg(zp + n);
        const cpx<T> pn = mk(fma(beta, pp.x, a.x), fma(beta, pp.y, a.y));
        st_cpx(zn + n, pn);
        v[b * R1 + r] = pn;
      } else {
        v[b * R1 + r] = ld_cpx_cg(z + j + r * (LR / R1));
        if (status) chk = fma(v[b * R1 + r].y, T(0), fma(v[b * R1 + r].x, T(0), chk));
      }
    }
  }
  if (!CG && status) {
    if (__any_sync(__activemask(), chk != chk) && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
  }
  fft<T, LR, false, false, PADDED>(v, sm, tid, tsf);
#pragma unroll
  for (int b = 0; b < E / RL; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < RL; ++r) sm[spad(j + r * (LR / RL))] = v[b * RL + r];
  }
  __syncthreads();
  // untangle Z = FFT(x_even + i x_odd) into X[v] = E[v] + W^v O[v], two bins per item:
  // E and O are spectra of real sequences, and W^(LR - v) = -conj(W^v), so
  // X[LR - v] = conj(E[v] - W^v O[v]); item v = 0 gives the packed (X[0], X[LR]) and
  // X[LR/2] = conj(Z[LR/2]).  Stores of both bins are coalesced (ascending / descending).
  constexpr int HL = LR / 2, RB = rows_per_group<RPC>();
#pragma unroll 4
  for (int it = 0; it < E / 2; ++it) {
    const int e = threadIdx.x + it * (RPC * TT);
    const int rr = e % RB, vv = (e / RB) % HL, lr = (e / RB) / HL * RB + rr, row = row0 + lr;
    const cpx<T>* smf = sm_all + lr * SME;
    cpx<T>* o = S + (long)(row >> 2) * LR * 4 + (row & 3);
    const cpx<T> Z = smf[spad(vv)];
    if (vv == 0) {
      const cpx<T> Zh = smf[spad(HL)];
      st_cpx(o, mk(Z.x + Z.y, Z.x - Z.y));  // (X[0], X[LR]) both real
      st_cpx(o + HL * 4, conj(Zh));
    } else {
      const cpx<T> Zm = conj(smf[spad(LR - vv)]);
      const cpx<T> Ev = scale(Z + Zm, T(0.5));
      const cpx<T> WO = cmul(scale(mul_mi<T, false>(Z - Zm), T(0.5)), ld_cpx(twc + vv));
      st_cpx(o + vv * 4, Ev + WO);
      st_cpx(o + (LR - vv) * 4, conj(Ev - WO));
    }
  }
}

// ------------------------------------------------------------------------------------
// K7: packed half spectra -> real rows, first LR outputs of 2 LR (crop)
// ------------------------------------------------------------------------------------
// RED != 0: also accumulate <p, y> over the block (p = the apply's input) into
// part[blockIdx.x]; the last CTA turns the sum into the step scalars of CG (RED_ALPHA)
// or of preconditioned CG (RED_RHO)
enum { RED_NONE = 0, RED_ALPHA = 1, RED_RHO = 2 };
template <typename T, int LR, int RPC, int RED = RED_NONE>
__global__ void __launch_bounds__(RPC * (LR / Plan<LR>::E))
k_rows_c2r(const cpx<T>* __restrict__ S, T* __restrict__ y, long ld_y,
           const cpx<T>* __restrict__ tsr, const cpx<T>* __restrict__ twc, const T* __restrict__ p = nullptr,
           double* __restrict__ part = nullptr, double* __restrict__ sc = nullptr) {
  constexpr int E = Plan<LR>::E, TT = LR / E, R1 = Plan<LR>::R[0], RL = Plan<LR>::R[Plan<LR>::NS - 1];
  constexpr int SME = row_region<T, LR, RPC>();
  static_assert(R1 % 2 == 0, "zero-padding / crop split needs an even first radix");
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* sm_all = reinterpret_cast<cpx<T>*>(smraw);
  const int f = threadIdx.x / TT, tid = threadIdx.x % TT;
  const int row0 = blockIdx.x * RPC;
  cpx<T>* sm = sm_all + f * SME;

  // inverse untangle straight from the half spectra, two bins per item: with
  // Ev = Y[v] + conj(Y[LR-v]) and Od = (Y[v] - conj(Y[LR-v])) conj(W^v), the row FFT input
  // is Zp[v] = Ev + i Od and Zp[LR - v] = conj(Ev - i Od); item v = 0 also gives
  // Zp[LR/2] = 2 conj(Y[LR/2]).  All loads of a thread are issued together.
  constexpr int HL = LR / 2, RB = rows_per_group<RPC>();
  pdl_trigger();
  pdl_wait();
#pragma unroll
  for (int it = 0; it < E / 2; ++it) {
    const int e = threadIdx.x + it * (RPC * TT);
    const int rr = e % RB, vv = (e / RB) % HL, lr = (e / RB) / HL * RB + rr, row = row0 + lr;
    const cpx<T>* ir = S + (long)(row >> 2) * LR * 4 + (row & 3);
    cpx<T>* smf = sm_all + lr * SME;
    const cpx<T> Y = ld_cpx_cg(ir + vv * 4);
    const cpx<T> Yo = ld_cpx_cg(ir + (vv == 0 ? HL : LR - vv) * 4);
    if (vv == 0) {
      smf[spad(0)] = mk(Y.x + Y.y, Y.x - Y.y);
      smf[spad(HL)] = mk(Yo.x + Yo.x, -(Yo.y + Yo.y));
    } else {
      const cpx<T> Ym = conj(Yo);
      const cpx<T> Ev = Y + Ym;
      const cpx<T> iOd = mul_mi<T, true>(cmulc(Y - Ym, ld_cpx(twc + vv)));
      smf[spad(vv)] = Ev + iOd;
      smf[spad(LR - vv)] = conj(Ev - iOd);
    }
  }
  __syncthreads();
  // the inverse runs the plan reversed: its first radix is the plan's last (RF) and its
  // last radix is the plan's first (R1, always even), so the crop m < LR/2 is r < R1/2
  constexpr int RF = RL;
  cpx<T> v[E];
#pragma unroll
  for (int b = 0; b < E / RF; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < RF; ++r) v[b * RF + r] = sm[spad(j + r * (LR / RF))];
  }
  __syncthreads();
  fft<T, LR, true, true>(v, sm, tid, tsr);
  cpx<T>* yr = reinterpret_cast<cpx<T>*>(y + (long)(row0 + f) * ld_y);
  T dot = T(0);
#pragma unroll
  for (int b = 0; b < E / R1; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < R1 / 2; ++r) {
      st_cpx(yr + j + r * (LR / R1), v[b * R1 + r]);
      if constexpr (RED != RED_NONE) {
        const cpx<T> pp = ld_cpx_cg(reinterpret_cast<const cpx<T>*>(p + (long)(row0 + f) * ld_y) + j + r * (LR / R1));
        dot = fma(pp.x, v[b * R1 + r].x, fma(pp.y, v[b * R1 + r].y, dot));
      }
    }
  }
  if constexpr (RED != RED_NONE) {
    // block sum in FP64 (the per-thread part is <= 16 products)
    constexpr int NTH = RPC * TT;
    double d = (double)dot;
    __syncthreads();  // the exchange buffer is free: reuse it for the partial sums
    double* ws = reinterpret_cast<double*>(sm_all);
    if constexpr (NTH % 32 == 0) {
      for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
      if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = d;
      __syncthreads();
      if (threadIdx.x < 32) {
        constexpr int NW = NTH / 32;
        double t = threadIdx.x < NW ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
      }
    } else {
      ws[threadIdx.x] = d;  // blocks of fewer than 32 threads (N = 16)
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < NTH; ++i) t += ws[i];
        part[blockIdx.x] = t;
      }
    }
    last_block_sum(part, sc_counter(sc, SC_CNT_PQ), ws, [&](double t) {
      if constexpr (RED == RED_ALPHA) {
        // <p, q> and alpha = <r, r> / <p, q> (0 when <p, q> <= 0)
        sc[SC_PQ] = t;
        sc[SC_ALPHA] = t > 0.0 ? __ldcg(sc + SC_RR) / t : 0.0;
      } else {
        // rho_new = <r, M^-1 r>, beta = rho_new / rho (0 before the first step)
        const double rho = __ldcg(sc + SC_RR);
        sc[SC_BETA] = rho > 0.0 ? t / rho : 0.0;
        sc[SC_RR] = t;
      }
    });
  }
}

// ------------------------------------------------------------------------------------
// K6: per packed column: forward 2N FFT (rows >= N are zero), multiply by the real
// spectrum, inverse, keep rows < N.  In place on S.
// Persistent CTAs walk over tiles of G columns; while a tile is transformed, the
// column data (32-byte row-block chunks) and spectrum rows of the next tile are already
// in flight into shared memory (cp.async), so HBM/L2 latency overlaps the FFT arithmetic.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N_> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N_) : "memory");
}

template <typename T, int LC, int G> __host__ __device__ constexpr int cols_threads() { return G * (LC / Plan<LC>::E); }
template <typename T, int LC, int G> __host__ __device__ constexpr size_t cols_smem() {
  return (size_t)G * smem_elems<LC>() * sizeof(cpx<T>) + (size_t)G * (LC / 2) * sizeof(cpx<T>) +
         (size_t)G * LC * sizeof(T);
}

// Shared memory: the FFT exchange buffers, one staging buffer for the next tile's column
// data and one for its spectrum columns.  The column data is consumed at the start of a
// tile and the spectrum after the forward FFT, so each buffer is refilled (one cp.async
// group each) right after it is consumed and has a whole tile of compute to arrive.
// Keeping to one staging set leaves L1 room for the stage twiddle table.
template <typename T, int LC, int G, int MINB>
__global__ void __launch_bounds__(G*(LC / Plan<LC>::E), MINB)
k_cols_conv(cpx<T>* __restrict__ S, const T* __restrict__ Gt, const cpx<T>* __restrict__ tsf,
            const cpx<T>* __restrict__ tsr, int ntiles) {
  constexpr int E = Plan<LC>::E, TT = LC / E, R1 = Plan<LC>::R[0], RL = Plan<LC>::R[Plan<LC>::NS - 1];
  constexpr int NT = G * TT;
  constexpr int NC = LC / 2;
  constexpr int SME = smem_elems<LC>();
  constexpr int IN_E = G * NC;  // complex per tile
  constexpr int GT_E = G * LC;  // reals per tile
  constexpr int PPC = 4 * (int)sizeof(cpx<T>) / 16;  // 16-byte pieces per 4-row chunk
  constexpr int RPP = 16 / (int)sizeof(cpx<T>);      // rows per piece
  static_assert(R1 % 2 == 0, "zero-padding / crop split needs an even first radix");
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* xsm = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* stin = xsm + G * SME;
  T* stg = reinterpret_cast<T*>(stin + IN_E);
  const int g = threadIdx.x / TT, tid = threadIdx.x % TT;
  cpx<T>* sm = xsm + g * SME;

  auto prefetch_in = [&](int tile) {
    if (tile < ntiles) {
      const int c0 = tile * G;
      for (int q = threadIdx.x; q < (NC / 4) * G * PPC; q += NT) {
        const int p = q % PPC, gc = (q / PPC) % G, k = q / (PPC * G);
        cp_async16(stin + gc * NC + 4 * k + p * RPP, S + ((long)k * NC + c0 + gc) * 4 + p * RPP);
      }
    }
    cp_async_commit();
  };
  auto prefetch_spec = [&](int tile) {
    if (tile < ntiles) {
      const T* src = Gt + (long)tile * G * LC;
      constexpr int EPP = 16 / (int)sizeof(T);
      for (int q = threadIdx.x; q < GT_E / EPP; q += NT) cp_async16(stg + q * EPP, src + q * EPP);
    }
    cp_async_commit();
  };

  int tile = blockIdx.x;
  pdl_trigger();
  // FP32 palindromic plans: the stage twiddles of this thread, the same for every tile and
  // (conjugated) for the inverse, go to registers once; constant data, so before the wait
  constexpr bool TWREG = sizeof(T) == 4 && plan_palindrome<LC>();
  TwCache<T, LC> twr;
  if constexpr (TWREG) tw_cache_load<T, LC, false>(twr, tid, tsf);
  pdl_wait();
  prefetch_in(tile);
  prefetch_spec(tile);
  // cp.async groups in commit order: in(t0), spec(t0), in(t1), spec(t1), ...; each wait
  // below leaves only the most recent group in flight
  for (; tile < ntiles; tile += gridDim.x) {
    cp_async_wait<1>();  // column data of this tile
    __syncthreads();
    const int col = tile * G + g;
    const cpx<T>* in = stin + g * NC;
    cpx<T> v[E];
#pragma unroll
    for (int b = 0; b < E / R1; ++b) {
      const int j = tid + b * TT;
#pragma unroll
      for (int r = 0; r < R1; ++r)
        v[b * R1 + r] = (r < R1 / 2) ? in[j + r * (LC / R1)] : mk(T(0), T(0));  // rows >= N are zero
    }
    __syncthreads();  // column staging consumed
    prefetch_in(tile + gridDim.x);
    if constexpr (TWREG) fft_cached<T, LC, false, false, true>(v, sm, tid, tsf, twr);
    else fft<T, LC, false, false, true>(v, sm, tid, tsf);
    cp_async_wait<1>();  // spectrum of this tile
    __syncthreads();
    const T* gs = stg + g * LC;
    if (tile == 0) {
      // column 0 holds a + i b (a = DC column, b = Nyquist column): needs Z[-u]
#pragma unroll
      for (int b = 0; b < E / RL; ++b) {
        const int j = tid + b * TT;
#pragma unroll
        for (int r = 0; r < RL; ++r) sm[spad(j + r * (LC / RL))] = v[b * RL + r];
      }
      __syncthreads();
#pragma unroll
      for (int b = 0; b < E / RL; ++b) {
        const int j = tid + b * TT;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int u = j + r * (LC / RL);
          const cpx<T> Z = v[b * RL + r];
          if (col == 0) {
            const int um = (u == 0) ? 0 : LC - u;
            const cpx<T> Zm = conj(sm[spad(um)]);
            const T P = gs[u], Q = Gt[(long)NC * LC + u];
            v[b * RL + r] = mk(P * Z.x + Q * Zm.x, P * Z.y + Q * Zm.y);
          } else {
            const T gv = gs[u];
            v[b * RL + r] = mk(gv * Z.x, gv * Z.y);
          }
        }
      }
    } else {
#pragma unroll
      for (int b = 0; b < E / RL; ++b) {
        const int j = tid + b * TT;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const T gv = gs[j + r * (LC / RL)];
          v[b * RL + r] = mk(gv * v[b * RL + r].x, gv * v[b * RL + r].y);
        }
      }
    }
    __syncthreads();  // spectrum staging (and, for tile 0, the exchange buffer) consumed
    prefetch_spec(tile + gridDim.x);
    if constexpr (TWREG) fft_cached<T, LC, true, true>(v, sm, tid, tsr, twr);
    else fft<T, LC, true, true>(v, sm, tid, tsr);
    // reversed plan: last radix = forward first radix R1; keep rows < N
#pragma unroll
    for (int b = 0; b < E / R1; ++b) {
      const int j = tid + b * TT;
#pragma unroll
      for (int r = 0; r < R1 / 2; ++r) st_cpx(S + blk_index(j + r * (LC / R1), col, NC), v[b * R1 + r]);
    }
  }
  cp_async_wait<0>();
}

// ------------------------------------------------------------------------------------
// Spectrum: per packed column, forward 2N FFT over all 2N rows, real part -> Gt (scaled)
// ------------------------------------------------------------------------------------
template <typename T, int LC, int CPC>
__global__ void __launch_bounds__(CPC * (LC / Plan<LC>::E))
k_cols_fwd_real(const cpx<T>* __restrict__ S2, T* __restrict__ Gt, const cpx<T>* __restrict__ tsf, T sc) {
  constexpr int E = Plan<LC>::E, TT = LC / E, R1 = Plan<LC>::R[0], RL = Plan<LC>::R[Plan<LC>::NS - 1];
  constexpr int NC = LC / 2;
  constexpr int SME = smem_elems<LC>();
  static_assert(R1 % 2 == 0, "zero-padding / crop split needs an even first radix");
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* sm_all = reinterpret_cast<cpx<T>*>(smraw);
  const int f = threadIdx.x / TT, tid = threadIdx.x % TT;
  const int col = blockIdx.x * CPC + f;
  cpx<T>* sm = sm_all + f * SME;

  cpx<T> v[E];
#pragma unroll
  for (int b = 0; b < E / R1; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < R1; ++r) v[b * R1 + r] = ld_cpx(S2 + blk_index(j + r * (LC / R1), col, NC));
  }
  fft<T, LC, false, false>(v, sm, tid, tsf);
  if (blockIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < E / RL; ++b) {
      const int j = tid + b * TT;
#pragma unroll
      for (int r = 0; r < RL; ++r) sm[spad(j + r * (LC / RL))] = v[b * RL + r];
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < E / RL; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int u = j + r * (LC / RL);
      const cpx<T> Z = v[b * RL + r];
      if (blockIdx.x == 0 && f == 0) {
        const int um = (u == 0) ? 0 : LC - u;
        const cpx<T> Zn = sm[spad(um)];     // Z[-u]
        const T g0 = T(0.5) * (Z.x + Zn.x);  // Re of DC-column spectrum
        const T gN = T(0.5) * (Z.y + Zn.y);  // Re of Nyquist-column spectrum
        Gt[u] = T(0.5) * (g0 + gN) * sc;
        Gt[(long)NC * LC + u] = T(0.5) * (g0 - gN) * sc;
      } else {
        Gt[(long)col * LC + u] = Z.x * sc;
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// FP32 path: the same three passes on the paired FFT of bsct_fft2.cuh.  Row passes
// transform two image rows per group of threads (rows r, r+1 in the two lanes); the
// column pass transforms columns v and v + N/2 of the half spectra together.  The half
// spectra live as column pairs: S2[p * N + row] (p < N/2) holds (X_row[p], X_row[p + N/2])
// in the lanes of one 16-byte value, X_row[0] being the packed (DC, Nyquist) pair.  The
// untangling pairs bins v and LR - v (LR = N), and the set {v, LR - v, N/2 - v, N/2 + v}
// is closed, so one item of the row passes produces or consumes whole column pairs.
// ------------------------------------------------------------------------------------

// shared words per image row in the row passes: the FFT buffer of a row pair (RS values of
// 16 bytes) holds the two rows' regions of RS complex values each during the untangling;
// RS = 16/RPC (mod 16) puts the RPC rows of one item group on distinct banks
template <int LR, int RPC> __host__ __device__ constexpr int row_stride2() {
  return smem_elems<LR>() + (((16 / RPC) % 16 - smem_elems<LR>() % 16) % 16 + 16) % 16;
}
template <int LR, int RPC> __host__ __device__ constexpr size_t rows_smem2() {
  return (size_t)RPC * row_stride2<LR, RPC>() * sizeof(cpx<float>);
}

// untangling of one bin pair (v, LR - v) of a row, 0 < v < LR/2: Z = FFT(x_even + i x_odd)
// -> X[v], X[LR - v] (half spectrum of the real row)
__device__ __forceinline__ void untangle_fwd(cpx<float> Z, cpx<float> Zo, cpx<float> w, cpx<float>& Xv,
                                             cpx<float>& Xm) {
  const cpx<float> Zm = conj(Zo);
  const cpx<float> Ev = scale(Z + Zm, 0.5f);
  const cpx<float> WO = cmul(scale(mul_mi<float, false>(Z - Zm), 0.5f), w);
  Xv = Ev + WO;
  Xm = conj(Ev - WO);
}
// the inverse: half spectrum bins Y[v], Y[LR - v] -> row FFT inputs Zp[v], Zp[LR - v]
__device__ __forceinline__ void untangle_inv(cpx<float> Y, cpx<float> Yo, cpx<float> w, cpx<float>& Zv,
                                             cpx<float>& Zm) {
  const cpx<float> Ym = conj(Yo);
  const cpx<float> Ev = Y + Ym;
  const cpx<float> iOd = mul_mi<float, true>(cmulc(Y - Ym, w));
  Zv = Ev + iOd;
  Zm = conj(Ev - iOd);
}
__device__ __forceinline__ void st_c2_lanes(c2* p, cpx<float> a, cpx<float> b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, b.x, a.y, b.y);
}
__device__ __forceinline__ void ld_c2_lanes(const c2* p, cpx<float>& a, cpx<float>& b) {
  const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
  a = mk(t.x, t.z);
  b = mk(t.y, t.w);
}

// K5 (FP32): real rows -> column-pair half spectra.  CG: the rows are p_new = x + beta p_old
// (written back), as in k_rows_r2c.  status: see k_rows_r2c.
template <int LR, int RPC, bool CG = false>
__global__ void __launch_bounds__((RPC / 2) * (LR / Plan<LR>::E))
k2_rows_r2c(const float* __restrict__ x, c2* __restrict__ S2, const cpx<float>* __restrict__ tsf,
            const cpx<float>* __restrict__ twc, const float* p_old, float* p_new, const double* __restrict__ cg_beta,
            unsigned int* status) {
  constexpr int E = Plan<LR>::E, TT = LR / E, R1 = Plan<LR>::R[0], RL = Plan<LR>::R[Plan<LR>::NS - 1];
  constexpr int RS = row_stride2<LR, RPC>(), NT = (RPC / 2) * TT, NR = LR;  // image rows = LR
  static_assert(R1 % 2 == 0, "zero-padding split needs an even first radix");
  extern __shared__ __align__(16) unsigned char smraw[];
  c2* smp = reinterpret_cast<c2*>(smraw);
  cpx<float>* smr = reinterpret_cast<cpx<float>*>(smraw);
  const int f = threadIdx.x / TT, tid = threadIdx.x % TT;
  const int row0 = blockIdx.x * RPC;
  c2* sm = smp + f * RS;
  const cpx<float>* z0 = reinterpret_cast<const cpx<float>*>(x + (long)(row0 + 2 * f) * NR);
  const cpx<float>* z1 = z0 + NR / 2;
  pdl_trigger();
  pdl_wait();
  const float beta = CG ? float(__ldcg(cg_beta)) : 0.f;

  c2 v[E];
  float2 chk = make_float2(0.f, 0.f);  // stays 0 unless an input is infinite or NaN
#pragma unroll
  for (int b = 0; b < E / R1; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int n = j + r * (LR / R1);
      if (r >= R1 / 2) {
        v[b * R1 + r] = c2zero();  // z[n] = 0 for n >= LR/2 (never read)
      } else if constexpr (CG) {
        const cpx<float>* q0 = reinterpret_cast<const cpx<float>*>(p_old + (long)(row0 + 2 * f) * NR);
        cpx<float>* n0 = reinterpret_cast<cpx<float>*>(p_new + (long)(row0 + 2 * f) * NR);
        const c2 a = c2pack(ld_cpx_cg(z0 + n), ld_cpx_cg(z1 + n));
        const c2 pp = c2pack(ld_cpx_cg(q0 + n), ld_cpx_cg(q0 + NR / 2 + n));
        const c2 pn = c2{fma2(bc2(beta), pp.re, a.re), fma2(bc2(beta), pp.im, a.im)};
        st_cpx(n0 + n, c2lane0(pn));
        st_cpx(n0 + NR / 2 + n, c2lane1(pn));
        v[b * R1 + r] = pn;
      } else {
        v[b * R1 + r] = c2pack(ld_cpx_cg(z0 + n), ld_cpx_cg(z1 + n));
        chk = fma2(v[b * R1 + r].im, bc2(0.f), fma2(v[b * R1 + r].re, bc2(0.f), chk));
      }
    }
  }
  if (!CG && status) {
    const bool bad = chk.x != chk.x || chk.y != chk.y;
    if (__any_sync(__activemask(), bad) && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
  }
  fft2<LR, false, false, true>(v, sm, tid, tsf);
  // outputs in natural order, one region per row
  cpx<float>* ra = smr + (2 * f) * RS;
  cpx<float>* rb = ra + RS;
#pragma unroll
  for (int b = 0; b < E / RL; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int k = spad(j + r * (LR / RL));
      ra[k] = c2lane0(v[b * RL + r]);
      rb[k] = c2lane1(v[b * RL + r]);
    }
  }
  __syncthreads();
  // items (row, v), v < LR/4: v = 0 makes column pairs 0 and LR/4, v > 0 makes pairs v and
  // LR/2 - v; consecutive threads take consecutive rows (coalesced 16-byte stores)
  constexpr int H = LR / 2, Q = LR / 4;
#pragma unroll
  for (int it = 0; it < E / 2; ++it) {
    const int e = threadIdx.x + it * NT;
    const int lr = e % RPC, vv = e / RPC, row = row0 + lr;
    const cpx<float>* zr = smr + lr * RS;
    if (vv == 0) {
      const cpx<float> Z0 = zr[spad(0)], Zh = zr[spad(H)];
      st_c2_lanes(S2 + row, mk(Z0.x + Z0.y, Z0.x - Z0.y), conj(Zh));  // (X[0], X[LR]) and X[LR/2]
      cpx<float> Xq, X3q;
      untangle_fwd(zr[spad(Q)], zr[spad(3 * Q)], ld_cpx(twc + Q), Xq, X3q);
      st_c2_lanes(S2 + (long)Q * NR + row, Xq, X3q);
    } else {
      const int u = H - vv;
      cpx<float> Xv, Xmv, Xu, Xmu;  // X[v], X[LR - v], X[u], X[LR - u] (LR - u = v + LR/2)
      untangle_fwd(zr[spad(vv)], zr[spad(LR - vv)], ld_cpx(twc + vv), Xv, Xmv);
      untangle_fwd(zr[spad(u)], zr[spad(LR - u)], ld_cpx(twc + u), Xu, Xmu);
      st_c2_lanes(S2 + (long)vv * NR + row, Xv, Xmu);
      st_c2_lanes(S2 + (long)u * NR + row, Xu, Xmv);
    }
  }
}

// K7 (FP32): column-pair half spectra -> real rows (first LR outputs of 2 LR).  RED as in
// k_rows_c2r (p = the apply's input, for <p, y>).
template <int LR, int RPC, int RED = RED_NONE>
__global__ void __launch_bounds__((RPC / 2) * (LR / Plan<LR>::E))
k2_rows_c2r(const c2* __restrict__ S2, float* __restrict__ y, const cpx<float>* __restrict__ tsr,
            const cpx<float>* __restrict__ twc, const float* __restrict__ p, double* __restrict__ part,
            double* __restrict__ sc) {
  constexpr int E = Plan<LR>::E, TT = LR / E, R1 = Plan<LR>::R[0], RL = Plan<LR>::R[Plan<LR>::NS - 1];
  constexpr int RS = row_stride2<LR, RPC>(), NT = (RPC / 2) * TT, NR = LR;
  static_assert(R1 % 2 == 0, "crop split needs an even first radix");
  extern __shared__ __align__(16) unsigned char smraw[];
  c2* smp = reinterpret_cast<c2*>(smraw);
  cpx<float>* smr = reinterpret_cast<cpx<float>*>(smraw);
  const int f = threadIdx.x / TT, tid = threadIdx.x % TT;
  const int row0 = blockIdx.x * RPC;
  c2* sm = smp + f * RS;
  constexpr int H = LR / 2, Q = LR / 4;
  pdl_trigger();
  pdl_wait();
  // inverse untangling straight from the column pairs (the loop is unrolled so that all
  // loads of a thread are in flight together)
#pragma unroll
  for (int it = 0; it < E / 2; ++it) {
    const int e = threadIdx.x + it * NT;
    const int lr = e % RPC, vv = e / RPC, row = row0 + lr;
    cpx<float>* zr = smr + lr * RS;
    if (vv == 0) {
      cpx<float> Y0, Yh, Yq, Y3q;
      ld_c2_lanes(S2 + row, Y0, Yh);
      ld_c2_lanes(S2 + (long)Q * NR + row, Yq, Y3q);
      zr[spad(0)] = mk(Y0.x + Y0.y, Y0.x - Y0.y);
      zr[spad(H)] = mk(Yh.x + Yh.x, -(Yh.y + Yh.y));
      cpx<float> Zq, Z3q;
      untangle_inv(Yq, Y3q, ld_cpx(twc + Q), Zq, Z3q);
      zr[spad(Q)] = Zq;
      zr[spad(3 * Q)] = Z3q;
    } else {
      const int u = H - vv;
      cpx<float> Yv, Ymu, Yu, Ymv;  // pair v holds (Y[v], Y[LR - u]), pair u holds (Y[u], Y[LR - v])
      ld_c2_lanes(S2 + (long)vv * NR + row, Yv, Ymu);
      ld_c2_lanes(S2 + (long)u * NR + row, Yu, Ymv);
      cpx<float> Zv, Zmv, Zu, Zmu;
      untangle_inv(Yv, Ymv, ld_cpx(twc + vv), Zv, Zmv);
      untangle_inv(Yu, Ymu, ld_cpx(twc + u), Zu, Zmu);
      zr[spad(vv)] = Zv;
      zr[spad(LR - vv)] = Zmv;
      zr[spad(u)] = Zu;
      zr[spad(LR - u)] = Zmu;
    }
  }
  __syncthreads();
  // the inverse runs the plan reversed: first radix RL, last radix R1 (crop: r < R1/2)
  constexpr int RF = RL;
  const cpx<float>* ra = smr + (2 * f) * RS;
  const cpx<float>* rb = ra + RS;
  c2 v[E];
#pragma unroll
  for (int b = 0; b < E / RF; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < RF; ++r) {
      const int k = spad(j + r * (LR / RF));
      v[b * RF + r] = c2pack(ra[k], rb[k]);
    }
  }
  __syncthreads();
  fft2<LR, true, true>(v, sm, tid, tsr);
  cpx<float>* y0 = reinterpret_cast<cpx<float>*>(y + (long)(row0 + 2 * f) * NR);
  cpx<float>* y1 = y0 + NR / 2;
  float dot = 0.f;
#pragma unroll
  for (int b = 0; b < E / R1; ++b) {
    const int j = tid + b * TT;
#pragma unroll
    for (int r = 0; r < R1 / 2; ++r) {
      const int n = j + r * (LR / R1);
      const cpx<float> a = c2lane0(v[b * R1 + r]), c = c2lane1(v[b * R1 + r]);
      st_cpx(y0 + n, a);
      st_cpx(y1 + n, c);
      if constexpr (RED != RED_NONE) {
        const cpx<float>* p0 = reinterpret_cast<const cpx<float>*>(p + (long)(row0 + 2 * f) * NR);
        const cpx<float> pa = ld_cpx_cg(p0 + n), pc = ld_cpx_cg(p0 + NR / 2 + n);
        dot = fmaf(pa.x, a.x, fmaf(pa.y, a.y, dot));
        dot = fmaf(pc.x, c.x, fmaf(pc.y, c.y, dot));
      }
    }
  }
  if constexpr (RED != RED_NONE) {
    double d = (double)dot;
    __syncthreads();  // the exchange buffer is free: reuse it for the partial sums
    double* ws = reinterpret_cast<double*>(smraw);
    if constexpr (NT % 32 == 0) {
      for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
      if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = d;
      __syncthreads();
      if (threadIdx.x < 32) {
        constexpr int NW = NT / 32;
        double t = threadIdx.x < NW ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
      }
    } else {
      ws[threadIdx.x] = d;  // blocks of fewer than 32 threads
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < NT; ++i) t += ws[i];
        part[blockIdx.x] = t;
      }
    }
    last_block_sum(part, sc_counter(sc, SC_CNT_PQ), ws, [&](double t) {
      if constexpr (RED == RED_ALPHA) {
        sc[SC_PQ] = t;
        sc[SC_ALPHA] = t > 0.0 ? __ldcg(sc + SC_RR) / t : 0.0;
      } else {
        const double rho = __ldcg(sc + SC_RR);
        sc[SC_BETA] = rho > 0.0 ? t / rho : 0.0;
        sc[SC_RR] = t;
      }
    });
  }
}

// K6 (FP32): per column pair (v, v + N/2): forward 2N FFT of the N non-zero rows, times
// the spectrum columns, inverse, keep rows < N; in place on S2.  Persistent CTAs walk over
// tiles of G pairs; the spectrum rows of the next tile are copied into shared memory
// (cp.async) while the current tile's inverse transform runs, and column data is read from
// L2 (the row pass has just written it).
template <int LC, int G> __host__ __device__ constexpr size_t cols_smem2() {
  return (size_t)G * smem_elems<LC>() * sizeof(c2) + (size_t)G * 2 * LC * sizeof(float);
}
template <int LC, int G, int MINB>
__global__ void __launch_bounds__(G*(LC / Plan<LC>::E), MINB)
k2_cols_conv(c2* __restrict__ S2, const float* __restrict__ Gt, const cpx<float>* __restrict__ tsf,
             const cpx<float>* __restrict__ tsr, int ntiles) {
  constexpr int E = Plan<LC>::E, TT = LC / E, R1 = Plan<LC>::R[0], RL = Plan<LC>::R[Plan<LC>::NS - 1];
  constexpr int NT = G * TT, NR = LC / 2, NP = LC / 4;  // image rows, column pairs
  constexpr int SME = smem_elems<LC>();
  static_assert(R1 % 2 == 0, "zero-padding / crop split needs an even first radix");
  extern __shared__ __align__(16) unsigned char smraw[];
  c2* xsm = reinterpret_cast<c2*>(smraw);
  float* stg = reinterpret_cast<float*>(xsm + G * SME);  // [G][2][LC]: spectrum rows v, v + N/2
  const int g = threadIdx.x / TT, tid = threadIdx.x % TT;
  c2* sm = xsm + g * SME;

  auto prefetch_spec = [&](int tile) {
    if (tile < ntiles) {
      for (int q = threadIdx.x; q < G * 2 * (LC / 4); q += NT) {
        const int c = q / (LC / 4), k = q % (LC / 4);  // c = 2 * gp + lane
        const int pp = tile * G + c / 2;
        const float* src = Gt + (long)(pp + (c & 1) * NP) * LC + 4 * k;
        cp_async16(stg + (long)c * LC + 4 * k, src);
      }
    }
    cp_async_commit();
  };

  // column data of a tile -> this group's exchange buffer at the padded positions the
  // first stage reads (cp.async; every thread copies the 16-byte values it will read)
  auto prefetch_cols = [&](int t) {
    if (t < ntiles) {
      const c2* src = S2 + (long)(t * G + g) * NR;
#pragma unroll
      for (int b = 0; b < E / R1; ++b) {
        const int j = tid + b * TT;
#pragma unroll
        for (int r = 0; r < R1 / 2; ++r) cp_async16(sm + spad(j + r * (LC / R1)), src + j + r * (LC / R1));
      }
    }
    cp_async_commit();
  };

  int tile = blockIdx.x;
  pdl_trigger();
  constexpr bool TWREG = plan_palindrome<LC>();
  TwCache<float, LC> twr;
  if constexpr (TWREG) tw_cache_load<float, LC, false>(twr, tid, tsf);
  pdl_wait();
  prefetch_cols(tile);
  prefetch_spec(tile);
  // cp.async groups in commit order: cols(t0), spec(t0), then per tile spec(t+1), cols(t+1).
  // The first tile waits for its column data only (its spectrum arrives during the forward
  // transform); later tiles' groups both had the previous inverse transform to arrive.
  bool first = true;
  for (; tile < ntiles; tile += gridDim.x) {
    const int pr = tile * G + g;  // column pair of this thread group
    if (first) cp_async_wait<1>();
    else cp_async_wait<0>();
    first = false;
    __syncthreads();
    c2 v[E];
#pragma unroll
    for (int b = 0; b < E / R1; ++b) {
      const int j = tid + b * TT;
#pragma unroll
      for (int r = 0; r < R1; ++r)
        v[b * R1 + r] = r < R1 / 2 ? ld_c2(sm + spad(j + r * (LC / R1))) : c2zero();  // rows >= N are zero
    }
    __syncthreads();  // the buffer is the first exchange's
    if constexpr (TWREG) fft2_cached<LC, false, false, true>(v, sm, tid, tsf, twr);
    else fft2<LC, false, false, true>(v, sm, tid, tsf);
    cp_async_wait<0>();  // spectrum rows of this tile (already complete after the first tile)
    __syncthreads();
    const float* gs0 = stg + (long)(2 * g) * LC;
    const float* gs1 = gs0 + LC;
    if (tile == 0) {
      // pair 0 (group 0 of tile 0): lane 0 is the packed (DC + i Nyquist) column and needs
      // its value at -u; every group stages its values so that the barrier is uniform
#pragma unroll
      for (int b = 0; b < E / RL; ++b) {
        const int j = tid + b * TT;
#pragma unroll
        for (int r = 0; r < RL; ++r) st_c2(sm + spad(j + r * (LC / RL)), v[b * RL + r]);
      }
      __syncthreads();
#pragma unroll
      for (int b = 0; b < E / RL; ++b) {
        const int j = tid + b * TT;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int u = j + r * (LC / RL);
          const c2 Z = v[b * RL + r];
          if (pr == 0) {
            const int um = (u == 0) ? 0 : LC - u;
            const c2 Zn = ld_c2(sm + spad(um));
            const float P = gs0[u], Qv = Gt[(long)NR * LC + u], g1 = gs1[u];
            v[b * RL + r] = c2{make_float2(P * Z.re.x + Qv * Zn.re.x, g1 * Z.re.y),
                               make_float2(P * Z.im.x - Qv * Zn.im.x, g1 * Z.im.y)};
          } else {
            const float2 gv = make_float2(gs0[u], gs1[u]);
            v[b * RL + r] = c2{mul2(Z.re, gv), mul2(Z.im, gv)};
          }
        }
      }
    } else {
#pragma unroll
      for (int b = 0; b < E / RL; ++b) {
        const int j = tid + b * TT;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int u = j + r * (LC / RL);
          const float2 gv = make_float2(gs0[u], gs1[u]);
          v[b * RL + r] = c2{mul2(v[b * RL + r].re, gv), mul2(v[b * RL + r].im, gv)};
        }
      }
    }
    __syncthreads();  // spectrum staging (and, for pair 0, the exchange buffer) consumed
    prefetch_spec(tile + gridDim.x);
    // the next tile's column data starts arriving while the last inverse stage runs
    auto next_cols = [&]() { prefetch_cols(tile + gridDim.x); };
    if constexpr (TWREG) fft2_cached<LC, true, true>(v, sm, tid, tsr, twr, next_cols);
    else fft2<LC, true, true>(v, sm, tid, tsr, next_cols);
    c2* out = S2 + (long)pr * NR;
#pragma unroll
    for (int b = 0; b < E / R1; ++b) {
      const int j = tid + b * TT;
#pragma unroll
      for (int r = 0; r < R1 / 2; ++r) st_c2(out + j + r * (LC / R1), v[b * R1 + r]);
    }
  }
  cp_async_wait<0>();
}

// ------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------
template <typename K> static int set_smem(K kern, size_t bytes) {
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) { bsct_set_last_cuda_error(e); return BSCT_ERR_CUDA; }
  }
  return BSCT_OK;
}
// twiddle tables of one size N, packed in one array (see FftTables)
template <typename T> struct TwPtrs {
  const cpx<T>*untangle, *rows_f, *rows_r, *cols_f, *cols_r;
};
template <typename T, int N> __host__ inline TwPtrs<T> tw_ptrs(const cpx<T>* tw) {
  TwPtrs<T> p;
  p.untangle = tw;
  p.rows_f = tw + 2 * N;
  p.rows_r = plan_palindrome<N>() ? p.rows_f : tw + 3 * N;  // identical tables
  p.cols_f = tw + 4 * N;
  p.cols_r = plan_palindrome<2 * N>() ? p.cols_f : tw + 6 * N;
  return p;
}

template <typename T, int LC> struct ColsCfg {
  static constexpr int TT = LC / Plan<LC>::E;
  static constexpr int G = TT >= 256 ? 1 : (256 / TT > LC / 2 ? LC / 2 : 256 / TT);
  static constexpr int MINB = (cols_smem<T, LC, G>() * 2 <= 227 * 1024 && sizeof(T) == 4) ? 2 : 1;
};

// One-time launch setup (shared-memory attributes, persistent grid sizes) is cached per
// device, so one process may drive several GPUs.
constexpr int MAX_DEVICES = 64;
static int device_slot() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev < 0 ? 0 : (dev < MAX_DEVICES ? dev : MAX_DEVICES - 1);
}
static int sm_count() {
  static int n[MAX_DEVICES] = {};
  const int d = device_slot();
  if (n[d] == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n[d] = v > 0 ? v : 1;
  }
  return n[d];
}

// ------------------------------------------------------------------------------------
// Launch shapes.  The forward row pass takes RPC image rows per CTA, the inverse row
// pass RPI, the persistent column pass up to its occupancy limit of CTAs per SM (or
// one).  Each row count has three candidates around the measured default (half, the
// default, double; those that do not fit a CTA are invalid); bsct_fft_autotune times
// them.  The choice is kept per device and precision; every shape computes the same
// numbers (the rows are transformed identically, only their grouping changes).
// ------------------------------------------------------------------------------------
template <int D> __host__ __device__ constexpr int shape_cand(int i) { return i == 0 ? D / 2 : (i == 1 ? D : 2 * D); }
template <typename T, int LR, int RP> __host__ __device__ constexpr bool rows_ok() {
  return RP >= 2 && (RP == 2 || RP % 4 == 0) && LR % RP == 0 && RP * (LR / Plan<LR>::E) <= 1024 &&
         (size_t)RP * row_region<T, LR, RP>() * sizeof(cpx<T>) <= 227 * 1024;
}
// FP32 (paired) row passes: about 256 threads per CTA forward (two rows per LR/E threads);
// long rows go one pair per CTA in the inverse pass
template <int LR> __host__ __device__ constexpr int rows_per_cta2() {
  return (512 / (LR / Plan<LR>::E)) < 2 ? 2 : ((512 / (LR / Plan<LR>::E)) > LR ? LR : (512 / (LR / Plan<LR>::E)));
}
template <int LR> __host__ __device__ constexpr int rows_per_cta_inv2() {
  return (LR / Plan<LR>::E) >= 64 ? 2 : rows_per_cta2<LR>();
}
template <int LR, int RP> __host__ __device__ constexpr bool rows_ok2() {
  return RP >= 2 && (RP == 2 || RP % 4 == 0) && LR % RP == 0 && (RP / 2) * (LR / Plan<LR>::E) <= 1024 &&
         rows_smem2<LR, RP>() <= 227 * 1024;
}
template <typename T, int LR> __host__ __device__ constexpr int def_rows_fwd() {
  return sizeof(T) == 4 ? rows_per_cta2<LR>() : rows_per_cta<LR>();
}
template <typename T, int LR> __host__ __device__ constexpr int def_rows_inv() {
  return sizeof(T) == 4 ? rows_per_cta_inv2<LR>() : rows_per_cta_inv<LR>();
}
template <typename T, int LR, int RP> __host__ __device__ constexpr bool rows_valid() {
  if constexpr (sizeof(T) == 4) return rows_ok2<LR, RP>();
  else return rows_ok<T, LR, RP>();
}
template <int LC> struct ColsCfg2 {
  static constexpr int TT = LC / Plan<LC>::E;
  static constexpr int G = TT >= 256 ? 1 : (256 / TT > LC / 4 ? LC / 4 : 256 / TT);
  static constexpr int MINB = cols_smem2<LC, G>() * 2 <= 227 * 1024 ? 2 : 1;
};

struct Shape {
  int fwd = 1, inv = 1, cols = 0;  // candidate indices; cols: 0 = occupancy limit, 1 = one CTA per SM
};
static Shape g_shape[MAX_DEVICES][2];
template <typename T> static Shape& cur_shape() { return g_shape[device_slot()][sizeof(T) == 4 ? 0 : 1]; }

enum { AP_PLAIN = 0, AP_CG = 1, AP_PC = 2 };

// One apply y = G x (or M^-1 x) in three passes.
//   AP_PLAIN: out = G in.
//   AP_CG:    K5 forms p = in + beta p (beta = sc[SC_BETA]), writes it back and transforms
//             it; K7 writes out = G p and reduces <p, out> into alpha (RED_ALPHA).
//   AP_PC:    out = M^-1 in with spectrum Gt = the preconditioner's; K7 reduces <in, out>
//             into beta and rho (RED_RHO).
template <typename T, int N, int MODE, int RPC, int RPI>
static int run_apply(const T* in, T* p, T* out, double* sc, double* part, cpx<T>* S, const T* Gt,
                     const cpx<T>* tw, int cols, cudaStream_t st) {
  constexpr int LR = N, LC = 2 * N;
  typedef ColsCfg<T, LC> CC;
  static_assert(N % CC::G == 0, "tile must divide N");
  constexpr int TR = RPC * (LR / Plan<LR>::E), TI = RPI * (LR / Plan<LR>::E), TC = cols_threads<T, LC, CC::G>();
  constexpr size_t smr = (size_t)RPC * row_region<T, LR, RPC>() * sizeof(cpx<T>);
  constexpr size_t smi = (size_t)RPI * row_region<T, LR, RPI>() * sizeof(cpx<T>);
  constexpr size_t smc = cols_smem<T, LC, CC::G>();
  constexpr int RED = MODE == AP_CG ? RED_ALPHA : (MODE == AP_PC ? RED_RHO : RED_NONE);
  auto k5 = k_rows_r2c<T, LR, true, RPC, MODE == AP_CG>;
  auto k7 = k_rows_c2r<T, LR, RPI, RED>;
  auto kc = k_cols_conv<T, LC, CC::G, CC::MINB>;
  static int per_sm_max[MAX_DEVICES] = {};  // 0 until this instance's launch setup is done
  const int d = device_slot();
  if (per_sm_max[d] == 0) {
    int rc = set_smem(k5, smr);
    if (rc == BSCT_OK) rc = set_smem(k7, smi);
    if (rc == BSCT_OK) rc = set_smem(kc, smc);
    if (rc != BSCT_OK) return rc;
    int per_sm = 0;
    BSCT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kc, TC, smc));
    per_sm_max[d] = per_sm < 1 ? 1 : per_sm;
  }
  const int per_sm = cols == 1 ? 1 : per_sm_max[d];
  const int tiles = N / CC::G;
  const int grid_c = per_sm * sm_count() < tiles ? per_sm * sm_count() : tiles;
  const TwPtrs<T> t = tw_ptrs<T, N>(tw);
  const T* k7_in = MODE == AP_CG ? (const T*)p : (MODE == AP_PC ? in : (const T*)nullptr);
  if (MODE == AP_PLAIN) timer_mark(st, 0);
  if constexpr (MODE == AP_CG)
    BSCT_CUDA_TRY(launch_overlap(k5, dim3(N / RPC), dim3(TR), smr, st, in, (long)N, S, t.rows_f, t.untangle,
                                 (const T*)p, p, (const double*)(sc + SC_BETA), (unsigned int*)nullptr));
  else
    BSCT_CUDA_TRY(launch_overlap(k5, dim3(N / RPC), dim3(TR), smr, st, in, (long)N, S, t.rows_f, t.untangle,
                                 (const T*)nullptr, (T*)nullptr, (const double*)nullptr,
                                 MODE == AP_PLAIN ? input_status_ptr() : (unsigned int*)nullptr));
  if (MODE == AP_PLAIN) timer_mark(st, 1);
  BSCT_CUDA_TRY(launch_overlap(kc, dim3(grid_c), dim3(TC), smc, st, S, Gt, t.cols_f, t.cols_r, N / CC::G));
  if (MODE == AP_PLAIN) timer_mark(st, 2);
  BSCT_CUDA_TRY(launch_overlap(k7, dim3(N / RPI), dim3(TI), smi, st, (const cpx<T>*)S, out, (long)N, t.rows_r,
                               t.untangle, k7_in, MODE == AP_PLAIN ? (double*)nullptr : part,
                               MODE == AP_PLAIN ? (double*)nullptr : sc));
  if (MODE == AP_PLAIN) timer_mark(st, 3);
  count_launch(3);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

// FP32: the paired kernels (column-pair layout of S)
template <int N, int MODE, int RPC, int RPI>
static int run_apply2(const float* in, float* p, float* out, double* sc, double* part, cpx<float>* S, const float* Gt,
                      const cpx<float>* tw, int cols, cudaStream_t st) {
  constexpr int LR = N, LC = 2 * N;
  typedef ColsCfg2<LC> CC;
  static_assert((N / 2) % CC::G == 0, "tile must divide the column pairs");
  constexpr int TR = (RPC / 2) * (LR / Plan<LR>::E), TI = (RPI / 2) * (LR / Plan<LR>::E);
  constexpr int TC = CC::G * (LC / Plan<LC>::E);
  constexpr size_t smr = rows_smem2<LR, RPC>(), smi = rows_smem2<LR, RPI>(), smc = cols_smem2<LC, CC::G>();
  constexpr int RED = MODE == AP_CG ? RED_ALPHA : (MODE == AP_PC ? RED_RHO : RED_NONE);
  auto k5 = k2_rows_r2c<LR, RPC, MODE == AP_CG>;
  auto k7 = k2_rows_c2r<LR, RPI, RED>;
  auto kc = k2_cols_conv<LC, CC::G, CC::MINB>;
  static int per_sm_max[MAX_DEVICES] = {};
  const int d = device_slot();
  if (per_sm_max[d] == 0) {
    int rc = set_smem(k5, smr);
    if (rc == BSCT_OK) rc = set_smem(k7, smi);
    if (rc == BSCT_OK) rc = set_smem(kc, smc);
    if (rc != BSCT_OK) return rc;
    int per_sm = 0;
    BSCT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kc, TC, smc));
    per_sm_max[d] = per_sm < 1 ? 1 : per_sm;
  }
  // the row passes load and store the rows as 8-byte complex pairs
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(p)) & 7) {
    bsct_set_last_message("FP32 Gram apply: x, y (and the CG direction) must be 8-byte aligned");
    return BSCT_ERR_INVALID_ARG;
  }
  const int per_sm = cols == 1 ? 1 : per_sm_max[d];
  const int tiles = (N / 2) / CC::G;
  const int grid_c = per_sm * sm_count() < tiles ? per_sm * sm_count() : tiles;
  const TwPtrs<float> t = tw_ptrs<float, N>(tw);
  c2* S2 = reinterpret_cast<c2*>(S);
  const float* k7_in = MODE == AP_CG ? (const float*)p : (MODE == AP_PC ? in : (const float*)nullptr);
  if (MODE == AP_PLAIN) timer_mark(st, 0);
  if constexpr (MODE == AP_CG)
    BSCT_CUDA_TRY(launch_overlap(k5, dim3(N / RPC), dim3(TR), smr, st, in, S2, t.rows_f, t.untangle, (const float*)p,
                                 p, (const double*)(sc + SC_BETA), (unsigned int*)nullptr));
  else
    BSCT_CUDA_TRY(launch_overlap(k5, dim3(N / RPC), dim3(TR), smr, st, in, S2, t.rows_f, t.untangle,
                                 (const float*)nullptr, (float*)nullptr, (const double*)nullptr,
                                 MODE == AP_PLAIN ? input_status_ptr() : (unsigned int*)nullptr));
  if (MODE == AP_PLAIN) timer_mark(st, 1);
  BSCT_CUDA_TRY(launch_overlap(kc, dim3(grid_c), dim3(TC), smc, st, S2, Gt, t.cols_f, t.cols_r, tiles));
  if (MODE == AP_PLAIN) timer_mark(st, 2);
  BSCT_CUDA_TRY(launch_overlap(k7, dim3(N / RPI), dim3(TI), smi, st, (const c2*)S2, out, t.rows_r, t.untangle, k7_in,
                               MODE == AP_PLAIN ? (double*)nullptr : part, MODE == AP_PLAIN ? (double*)nullptr : sc));
  if (MODE == AP_PLAIN) timer_mark(st, 3);
  count_launch(3);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

template <typename T, int N, int MODE, int RPC, int RPI>
static int run_if_ok(const T* in, T* p, T* out, double* sc, double* part, cpx<T>* S, const T* Gt, const cpx<T>* tw,
                     int cols, cudaStream_t st) {
  if constexpr (rows_valid<T, N, RPC>() && rows_valid<T, N, RPI>()) {
    if constexpr (sizeof(T) == 4)
      return run_apply2<N, MODE, RPC, RPI>(in, p, out, sc, part, S, Gt, tw, cols, st);
    else
      return run_apply<T, N, MODE, RPC, RPI>(in, p, out, sc, part, S, Gt, tw, cols, st);
  } else {
    bsct_set_last_message("FFT launch shape not valid for this size");
    return BSCT_ERR_INVALID_ARG;
  }
}

template <typename T, int N, int MODE>
static int dispatch(const T* in, T* p, T* out, double* sc, double* part, cpx<T>* S, const T* Gt, const cpx<T>* tw,
                    cudaStream_t st) {
  constexpr int DF = def_rows_fwd<T, N>(), DI = def_rows_inv<T, N>();
  const Shape sh = cur_shape<T>();
#define BSCT_SHAPE(F_, I_)                                                                                      \
  case F_ * 3 + I_:                                                                                             \
    return run_if_ok<T, N, MODE, shape_cand<DF>(F_), shape_cand<DI>(I_)>(in, p, out, sc, part, S, Gt, tw, sh.cols, \
                                                                        st);
  switch (sh.fwd * 3 + sh.inv) {
    BSCT_SHAPE(0, 0) BSCT_SHAPE(0, 1) BSCT_SHAPE(0, 2)
    BSCT_SHAPE(1, 0) BSCT_SHAPE(1, 1) BSCT_SHAPE(1, 2)
    BSCT_SHAPE(2, 0) BSCT_SHAPE(2, 1) BSCT_SHAPE(2, 2)
  }
#undef BSCT_SHAPE
  bsct_set_last_message("FFT launch shape index out of range");
  return BSCT_ERR_INVALID_ARG;
}

template <typename T, int N>
static int apply_impl(const T* x, T* y, cpx<T>* S, const T* Gt, const cpx<T>* tw, cudaStream_t st) {
  return dispatch<T, N, AP_PLAIN>(x, (T*)nullptr, y, (double*)nullptr, (double*)nullptr, S, Gt, tw, st);
}

// q = G p for CG with the direction update fused into the first pass (p = r + beta p) and
// <p, q> into the last, whose last CTA forms alpha
template <typename T, int N>
static int apply_cg_impl(const T* r, T* p, T* q, double* sc, double* part, cpx<T>* S, const T* Gt,
                         const cpx<T>* tw, cudaStream_t st) {
  return dispatch<T, N, AP_CG>(r, p, q, sc, part, S, Gt, tw, st);
}

// z = M^-1 r for preconditioned CG: the plain apply with the preconditioner's spectrum,
// <r, z> fused into the last pass, whose last CTA forms beta and rho
template <typename T, int N>
static int apply_pc_impl(const T* r, T* z, double* sc, double* part, cpx<T>* S, const T* Mt, const cpx<T>* tw,
                         cudaStream_t st) {
  return dispatch<T, N, AP_PC>(r, (T*)nullptr, z, sc, part, S, Mt, tw, st);
}

// shapes: the three row-count candidates of each row pass (0 where not valid) ...
template <typename T, int N> static void shape_cands(int fwd[3], int inv[3]) {
  constexpr int DF = def_rows_fwd<T, N>(), DI = def_rows_inv<T, N>();
  fwd[0] = rows_valid<T, N, shape_cand<DF>(0)>() ? shape_cand<DF>(0) : 0;
  fwd[1] = rows_valid<T, N, shape_cand<DF>(1)>() ? shape_cand<DF>(1) : 0;
  fwd[2] = rows_valid<T, N, shape_cand<DF>(2)>() ? shape_cand<DF>(2) : 0;
  inv[0] = rows_valid<T, N, shape_cand<DI>(0)>() ? shape_cand<DI>(0) : 0;
  inv[1] = rows_valid<T, N, shape_cand<DI>(1)>() ? shape_cand<DI>(1) : 0;
  inv[2] = rows_valid<T, N, shape_cand<DI>(2)>() ? shape_cand<DI>(2) : 0;
}
// ... and the current choice as candidate indices (get, or set after validation)
template <typename T, int N> static int shape_index(int idx[3], int set) {
  Shape& sh = cur_shape<T>();
  if (!set) {
    idx[0] = sh.fwd;
    idx[1] = sh.inv;
    idx[2] = sh.cols;
    return BSCT_OK;
  }
  int fwd[3], inv[3];
  shape_cands<T, N>(fwd, inv);
  if (idx[0] < 0 || idx[0] > 2 || idx[1] < 0 || idx[1] > 2 || idx[2] < 0 || idx[2] > 1 || !fwd[idx[0]] ||
      !inv[idx[1]]) {
    bsct_set_last_message("FFT launch shape not valid for this size");
    return BSCT_ERR_INVALID_ARG;
  }
  sh.fwd = idx[0];
  sh.inv = idx[1];
  sh.cols = idx[2];
  return BSCT_OK;
}

template <typename T, int N>
static int spectrum_impl(const T* emb, cpx<T>* S2, T* Gt, const cpx<T>* tw, cudaStream_t st) {
  constexpr int LR = N, LC = 2 * N;
  constexpr int RPC = rows_per_cta<LR>();
  constexpr int CPC = cols_per_cta<T, LC>();
  constexpr int TR = RPC * (LR / Plan<LR>::E), TC = CPC * (LC / Plan<LC>::E);
  const size_t smr = (size_t)RPC * row_region<T, LR, RPC>() * sizeof(cpx<T>);
  const size_t smc = (size_t)CPC * smem_elems<LC>() * sizeof(cpx<T>);
  static bool attr_dones[MAX_DEVICES] = {};
  bool& attr_done = attr_dones[device_slot()];
  if (!attr_done) {
    int rc = set_smem(k_rows_r2c<T, LR, false, RPC>, smr);
    if (rc == BSCT_OK) rc = set_smem(k_cols_fwd_real<T, LC, CPC>, smc);
    if (rc != BSCT_OK) return rc;
    attr_done = true;
  }
  const TwPtrs<T> t = tw_ptrs<T, N>(tw);
  k_rows_r2c<T, LR, false, RPC><<<LC / RPC, TR, smr, st>>>(emb, LC, S2, t.rows_f, t.untangle);
  k_cols_fwd_real<T, LC, CPC><<<N / CPC, TC, smc, st>>>(S2, Gt, t.cols_f, T(1.0 / ((double)LC * (double)LC)));
  count_launch(2);
  BSCT_CUDA_TRY(cudaGetLastError());
  return BSCT_OK;
}

template <typename T, int N> FftOps<T> fft_ops() {
  FftOps<T> o;
  o.apply = &apply_impl<T, N>;
  o.apply_cg = &apply_cg_impl<T, N>;
  o.apply_pc = &apply_pc_impl<T, N>;
  o.cg_partials = N / 2;  // the fewest rows per CTA any shape of the inverse pass takes
  o.shape_cands = &shape_cands<T, N>;
  o.shape_index = &shape_index<T, N>;
  o.spectrum = &spectrum_impl<T, N>;
  return o;
}

template FftOps<float> fft_ops<float, BSCT_FFT_N>();
template FftOps<double> fft_ops<double, BSCT_FFT_N>();

}  // namespace bsct
