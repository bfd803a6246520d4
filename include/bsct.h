/*
 * libbsct - pixel-basis (box-spline) Gram filtering for parallel-beam X-ray CT on one
 * GB300 GPU (sm_103a).  C ABI: plain pointers and sizes, no C++ or torch types.
 *
 * Method: Shu & Entezari, "Gram Filtering and Sinogram Interpolation for Pixel-basis
 * in Parallel-beam X-ray CT Reconstruction" (arXiv 2005.13471).  The reconstruction
 * solves the normal equations  G c = b  of the least-squares problem of Sec. 2, where
 *   G = H^T H is applied as a (2N-1) x (2N-1) Gram filter (Sec. 4), and
 *   b = H^T g_hat is the back projection of the B-spline-interpolated sinogram (Sec. 5).
 *
 * Conventions used by every entry point:
 *   - coefficient images are N x N, row-major, element [k2][k1]; unit pixels; pixel
 *     centre x_k = (k1 - (N-1)/2, k2 - (N-1)/2);
 *   - view theta projects x onto y = x . (cos theta, sin theta);
 *   - detector sample m (0 <= m < n_bins) sits at y_m = (m - (n_bins-1)/2) * lambda_y;
 *   - angles are given in half turns (theta / pi) so that 0 and 1/2 are exact;
 *   - the detector blur is a unit-mass box of width zeta_blur (0 = no blur);
 *   - Gram filter taps G[d], d = (d1, d2) in [-(N-1), N-1]^2, stored [d2+N-1][d1+N-1].
 *
 * Memory: every device buffer passed in (d_*) is allocated and owned by the caller
 * and must stay valid until the stream reaches the end of the call.  Handles
 * (bsct_gram) own their device memory and free it in bsct_gram_free.  All calls are
 * asynchronous on the given stream (a cudaStream_t passed as void*, NULL = legacy
 * default stream) except where stated.
 *
 * Errors: every int-returning call returns BSCT_OK (0) on success, a negative
 * BSCT_ERR_* code on failure (nothing was launched, or a CUDA call failed), or a
 * positive BSCT_WARN_* code.  bsct_status_string / bsct_last_error_string describe
 * the code and the last failure.  No exception crosses the ABI.
 */
#ifndef BSCT_H
#define BSCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSCT_OK 0
#define BSCT_ERR_INVALID_ARG (-1)
#define BSCT_ERR_UNSUPPORTED_SIZE (-2)
#define BSCT_ERR_CUDA (-3)
#define BSCT_ERR_TIMEOUT (-4)
#define BSCT_ERR_NONFINITE (-5)
#define BSCT_WARN_NOT_CONVERGED 1

#define BSCT_F32 0 /* FP32 data path */
#define BSCT_F64 1 /* FP64 data path */

#define BSCT_APPLY_FFT32 0         /* FP32 zero-padded 2N x 2N FFT convolution */
#define BSCT_APPLY_F64 1           /* FP64 zero-padded FFT convolution */
#define BSCT_APPLY_DFTGEMM_BF16 2  /* DFTs as split-BF16 GEMMs on tensor cores, FP32 accumulate */

/* Problem geometry (Sec. 2: coefficients c_k on an N x N grid, n_angles views, a
 * detector of n_bins samples with step lambda_y, blur width zeta_blur).
 * angles_pi: HOST array of n_angles values theta_j / pi (any real values; theta and
 * theta + pi are distinct views).  Read during the call only.
 * Detector kernel (Sec. 2 allows a convolution of several boxes): with n_blur = 0 it is one
 * unit-mass box of width zeta_blur (0 = none); with n_blur = 1 or 2 it is the convolution of
 * the unit-mass boxes of widths blur_widths[0 .. n_blur) (HOST array, each in [0.2, 4]) and
 * zeta_blur must be 0.  Two boxes are supported by bsct_gram_build, bsct_backproject and
 * bsct_forward_project (FP32 and FP64); the batch takes one box. */
typedef struct bsct_geom {
  int32_t N;
  int32_t n_angles;
  int32_t n_bins;
  int32_t n_blur;
  const double* angles_pi;
  double lambda_y;
  double zeta_blur;
  const double* blur_widths;
} bsct_geom;

typedef struct bsct_gram bsct_gram; /* opaque, library-owned */

typedef struct bsct_cg_report {
  int32_t iterations;        /* CG iterations run */
  int32_t converged;         /* 1 if the recursive residual reached rel_tol */
  double rel_residual;       /* recursive ||r|| / ||b|| at exit */
  double true_rel_residual;  /* ||b - G x|| / ||b|| recomputed at exit (or -1 if not computed) */
} bsct_cg_report;

/* Supported image sizes N (the FFT lengths are N and 2N). */
int bsct_supported_size(int32_t N);

/* Launch shape of the three FFT passes of the Gram apply for one size N and precision:
 * image rows per CTA of the forward row pass and of the inverse row pass, and whether
 * the persistent column pass runs one CTA per SM (1) or as many as fit (0).  Every
 * shape computes bit-identical results; only the speed differs.  The shape is kept per
 * device (the current one), size and precision, and applies to every apply of that
 * size: gram_apply, cg_solve, pcg_solve, the batch and the no-allocation apply. */
typedef struct bsct_fft_shape {
  int32_t rows_fwd;
  int32_t rows_inv;
  int32_t cols_one_per_sm;
  int32_t reserved;
} bsct_fft_shape;
/* The three candidate row counts of each row pass (half, the built-in default, double;
 * 0 where a candidate does not fit a CTA for this size).  Host arrays of 3. */
int bsct_fft_shape_candidates(int32_t N, int precision, int32_t* rows_fwd, int32_t* rows_inv);
int bsct_fft_get_shape(int32_t N, int precision, bsct_fft_shape* out);
/* Errors: INVALID_ARG when a row count is not one of the valid candidates. */
int bsct_fft_set_shape(int32_t N, int precision, const bsct_fft_shape* shape);
/* Autotuner: times `reps` applies of every valid shape (up to 18) on scratch data of
 * size N (allocated and freed inside; synchronous on the stream), keeps the fastest as
 * the current shape and returns it in *best (may be NULL), its time per apply in µs in
 * *best_us (may be NULL) and every candidate's time in all_us[18] (may be NULL; -1 for
 * invalid shapes; index = 6 fwd + 2 inv + cols over candidate indices). */
int bsct_fft_autotune(int32_t N, int precision, int reps, bsct_fft_shape* best, double* best_us,
                      double* all_us, void* stream);
/* The same with a cold L2 for every timed apply: before each of the `reps` applies a write
 * of flush_bytes bytes (allocated and freed inside) evicts the previous apply's data, and
 * only the applies are timed (one by one).  flush_bytes = 0 is bsct_fft_autotune. */
int bsct_fft_autotune_flushed(int32_t N, int precision, int reps, int64_t flush_bytes, bsct_fft_shape* best,
                              double* best_us, double* all_us, void* stream);

/* Build the Gram filter of a geometry (Sec. 4): for every offset d,
 *   G[d] = sum_theta M_[c, c, s, s, zeta, zeta](d . u_theta)
 * (the unit-mass box spline of the Gram entry; zeta terms only when zeta > 0), then
 * its 2N x 2N circulant spectrum for the FFT apply (Sec. 4, Toeplitz-block-Toeplitz
 * remark).  Taps and spectrum are computed in FP64 on the GPU; precision selects the
 * stored spectrum (BSCT_F32 or BSCT_F64) and the data path of gram_apply / cg_solve.
 * The handle keeps the scratch for gram_apply and cg_solve, so calls sharing one
 * handle must be serialised on one stream.
 * Errors: INVALID_ARG (null pointers, n_angles < 1, lambda_y <= 0, zeta_blur < 0 or
 * 0 < zeta_blur < 0.2), UNSUPPORTED_SIZE (N not supported), CUDA. */
int bsct_gram_build(const bsct_geom* geom, int precision, bsct_gram** out, void* stream);

/* Release a handle (synchronises its stream first).  NULL is a no-op. */
void bsct_gram_free(bsct_gram* g);

/* Copy the (2N-1)^2 FP64 taps, layout [d2+N-1][d1+N-1], into d_out (device). */
int bsct_gram_taps(const bsct_gram* g, double* d_out, void* stream);

/* Copy the real spectrum of the circulant embedding, [2N][N+1] FP64, entry [u][v] =
 * sum_d G[d] exp(-2 pi i (d2 u + d1 v) / 2N) (device). */
int bsct_gram_spectrum(const bsct_gram* g, double* d_out, void* stream);

/* y = G x: y[i] = sum_j G[i - j] x[j] on the N x N grid (Sec. 4), computed as a
 * zero-padded 2N x 2N FFT convolution.  mode BSCT_APPLY_FFT32 needs a BSCT_F32
 * handle and float buffers, BSCT_APPLY_F64 a BSCT_F64 handle and double buffers.
 * BSCT_APPLY_DFTGEMM_BF16 (F32 handle, float buffers) computes the same convolution
 * with every length-2N DFT as two split-BF16 GEMMs on the tensor cores (operands split
 * into BF16 high + low parts, FP32 accumulation; relative error ~5e-6 to 1e-5); its
 * ~12 (2N)^2-float scratch is allocated in the handle on the first such call.
 * d_x and d_y: N*N elements, may not alias; for the FP32 FFT apply both must be 8-byte
 * aligned (as every cudaMalloc'd buffer is), else BSCT_ERR_INVALID_ARG.  The solvers
 * below apply G to their caller's x0 / x as well and carry the same requirement. */
int bsct_gram_apply(const bsct_gram* g, const void* d_x, void* d_y, int mode, void* stream);

/* y_k = G x_k for n images held in HOST memory: h_x and h_y hold n consecutive [N][N]
 * images in the handle's precision (pinned memory - cudaHostAlloc / cudaHostRegister -
 * lets the copies overlap; pageable memory works but serialises them).  The copy in, the
 * apply (the handle's FFT mode) and the copy out of consecutive images run on three
 * library streams over two device images per direction, so the transfers of images
 * k + 1 and k - 1 overlap the apply of image k.  n = 0 accepts NULL image pointers.
 * The first call creates the streams,
 * events and the 4 N^2 device images in the handle (freed by bsct_gram_free).  The work
 * starts after what is queued on `stream`, and `stream` waits for the last copy out
 * (asynchronous: synchronise `stream` before reading h_y).  Not to be called
 * concurrently with other work on the same handle.  n = 0 is a no-op. */
int bsct_gram_apply_host(bsct_gram* g, const void* h_x, void* h_y, int32_t n, void* stream);

/* Largest N accepted by bsct_gram_apply_noalloc. */
#define BSCT_NOALLOC_MAX_N 512

/* y = G x in FP32 without allocating any device memory.  The paper has no
 * counterpart: this is a library service for callers that cannot allocate device
 * memory - for example a plug-in inside a host application that owns the whole
 * device memory pool, or code on a latency-critical path where cudaMalloc / cudaFree
 * would synchronise the device or could fail under memory pressure.  Everything the
 * three FFT passes need besides the caller's buffers (the N x N complex scratch, the
 * packed spectrum, the twiddle tables) lives in fixed-size arrays inside the library
 * that every GPU which loads it holds until the process exits (about 4 MiB).
 *   N          : supported size <= BSCT_NOALLOC_MAX_N, else BSCT_ERR_UNSUPPORTED_SIZE
 *                (nothing is launched);
 *   d_spectrum : [2N][N+1] FP64 real spectrum of the Gram filter's circulant
 *                embedding, the layout bsct_gram_spectrum writes (caller-owned,
 *                device, read every call);
 *   d_x, d_y   : [N][N] float on the device, may not alias.
 * The first call on a device looks up the device addresses of those arrays (no
 * allocation).  All calls share the
 * arrays and leave the last call's contents in them; every element a call reads
 * (twiddle tables of its N, packed spectrum, scratch) is written by the same call
 * first, so nothing has to be cleared and calls with different N may follow one
 * another in any order.  Calls that overlap on the GPU (two streams, or two host
 * threads) race on the shared arrays: serialise them.  Calls no cudaMalloc, cudaFree
 * or allocating library routine.
 * Returns BSCT_OK or a negative error. */
int bsct_gram_apply_noalloc(int32_t N, const double* d_spectrum, const float* d_x, float* d_y,
                            void* stream);

/* Bytes of device workspace bsct_backproject needs for this geometry/precision. */
int bsct_backproject_workspace(const bsct_geom* geom, int precision, size_t* bytes);

/* b = H^T g_hat (Sec. 5): per view the sinogram row is prefiltered by the correction
 * filter q of Eq. 5 (degree-2 views only; q[m] = sqrt(2)(2 sqrt(2) - 3)^|m|, |m| <= 40),
 * interpolated with the B-spline of degree d = (#non-zero of |cos|, |sin|, zeta) - 1,
 * and integrated against the blurred pixel footprint, i.e.
 *   b_k = sum_theta sum_m c~[m] lambda_y M_[c, s, zeta, lambda_y x (d+1)](y_m - x_k . u).
 * d_sino: [n_angles][n_bins] in view order of geom->angles_pi; d_b: [N][N] (output,
 * overwritten).  float for BSCT_F32, double for BSCT_F64.  d_work: workspace of at
 * least the size bsct_backproject_workspace reports.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE (N > 16384 or too many detector samples per
 * view), CUDA. */
int bsct_backproject(const bsct_geom* geom, const void* d_sino, void* d_b, int precision,
                     void* d_work, size_t work_bytes, void* stream);

/* Forward projection g_s = S H c (Sec. 2, Eq. 3-4): detector samples of the blurred
 * X-ray transform of the pixel-basis image,
 *   g_s[j][m] = sum_k c_k M_[|cos theta_j|, |sin theta_j|, zeta](y_m - x_k . u_theta_j),
 * the pixel footprint being the box spline of the pixel's projection (directions |cos|,
 * |sin|, Eq. 3) averaged over the detector cell (one more direction zeta, Eq. 4), with
 * the geometry conventions of bsct_geom.  d_coeffs: [N][N] image (row k2, column k1);
 * d_sino: [n_angles][n_bins] (output, overwritten).  float for BSCT_F32, double for
 * BSCT_F64.  d_work: device workspace of at least bsct_forward_project_workspace bytes
 * (per-view tables and a transposed copy of the image).  Asynchronous on the stream.
 * A sample exactly on the edge of an unblurred axis-aligned footprint (a box) counts the
 * pixel as outside.  Errors: INVALID_ARG, UNSUPPORTED_SIZE (N > 16384,
 * n_angles x n_bins >= 2^31, zeta_blur > 4), CUDA. */
int bsct_forward_project_workspace(const bsct_geom* geom, int precision, size_t* bytes);
int bsct_forward_project(const bsct_geom* geom, const void* d_coeffs, void* d_sino, int precision,
                         void* d_work, size_t work_bytes, void* stream);

/* Conjugate gradients on G x = b (normal equations of Sec. 2) with the handle's data
 * precision; inner products and step scalars in FP64 on the device.
 * d_b: right-hand side [N][N]; d_x: in = initial guess (ignored if x0_is_zero),
 * out = solution.  Runs max_iter iterations, or stops early once the recursive
 * relative residual <= rel_tol (checked every check_every iterations; rel_tol <= 0
 * disables the check and the host never waits inside the loop).  Synchronous: returns
 * after the stream has finished, with *report filled (report may be NULL).
 * Returns BSCT_OK, BSCT_WARN_NOT_CONVERGED (rel_tol > 0 not reached), or an error. */
int bsct_cg_solve(bsct_gram* g, const void* d_b, void* d_x, int x0_is_zero, int max_iter,
                  double rel_tol, int check_every, bsct_cg_report* report, void* stream);

/* The whole solve from x = 0 as one CUDA graph: CG (method 0) or preconditioned CG with
 * the circulant preconditioner of bsct_pcg_solve (method 1, floor eps).  The iterations
 * run as the body of a conditional WHILE node; a one-thread kernel after each iteration
 * decides on the device whether another follows (recursive ||r|| / ||b|| > rel_tol, or
 * always when rel_tol <= 0, and fewer than max_iter iterations so far), so the solve
 * needs one graph launch and one host synchronisation.  Same iterates, report and
 * return codes as bsct_cg_solve / bsct_pcg_solve (report->iterations = iterations run).
 * The executable graph is kept in the handle (rebuilt when method, d_x, max_iter or
 * rel_tol change).  Synchronous. */
int bsct_solve_graph(bsct_gram* g, int method, double eps, const void* d_b, void* d_x, int max_iter,
                     double rel_tol, bsct_cg_report* report, void* stream);

/* Steepest descent on G x = b, the unregularised solver of the paper's reconstruction
 * study (Sec. 6): x += alpha r with alpha = <r, r> / <r, G r>.  Arguments, stopping rule,
 * report and return codes as bsct_cg_solve; four kernels per iteration. */
int bsct_sd_solve(bsct_gram* g, const void* d_b, void* d_x, int x0_is_zero, int max_iter,
                  double rel_tol, int check_every, bsct_cg_report* report, void* stream);

/* Run exactly n_iter CG iterations without any host synchronisation (the body every
 * CG step of bsct_cg_solve runs; suitable for timing and CUDA-graph capture).  The
 * state (x, r, p and the scalars) lives in the handle: call bsct_cg_begin first. */
int bsct_cg_begin(bsct_gram* g, const void* d_b, void* d_x, int x0_is_zero, void* stream);
int bsct_cg_iterate(bsct_gram* g, void* d_x, int n_iter, void* stream);
/* Mixed-precision CG: n_low iterations whose operator is the split-BF16 DFT-GEMM apply
 * (BSCT_APPLY_DFTGEMM_BF16), then refinement by a residual CG step - the true residual
 * b - G x is recomputed with the FP32 FFT apply and n_refine FP32 CG iterations continue
 * from x.  F32 handle only; x starts at 0.  Synchronous; report->true_rel_residual is
 * measured with the FP32 apply. */
int bsct_cg_solve_mixed(bsct_gram* g, const void* d_b, void* d_x, int n_low, int n_refine,
                        bsct_cg_report* report, void* stream);

/* Copy the current recursive squared residual ||r||^2 and ||b||^2 to host (synchronous). */
int bsct_cg_residual(const bsct_gram* g, double* rr, double* bb, void* stream);

/* Circulant preconditioner of the Gram filter.  G is Toeplitz-block-Toeplitz (Sec. 4,
 * closing remark): it is the N x N section of the 2N-periodic circulant C whose
 * eigenvalues are the spectrum G^ of the zero-padded filter.  The preconditioner is the
 * same section of C^-1, with C's symbol floored:
 *     M^-1 x = crop_N( F^-1 [ F(pad_2N x) / max(G^, eps G^(0)) ] ),
 * G^(0) = the sum of the taps = the largest |G^| (all taps are >= 0).  The floor keeps
 * M^-1 symmetric positive definite where the truncated filter's symbol dips below zero
 * (sparse angle sets, blur); eps must lie in (0, 1].  Not part of the paper: a
 * non-learned preconditioner beside the learned one.
 * bsct_precond_apply: d_y = M^-1 d_x, [N][N] in the handle's precision (the Gram apply
 * with the reciprocal spectrum).  The first call, and any call with another eps, builds
 * the reciprocal spectrum (one kernel); the first call also allocates it and one N x N
 * vector in the handle.  Asynchronous on the stream; use one stream per handle.
 * bsct_pcg_solve: preconditioned CG on G x = b with that M^-1; arguments, stopping rule
 * (on the recursive ||r|| / ||b||, checked every check_every iterations), report and
 * return codes as bsct_cg_solve.  Each iteration costs two applies (G and M^-1) and one
 * vector update, seven kernels with no host synchronisation.  Synchronous. */
int bsct_precond_apply(bsct_gram* g, double eps, const void* d_x, void* d_y, void* stream);
int bsct_pcg_solve(bsct_gram* g, double eps, const void* d_b, void* d_x, int x0_is_zero, int max_iter,
                   double rel_tol, int check_every, bsct_cg_report* report, void* stream);

/* Batched reconstruction of many independent slices (FP32).  Each slice i has its own
 * geometry geoms[i] (sizes, views, detector, blur may all differ; slices with an
 * identical geometry share one Gram filter and one set of back-projection tables).
 * bsct_batch_create builds the shared filters / tables and every slice's CG state
 * (synchronous; library-owned memory, released by bsct_batch_free).
 * bsct_batch_solve runs, for every slice, the back projection of its sinogram
 * (Sec. 5) and cg_iters CG iterations on G x = b from x = 0 (Sec. 2, Sec. 4): the
 * whole batch is recorded once into a CUDA graph whose per-slice branches run
 * concurrently, and replayed with a single graph launch on the stream; it is
 * re-recorded only when a pointer or cg_iters changes.  Asynchronous.
 *   d_sino: HOST array of n_slices DEVICE pointers to float [n_angles_i][n_bins_i];
 *   d_x:    HOST array of n_slices DEVICE pointers to float [N_i][N_i] (outputs).
 * Buffers must stay valid while the batch may replay them.  Errors as elsewhere. */
typedef struct bsct_batch bsct_batch;
int bsct_batch_create(int32_t n_slices, const bsct_geom* geoms, bsct_batch** out, void* stream);
int bsct_batch_solve(bsct_batch* b, const float* const* d_sino, float* const* d_x, int cg_iters, void* stream);
/* Distinct geometries, nodes of the recorded graph, kernels per replay. */
int bsct_batch_info(const bsct_batch* b, int* n_geometries, long long* graph_nodes,
                    long long* kernels_per_launch);
void bsct_batch_free(bsct_batch* b);

/* C[b] = alpha op(A[b]) op(B[b]) + beta C[b] with BF16 A, B and FP32 C on the tensor
 * cores (building block of the DFT-GEMM apply and the learned warm start; the paper has
 * no counterpart).  op(A) is M x K: A row-major M x K (lda) or, with trans_a, K x M;
 * op(B) is K x N: B row-major K x N (ldb) or, with trans_b, N x K.  C row-major (ldc).
 * Batch b advances A, B, C by stride_a, stride_b, stride_c elements.  K, lda, ldb and
 * the A/B strides must be multiples of 8, A and B 16-byte aligned; trans_a needs
 * M % 8 == 0 and !trans_b needs N % 8 == 0.  All pointers device. */
/* Which tensor-core GEMM bsct_gemm_bf16 (and every GEMM inside the library) runs:
 * 0 (default) the fifth-generation tensor cores - tcgen05.mma with the accumulator in
 * tensor memory and operand tiles copied into shared memory by the tensor-memory
 * accelerator; 1 the warp-level mma.sync kernel (the comparison path).  Process-wide.
 * Errors: INVALID_ARG. */
int bsct_set_gemm_path(int path);
int bsct_gemm_bf16(int trans_a, int trans_b, int32_t M, int32_t N, int32_t K, float alpha, const void* d_A,
                   int64_t lda, int64_t stride_a, const void* d_B, int64_t ldb, int64_t stride_b, float beta,
                   float* d_C, int64_t ldc, int64_t stride_c, int32_t batch, void* stream);

/* Learned warm start (no counterpart in the paper): a 4-level encoder-decoder CNN
 * (U-Net, base_channels / 2x / 4x / 8x channels, two 3x3 conv + ReLU per level, 2x2
 * max-pool, 2x2 transposed convolutions, skip connections, 1x1 head; 1.92M parameters
 * at base 32) whose 3x3 and transposed convolutions run as BF16 tensor-core GEMMs with
 * FP32 accumulation.  Parameters are FP32 masters with a BF16 copy for the GEMMs,
 * trained with Adam by the library's own backward kernels.
 *   create: He-normal initialisation from a counter-based generator seeded by seed;
 *   params: device pointers to the flat FP32 parameters / gradients (library-owned;
 *           after writing parameters call bsct_unet_sync_weights);
 *   forward: d_in, d_out device float [n][H][W], H and W multiples of 64; keeps the
 *           activations for one following backward;
 *   backward: d_gout = dLoss/d_out of the last forward; adds into the gradients;
 *   adam_step: Adam update (bias-corrected with step >= 1), then zeroes the gradients. */
typedef struct bsct_unet bsct_unet;
int bsct_unet_create(int32_t base_channels, uint64_t seed, bsct_unet** out, void* stream);
int bsct_unet_params(bsct_unet* net, float** d_params, float** d_grads, int64_t* n_params);
int bsct_unet_sync_weights(bsct_unet* net, void* stream);
/* Copy the n_params FP32 parameters (which = 0) or gradients (which = 1) between the
 * net and the caller's device buffer d_buf (to_net = 1: into the net; parameters are
 * then re-rounded into the BF16 copy). */
int bsct_unet_copy(bsct_unet* net, int which, int to_net, float* d_buf, void* stream);
int bsct_unet_forward(bsct_unet* net, const float* d_in, float* d_out, int32_t n, int32_t H, int32_t W, void* stream);
int bsct_unet_backward(bsct_unet* net, const float* d_gout, void* stream);
int bsct_unet_adam_step(bsct_unet* net, float lr, float beta1, float beta2, float eps, int32_t step, void* stream);
void bsct_unet_free(bsct_unet* net);
/* Mean-squared-error loss for training: d_grad = 2 (pred - target) / n and
 * *d_loss += mean (pred - target)^2 (device double, not cleared). */
int bsct_mse_loss_grad(const float* d_pred, const float* d_target, int64_t n, float* d_grad, double* d_loss,
                       void* stream);

/* Single layers of that network (no counterpart in the paper), for checking them one by
 * one: the same kernels and BF16 tensor-core GEMMs the network runs, with FP32 data.
 * Activations are [C][n][H][W] FP32; n*H*W and cout must be multiples of 8.
 * bsct_conv3x3_forward: out = act(conv3x3(bf16(in), bf16(w)) + b), zero padding 1, act =
 *   ReLU when relu != 0, else identity; w [cout][kpad] with column ci*9 + ky*3 + kx and
 *   kpad = 9 cin rounded up to a multiple of 8 (padding columns must be zero).
 * bsct_conv3x3_backward: from d_gout = dLoss/d out, with d = bf16(gout masked by out > 0
 *   when relu != 0): gw = d x im2col(bf16(in))^T ([cout][kpad], overwritten), gb = sum of
 *   the unrounded masked gradient (overwritten), gin = col2im(bf16(w)^T d) (overwritten;
 *   NULL skips it).  d_out (the forward output) is read only when relu != 0.
 * bsct_tconv2x2_forward: 2x2 stride-2 transposed convolution [cin][n][H][W] ->
 *   [cout][n][2H][2W], out[co][n][2y+dy][2x+dx] = sum_ci w[co*4+dy*2+dx][ci] bf16(in) + b;
 *   cin a multiple of 8.  bsct_tconv2x2_backward: gw ([cout*4][cin]), gb, gin (NULL skips
 *   it) from gout, rounded to BF16 before both products.
 * Scratch comes from the stream-ordered allocator (cudaMallocAsync / cudaFreeAsync on the
 * stream).  Asynchronous.  Errors: INVALID_ARG, CUDA. */
int bsct_conv3x3_forward(int32_t n, int32_t cin, int32_t cout, int32_t H, int32_t W, const float* d_in,
                         const float* d_w, const float* d_b, int relu, float* d_out, void* stream);
int bsct_conv3x3_backward(int32_t n, int32_t cin, int32_t cout, int32_t H, int32_t W, const float* d_in,
                          const float* d_w, const float* d_out, const float* d_gout, int relu, float* d_gin,
                          float* d_gw, float* d_gb, void* stream);
int bsct_tconv2x2_forward(int32_t n, int32_t cin, int32_t cout, int32_t H, int32_t W, const float* d_in,
                          const float* d_w, const float* d_b, float* d_out, void* stream);
int bsct_tconv2x2_backward(int32_t n, int32_t cin, int32_t cout, int32_t H, int32_t W, const float* d_in,
                           const float* d_w, const float* d_gout, float* d_gin, float* d_gw, float* d_gb,
                           void* stream);

/* G-norm training loss of the learned warm start (no counterpart in the paper): for n
 * images of the handle's size N (d_pred, d_target, d_grad: [n][N][N] FP32, device),
 *   *d_loss += (1/n) sum_i w_i <e_i, G e_i>,   d_grad_i = (2 w_i / n) G e_i,
 * with e_i = pred_i - target_i and G the handle's Gram filter (FP32 FFT apply); the error
 * is measured in the norm CG minimises.  d_weight: n per-image weights (device FP64) or
 * NULL for 1.  d_loss: one device FP64 value, accumulated (not cleared).  F32 handle.
 * Scratch (n N^2 floats) from the stream-ordered allocator.  Asynchronous.  The sum runs in
 * a fixed order (reproducible). */
int bsct_gnorm_loss_grad(const bsct_gram* g, const float* d_pred, const float* d_target, int32_t n,
                         const double* d_weight, float* d_grad, double* d_loss, void* stream);

/* CG with a learned warm start: x_hat = net(in_scale * b); x0 = alpha x_hat with
 * alpha = <x_hat, b> / <x_hat, G x_hat> (the G-norm-optimal scaling); if alpha is not
 * positive and finite, x0 = 0 (plain CG).  Then bsct_cg_solve from x0 with the given
 * tolerance: plain CG removes whatever error the warm start leaves.  *alpha_out (may be
 * NULL) receives alpha.  F32 handle; N a multiple of 64.  Synchronous. */
int bsct_cg_solve_learned(bsct_gram* g, bsct_unet* net, const void* d_b, void* d_x, float in_scale, int max_iter,
                          double rel_tol, int check_every, bsct_cg_report* report, double* alpha_out, void* stream);
/* The same learned warm start followed by preconditioned CG with the circulant
 * preconditioner of bsct_pcg_solve (floor eps); measures whether the warm start still
 * helps once the preconditioner has removed the slow directions.  Synchronous. */
int bsct_pcg_solve_learned(bsct_gram* g, bsct_unet* net, double eps, const void* d_b, void* d_x, float in_scale,
                           int max_iter, double rel_tol, int check_every, bsct_cg_report* report,
                           double* alpha_out, void* stream);

/* Flexible CG with the network as preconditioner (a learned extension; the paper solves
 * with steepest descent, Sec. 6).  Truncated flexible CG, FCG(1), on G x = b from x0 = 0:
 *   alpha = <p, r> / <p, G p>,  x += alpha p,  r -= alpha G p,
 *   z = M(r),  beta = -<z, G p> / <p, G p>,  p = z + beta p,
 * with M(r) = net(in_scale * s r) / s, s = ||b|| / ||r|| (the network maps right-hand
 * sides scaled by in_scale to solutions, so it approximates G^-1 on residuals brought
 * to the scale of b).  The network is applied every precond_every iterations
 * (1 = every iteration) and M = identity in between; whenever <r, M(r)> <= 0 the
 * identity is used instead (fallback).  Stops when ||r|| / ||b|| <= rel_tol (r the
 * recursive residual) or after max_iter iterations; report as for bsct_cg_solve with the
 * true residual ||b - G x|| / ||b|| recomputed at exit.  *n_precond / *n_fallback (may
 * be NULL) receive the network applications and the fallbacks.  F32 handle, N a multiple
 * of 64; d_b, d_x device FP32 N x N.  Uses the handle's CG scratch (not with a CG in
 * flight on it) and allocates 2 N^2 floats for the call.  Synchronous. */
int bsct_fcg_solve_learned(bsct_gram* g, bsct_unet* net, const void* d_b, void* d_x, float in_scale, int max_iter,
                           double rel_tol, int precond_every, bsct_cg_report* report, int32_t* n_precond,
                           int32_t* n_fallback, void* stream);

/* Non-finite input values (NaN, +-Inf).  The synchronous solvers (cg_solve, sd_solve,
 * pcg_solve, solve_graph, cg_solve_mixed and the learned variants) find a non-finite
 * right-hand side or initial guess in <b, b> / <r, r> before their first iteration and
 * a non-finite residual at their synchronisation points, and return BSCT_ERR_NONFINITE.
 * The asynchronous calls cannot return what their kernels find: bsct_gram_apply,
 * bsct_backproject and bsct_forward_project set a per-device input status when their
 * input (x, the sinogram, the coefficients) holds a non-finite value, and still run.
 * bsct_input_status synchronises `stream`, then reads and clears that status: it returns
 * BSCT_ERR_NONFINITE if such an input was seen by work completed since the last call,
 * else BSCT_OK.  (The status is shared by all streams of the device.)
 * bsct_check_finite checks n values of a caller buffer (float for BSCT_F32, double for
 * BSCT_F64) and returns BSCT_ERR_NONFINITE or BSCT_OK (synchronous). */
int bsct_input_status(void* stream);
int bsct_check_finite(const void* d_buf, int64_t n, int precision, void* stream);

/* Human-readable text of a status code, and of the last failure on this thread. */
const char* bsct_status_string(int status);
const char* bsct_last_error_string(void);

/* Kernel timing of bsct_gram_apply (measurement aid, not needed for computing).
 * bsct_set_kernel_timing(1) makes every following gram_apply record CUDA events on its
 * stream before and after each of its three kernels (row R2C, column convolution,
 * row C2R); bsct_kernel_times waits for the events of the last timed apply and writes
 * up to n kernel durations in milliseconds to the host array ms.  Returns the number
 * written, or a negative error (no timed apply recorded yet).  Not thread-safe. */
int bsct_set_kernel_timing(int on);
int bsct_kernel_times(float* ms, int n);

/* Launch overlap of the Gram-apply kernels (a scheduling choice, not part of the method).
 * When on (the default), each of the three kernels of an FFT-mode apply (and of the CG
 * applies) is launched as a programmatic dependent launch: its CTAs may be scheduled
 * while the previous kernel on the stream is finishing, and each kernel waits for its
 * predecessor's completion before its first global-memory access, so results and stream
 * order are the same either way.  bsct_set_launch_overlap(0) launches them plainly.
 * Process-wide; returns BSCT_OK.  Not thread-safe with concurrent applies. */
int bsct_set_launch_overlap(int on);

/* Number of kernel launches issued by this library since load (all threads). */
uint64_t bsct_launch_count(void);

/* FMA throughput of the current device (measurement aid, not part of the method): the
 * best of three timed runs of a kernel in which every thread runs 8 independent FMA
 * chains, in FP32 (precision BSCT_F32) or FP64 (BSCT_F64); *flops_per_s receives
 * 2 x FMAs / s.  Allocates and frees a small device buffer.  Synchronous. */
int bsct_fma_peak(int precision, double* flops_per_s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BSCT_H */
