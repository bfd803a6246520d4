"""GB300-native pixel-basis (box-spline) Gram filtering for parallel-beam X-ray CT.

Thin Python binding of ``libbsct.so`` (include/bsct.h): argument marshalling only.
Every step of the method runs in the library's CUDA kernels; torch provides device
memory and the current CUDA stream.  The binding raises if the library is missing
or a tensor is not a contiguous CUDA tensor of the expected dtype and shape -
there is no CPU fallback.

Entry points (same names as the C ABI):
    gram_build(geom, precision)          -> GramFilter   (Sec. 4 Gram filter + spectrum)
    gram_apply(gram, x, out=None)        -> y = G x      (zero-padded FFT convolution)
    backproject(geom, sino, precision)   -> b = H^T g    (Sec. 5)
    cg_solve(gram, b, x0=None, ...)      -> (x, report)  (normal equations of Sec. 2)
"""
import ctypes
import os

import numpy as np

__all__ = [
    "F32", "F64", "Geometry", "GramFilter", "gram_build", "gram_apply", "backproject", "forward_project", "cg_solve",
    "library_path", "lib", "supported_size", "launch_count", "input_status", "check_finite",
]

F32 = 0
F64 = 1
APPLY_FFT32 = 0
APPLY_F64 = 1
APPLY_DFTGEMM_BF16 = 2
OK = 0
WARN_NOT_CONVERGED = 1
# floor of the circulant preconditioner's symbol, relative to G^(0): the fewest PCG
# iterations to a 1e-4 residual on ellipse and white-noise targets (N = 64 .. 256)
PRECOND_EPS = 1e-4

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def library_path():
    return os.path.join(_HERE, "libbsct.so")


class _Geom(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32),
        ("n_angles", ctypes.c_int32),
        ("n_bins", ctypes.c_int32),
        ("n_blur", ctypes.c_int32),
        ("angles_pi", ctypes.POINTER(ctypes.c_double)),
        ("lambda_y", ctypes.c_double),
        ("zeta_blur", ctypes.c_double),
        ("blur_widths", ctypes.POINTER(ctypes.c_double)),
    ]


class _CGReport(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("rel_residual", ctypes.c_double),
        ("true_rel_residual", ctypes.c_double),
    ]


class FftShape(ctypes.Structure):
    _fields_ = [("rows_fwd", ctypes.c_int32), ("rows_inv", ctypes.c_int32), ("cols_one_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def _declare(L):
    vp, i32, dbl, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
    gp = ctypes.POINTER(_Geom)
    L.bsct_supported_size.argtypes = [i32]
    L.bsct_supported_size.restype = ctypes.c_int
    L.bsct_gram_build.argtypes = [gp, ctypes.c_int, ctypes.POINTER(vp), vp]
    L.bsct_gram_free.argtypes = [vp]
    L.bsct_gram_free.restype = None
    L.bsct_gram_taps.argtypes = [vp, vp, vp]
    L.bsct_gram_spectrum.argtypes = [vp, vp, vp]
    L.bsct_gram_apply.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    L.bsct_backproject_workspace.argtypes = [gp, ctypes.c_int, ctypes.POINTER(sz)]
    L.bsct_backproject.argtypes = [gp, vp, vp, ctypes.c_int, vp, sz, vp]
    L.bsct_cg_solve.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, dbl, ctypes.c_int,
                                ctypes.POINTER(_CGReport), vp]
    L.bsct_cg_begin.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    L.bsct_sd_solve.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, dbl, ctypes.c_int,
                                ctypes.POINTER(_CGReport), vp]
    L.bsct_cg_iterate.argtypes = [vp, vp, ctypes.c_int, vp]
    L.bsct_cg_residual.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp]
    L.bsct_precond_apply.argtypes = [vp, dbl, vp, vp, vp]
    L.bsct_solve_graph.argtypes = [vp, ctypes.c_int, dbl, vp, vp, ctypes.c_int, dbl, ctypes.POINTER(_CGReport), vp]
    L.bsct_gram_apply_host.argtypes = [vp, vp, vp, i32, vp]
    L.bsct_fft_shape_candidates.argtypes = [i32, ctypes.c_int, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.bsct_fft_get_shape.argtypes = [i32, ctypes.c_int, ctypes.POINTER(FftShape)]
    L.bsct_fft_set_shape.argtypes = [i32, ctypes.c_int, ctypes.POINTER(FftShape)]
    L.bsct_fft_autotune.argtypes = [i32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(FftShape), ctypes.POINTER(dbl),
                                    ctypes.POINTER(dbl), vp]
    L.bsct_pcg_solve_learned.argtypes = [vp, vp, dbl, vp, vp, ctypes.c_float, ctypes.c_int, dbl, ctypes.c_int,
                                         ctypes.POINTER(_CGReport), ctypes.POINTER(dbl), vp]
    L.bsct_forward_project_workspace.argtypes = [gp, ctypes.c_int, ctypes.POINTER(sz)]
    L.bsct_forward_project.argtypes = [gp, vp, vp, ctypes.c_int, vp, sz, vp]
    L.bsct_pcg_solve.argtypes = [vp, dbl, vp, vp, ctypes.c_int, ctypes.c_int, dbl, ctypes.c_int,
                                 ctypes.POINTER(_CGReport), vp]
    L.bsct_status_string.argtypes = [ctypes.c_int]
    L.bsct_status_string.restype = ctypes.c_char_p
    L.bsct_last_error_string.argtypes = []
    L.bsct_last_error_string.restype = ctypes.c_char_p
    L.bsct_cg_solve_mixed.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_CGReport), vp]
    L.bsct_cg_solve_mixed.restype = ctypes.c_int
    L.bsct_gemm_bf16.argtypes = [ctypes.c_int, ctypes.c_int, i32, i32, i32, ctypes.c_float, vp, ctypes.c_int64,
                                 ctypes.c_int64, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_float, vp,
                                 ctypes.c_int64, ctypes.c_int64, i32, vp]
    L.bsct_gemm_bf16.restype = ctypes.c_int
    L.bsct_unet_create.argtypes = [i32, ctypes.c_uint64, ctypes.POINTER(vp), vp]
    L.bsct_unet_params.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64)]
    L.bsct_unet_sync_weights.argtypes = [vp, vp]
    L.bsct_unet_copy.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp]
    L.bsct_unet_copy.restype = ctypes.c_int
    L.bsct_unet_forward.argtypes = [vp, vp, vp, i32, i32, i32, vp]
    L.bsct_unet_backward.argtypes = [vp, vp, vp]
    L.bsct_unet_adam_step.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, i32, vp]
    L.bsct_unet_free.argtypes = [vp]
    L.bsct_unet_free.restype = None
    L.bsct_mse_loss_grad.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp]
    L.bsct_cg_solve_learned.argtypes = [vp, vp, vp, vp, ctypes.c_float, ctypes.c_int, dbl, ctypes.c_int,
                                        ctypes.POINTER(_CGReport), ctypes.POINTER(dbl), vp]
    L.bsct_fcg_solve_learned.argtypes = [vp, vp, vp, vp, ctypes.c_float, ctypes.c_int, dbl, ctypes.c_int,
                                         ctypes.POINTER(_CGReport), ctypes.POINTER(i32), ctypes.POINTER(i32), vp]
    for name in ("bsct_unet_create", "bsct_unet_params", "bsct_unet_sync_weights", "bsct_unet_forward",
                 "bsct_unet_backward", "bsct_unet_adam_step", "bsct_mse_loss_grad", "bsct_cg_solve_learned",
                 "bsct_fcg_solve_learned"):
        getattr(L, name).restype = ctypes.c_int
    L.bsct_batch_create.argtypes = [i32, gp, ctypes.POINTER(vp), vp]
    L.bsct_batch_create.restype = ctypes.c_int
    L.bsct_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, vp]
    L.bsct_batch_solve.restype = ctypes.c_int
    L.bsct_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(ctypes.c_longlong)]
    L.bsct_batch_info.restype = ctypes.c_int
    L.bsct_batch_free.argtypes = [vp]
    L.bsct_batch_free.restype = None
    L.bsct_set_kernel_timing.argtypes = [ctypes.c_int]
    L.bsct_set_kernel_timing.restype = ctypes.c_int
    L.bsct_kernel_times.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    L.bsct_kernel_times.restype = ctypes.c_int
    L.bsct_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    L.bsct_fma_peak.restype = ctypes.c_int
    L.bsct_set_launch_overlap.argtypes = [ctypes.c_int]
    L.bsct_set_launch_overlap.restype = ctypes.c_int
    L.bsct_launch_count.argtypes = []
    L.bsct_launch_count.restype = ctypes.c_uint64
    L.bsct_conv3x3_forward.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, ctypes.c_int, vp, vp]
    L.bsct_conv3x3_backward.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp, ctypes.c_int, vp, vp, vp, vp]
    L.bsct_tconv2x2_forward.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp, vp]
    L.bsct_tconv2x2_backward.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]
    for name in ("bsct_conv3x3_forward", "bsct_conv3x3_backward", "bsct_tconv2x2_forward",
                 "bsct_tconv2x2_backward"):
        getattr(L, name).restype = ctypes.c_int
    L.bsct_fft_autotune_flushed.argtypes = [i32, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                            ctypes.POINTER(FftShape), ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp]
    L.bsct_fft_autotune_flushed.restype = ctypes.c_int
    L.bsct_gnorm_loss_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
    L.bsct_gnorm_loss_grad.restype = ctypes.c_int
    L.bsct_set_gemm_path.argtypes = [ctypes.c_int]
    L.bsct_set_gemm_path.restype = ctypes.c_int
    L.bsct_input_status.argtypes = [vp]
    L.bsct_input_status.restype = ctypes.c_int
    L.bsct_check_finite.argtypes = [vp, ctypes.c_int64, ctypes.c_int, vp]
    L.bsct_check_finite.restype = ctypes.c_int
    for name in ("bsct_gram_build", "bsct_gram_taps", "bsct_gram_spectrum", "bsct_gram_apply",
                 "bsct_backproject_workspace", "bsct_backproject", "bsct_cg_solve", "bsct_cg_begin",
                 "bsct_cg_iterate", "bsct_cg_residual"):
        getattr(L, name).restype = ctypes.c_int


def lib():
    """Load libbsct.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        _declare(L)
        _LIB = L
    return _LIB


def _check(rc, what):
    if rc < 0:
        L = lib()
        raise RuntimeError(f"{what} failed: {L.bsct_status_string(rc).decode()} "
                           f"({L.bsct_last_error_string().decode()})")
    return rc


def supported_size(N):
    return bool(lib().bsct_supported_size(int(N)))


def launch_count():
    return int(lib().bsct_launch_count())


ERR_NONFINITE = -5


def input_status():
    """Read and clear the library's input status (synchronises the current stream):
    ERR_NONFINITE if a Gram apply, back projection or forward projection whose work has
    completed met a non-finite input value since the last call, else OK."""
    return int(lib().bsct_input_status(_stream()))


def check_finite(t):
    """True if every value of the CUDA tensor t (float32 or float64) is finite (synchronous)."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype not in (torch.float32, torch.float64):
        raise TypeError("check_finite needs a float32 / float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("check_finite needs a contiguous tensor")
    prec = F32 if t.dtype == torch.float32 else F64
    rc = lib().bsct_check_finite(ctypes.c_void_p(t.data_ptr()), int(t.numel()), prec, _stream())
    if rc == ERR_NONFINITE:
        return False
    _check(rc, "bsct_check_finite")
    return True


def set_gemm_path(path):
    """0: tcgen05 tensor-core GEMMs (default); 1: the warp-level mma.sync comparison path."""
    _check(lib().bsct_set_gemm_path(int(path)), "bsct_set_gemm_path")


def _fptr(t, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def conv3x3_layer(x, w, b, relu=True, gout=None):
    """One 3x3 convolution layer of the learned CNN (bsct_conv3x3_forward / _backward).

    x [cin, n, H, W], w [cout, kpad], b [cout] (float32 CUDA).  Returns out, and with gout
    also (gin, gw, gb)."""
    import torch

    cin, n, H, W = x.shape
    cout = w.shape[0]
    out = torch.empty((cout, n, H, W), dtype=torch.float32, device=x.device)
    _check(lib().bsct_conv3x3_forward(n, cin, cout, H, W, _fptr(x, "x"), _fptr(w, "w"), _fptr(b, "b"),
                                      1 if relu else 0, _fptr(out, "out"), _stream()), "bsct_conv3x3_forward")
    if gout is None:
        return out
    gin, gw, gb = torch.empty_like(x), torch.empty_like(w), torch.empty_like(b)
    _check(lib().bsct_conv3x3_backward(n, cin, cout, H, W, _fptr(x, "x"), _fptr(w, "w"), _fptr(out, "out"),
                                       _fptr(gout, "gout"), 1 if relu else 0, _fptr(gin, "gin"), _fptr(gw, "gw"),
                                       _fptr(gb, "gb"), _stream()), "bsct_conv3x3_backward")
    return out, gin, gw, gb


def tconv2x2_layer(x, w, b, gout=None):
    """One 2x2 stride-2 transposed convolution of the learned CNN: x [cin, n, H, W],
    w [cout * 4, cin], b [cout].  Returns out [cout, n, 2H, 2W], and with gout (gin, gw, gb)."""
    import torch

    cin, n, H, W = x.shape
    cout = w.shape[0] // 4
    out = torch.empty((cout, n, 2 * H, 2 * W), dtype=torch.float32, device=x.device)
    _check(lib().bsct_tconv2x2_forward(n, cin, cout, H, W, _fptr(x, "x"), _fptr(w, "w"), _fptr(b, "b"),
                                       _fptr(out, "out"), _stream()), "bsct_tconv2x2_forward")
    if gout is None:
        return out
    gin, gw, gb = torch.empty_like(x), torch.empty_like(w), torch.empty_like(b)
    _check(lib().bsct_tconv2x2_backward(n, cin, cout, H, W, _fptr(x, "x"), _fptr(w, "w"), _fptr(gout, "gout"),
                                        _fptr(gin, "gin"), _fptr(gw, "gw"), _fptr(gb, "gb"), _stream()),
           "bsct_tconv2x2_backward")
    return out, gin, gw, gb


def set_kernel_timing(on):
    """Record CUDA events between the three Gram-apply kernels (see bsct_kernel_times)."""
    _check(lib().bsct_set_kernel_timing(1 if on else 0), "bsct_set_kernel_timing")


def fma_peak(precision):
    """Measured FMA throughput of the device in flop/s (FP32 for F32, FP64 for F64)."""
    v = ctypes.c_double()
    _check(lib().bsct_fma_peak(int(precision), ctypes.byref(v), _stream()), "bsct_fma_peak")
    return v.value


def set_launch_overlap(on):
    """Programmatic dependent launch of the Gram-apply kernels (on by default; see bsct_set_launch_overlap)."""
    _check(lib().bsct_set_launch_overlap(1 if on else 0), "bsct_set_launch_overlap")


def kernel_times():
    """Durations (ms) of the row R2C, column convolution and row C2R kernels of the last timed apply."""
    buf = (ctypes.c_float * 3)()
    n = _check(lib().bsct_kernel_times(buf, 3), "bsct_kernel_times")
    return [float(buf[i]) for i in range(n)]


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype(precision):
    import torch

    return torch.float32 if precision == F32 else torch.float64


def _dev(t, shape, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Geometry:
    """Problem geometry of Sec. 2: N x N unit-pixel grid, views, detector of n_bins samples.

    angles_pi: view angles in half turns (theta / pi), e.g. ``np.arange(n) / n``.
    """

    def __init__(self, N, angles_pi, n_bins, lambda_y=1.0, zeta_blur=0.0):
        """zeta_blur: one detector box width, or a sequence of box widths (the detector kernel is
        then the convolution of those unit-mass boxes, Sec. 2)."""
        self.N = int(N)
        self.angles_pi = np.ascontiguousarray(np.asarray(angles_pi, dtype=np.float64).reshape(-1))
        self.n_angles = int(self.angles_pi.size)
        self.n_bins = int(n_bins)
        self.lambda_y = float(lambda_y)
        if np.ndim(zeta_blur) == 0:
            self.zeta_blur = float(zeta_blur)
            self.blur_widths = np.zeros(0)
        else:
            self.zeta_blur = 0.0
            w = np.asarray(zeta_blur, dtype=np.float64).reshape(-1)
            self.blur_widths = np.ascontiguousarray(w[w != 0.0])  # zero widths are no box
        wp = self.blur_widths.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if self.blur_widths.size else None
        self._c = _Geom(self.N, self.n_angles, self.n_bins, int(self.blur_widths.size),
                        self.angles_pi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        self.lambda_y, self.zeta_blur, wp)

    @classmethod
    def uniform(cls, N, n_angles, n_bins, lambda_y=1.0, zeta_blur=0.0):
        return cls(N, np.arange(n_angles, dtype=np.float64) / n_angles, n_bins, lambda_y, zeta_blur)

    def cptr(self):
        return ctypes.byref(self._c)


class GramFilter:
    """Library-owned Gram filter of one geometry (taps, spectrum, apply/CG scratch)."""

    def __init__(self, geom, precision=F32):
        self.geom = geom
        self.N = geom.N
        self.precision = precision
        self._h = ctypes.c_void_p()
        _check(lib().bsct_gram_build(geom.cptr(), precision, ctypes.byref(self._h), _stream()), "bsct_gram_build")

    def close(self):
        if self._h:
            lib().bsct_gram_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype(self):
        return _dtype(self.precision)

    def taps(self):
        import torch

        out = torch.empty((2 * self.N - 1, 2 * self.N - 1), dtype=torch.float64, device="cuda")
        _check(lib().bsct_gram_taps(self._h, ctypes.c_void_p(out.data_ptr()), _stream()), "bsct_gram_taps")
        return out

    def spectrum(self):
        import torch

        out = torch.empty((2 * self.N, self.N + 1), dtype=torch.float64, device="cuda")
        _check(lib().bsct_gram_spectrum(self._h, ctypes.c_void_p(out.data_ptr()), _stream()), "bsct_gram_spectrum")
        return out

    def apply(self, x, out=None, mode=None):
        """y = G x; mode APPLY_DFTGEMM_BF16 selects the split-BF16 tensor-core DFT-GEMM path."""
        import torch

        n = self.N
        px = _dev(x, (n, n), self.dtype, "x")
        if out is None:
            out = torch.empty((n, n), dtype=self.dtype, device=x.device)
        py = _dev(out, (n, n), self.dtype, "out")
        if mode is None:
            mode = APPLY_FFT32 if self.precision == F32 else APPLY_F64
        _check(lib().bsct_gram_apply(self._h, px, py, int(mode), _stream()), "bsct_gram_apply")
        return out

    def precond_apply(self, x, out=None, eps=PRECOND_EPS):
        """y = M^-1 x, the circulant preconditioner (symbol 1 / max(G^, eps G^(0)))."""
        import torch

        n = self.N
        px = _dev(x, (n, n), self.dtype, "x")
        if out is None:
            out = torch.empty((n, n), dtype=self.dtype, device=x.device)
        _check(lib().bsct_precond_apply(self._h, float(eps), px, _dev(out, (n, n), self.dtype, "out"), _stream()),
               "bsct_precond_apply")
        return out

    def pcg_solve(self, b, x0=None, max_iter=100, rel_tol=0.0, check_every=10, eps=PRECOND_EPS):
        """Preconditioned CG on G x = b with the circulant preconditioner."""
        import torch

        n = self.N
        pb = _dev(b, (n, n), self.dtype, "b")
        x = torch.empty((n, n), dtype=self.dtype, device=b.device) if x0 is None else x0.clone()
        rep = _CGReport()
        rc = _check(lib().bsct_pcg_solve(self._h, float(eps), pb, _dev(x, (n, n), self.dtype, "x"),
                                         1 if x0 is None else 0, int(max_iter), float(rel_tol), int(check_every),
                                         ctypes.byref(rep), _stream()), "bsct_pcg_solve")
        return x, dict(iterations=rep.iterations, converged=bool(rep.converged), rel_residual=rep.rel_residual,
                       true_rel_residual=rep.true_rel_residual, status=rc)

    def apply_host(self, x, out=None):
        """y_k = G x_k for host tensors [n, N, N] (pinned for overlapped copies); asynchronous
        on the current stream - synchronise before reading `out`."""
        import torch

        n = self.N
        if x.is_cuda or x.dtype != self.dtype or x.dim() != 3 or tuple(x.shape[1:]) != (n, n) or not x.is_contiguous():
            raise ValueError("x must be a contiguous host tensor [k, N, N] of the handle's dtype")
        if out is None:
            out = torch.empty(x.shape, dtype=self.dtype, pin_memory=x.is_pinned())
        if out.is_cuda or out.shape != x.shape or out.dtype != self.dtype or not out.is_contiguous():
            raise ValueError("out must be a contiguous host tensor like x")
        _check(lib().bsct_gram_apply_host(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          int(x.shape[0]), _stream()), "bsct_gram_apply_host")
        return out

    def cg_solve_learned(self, net, b, in_scale, max_iter=1000, rel_tol=1e-4, check_every=5):
        """CG from the learned warm start alpha * net(in_scale * b) (plain CG if alpha <= 0)."""
        import torch

        n = self.N
        x = torch.empty((n, n), dtype=self.dtype, device=b.device)
        rep = _CGReport()
        alpha = ctypes.c_double()
        rc = _check(lib().bsct_cg_solve_learned(self._h, net._h, _dev(b, (n, n), self.dtype, "b"),
                                                _dev(x, (n, n), self.dtype, "x"), float(in_scale), int(max_iter),
                                                float(rel_tol), int(check_every), ctypes.byref(rep),
                                                ctypes.byref(alpha), _stream()), "bsct_cg_solve_learned")
        return x, dict(iterations=rep.iterations, converged=bool(rep.converged), rel_residual=rep.rel_residual,
                       true_rel_residual=rep.true_rel_residual, alpha=alpha.value, status=rc)

    def pcg_solve_learned(self, net, b, in_scale, max_iter=1000, rel_tol=1e-4, check_every=2, eps=PRECOND_EPS):
        """Circulant-preconditioned CG from the learned warm start alpha * net(in_scale * b)."""
        import torch

        n = self.N
        x = torch.empty((n, n), dtype=self.dtype, device=b.device)
        rep = _CGReport()
        alpha = ctypes.c_double()
        rc = _check(lib().bsct_pcg_solve_learned(self._h, net._h, float(eps), _dev(b, (n, n), self.dtype, "b"),
                                                 _dev(x, (n, n), self.dtype, "x"), float(in_scale), int(max_iter),
                                                 float(rel_tol), int(check_every), ctypes.byref(rep),
                                                 ctypes.byref(alpha), _stream()), "bsct_pcg_solve_learned")
        return x, dict(iterations=rep.iterations, converged=bool(rep.converged), rel_residual=rep.rel_residual,
                       true_rel_residual=rep.true_rel_residual, alpha=alpha.value, status=rc)

    def fcg_solve_learned(self, net, b, in_scale, max_iter=1000, rel_tol=1e-4, precond_every=1):
        """Flexible CG with the network as preconditioner (identity fallback when <r, z> <= 0)."""
        import torch

        n = self.N
        x = torch.empty((n, n), dtype=self.dtype, device=b.device)
        rep = _CGReport()
        npre, nfb = ctypes.c_int32(), ctypes.c_int32()
        rc = _check(lib().bsct_fcg_solve_learned(self._h, net._h, _dev(b, (n, n), self.dtype, "b"),
                                                 _dev(x, (n, n), self.dtype, "x"), float(in_scale), int(max_iter),
                                                 float(rel_tol), int(precond_every), ctypes.byref(rep),
                                                 ctypes.byref(npre), ctypes.byref(nfb), _stream()),
                    "bsct_fcg_solve_learned")
        return x, dict(iterations=rep.iterations, converged=bool(rep.converged), rel_residual=rep.rel_residual,
                       true_rel_residual=rep.true_rel_residual, n_precond=npre.value, n_fallback=nfb.value, status=rc)

    def cg_solve_mixed(self, b, n_low, n_refine):
        """CG with the split-BF16 DFT-GEMM operator, refined by FP32 residual CG steps."""
        import torch

        n = self.N
        x = torch.empty((n, n), dtype=self.dtype, device=b.device)
        rep = _CGReport()
        _check(lib().bsct_cg_solve_mixed(self._h, _dev(b, (n, n), self.dtype, "b"), _dev(x, (n, n), self.dtype, "x"),
                                         int(n_low), int(n_refine), ctypes.byref(rep), _stream()),
               "bsct_cg_solve_mixed")
        return x, dict(iterations=rep.iterations, rel_residual=rep.rel_residual,
                       true_rel_residual=rep.true_rel_residual)

    def cg_solve(self, b, x0=None, max_iter=100, rel_tol=0.0, check_every=10):
        import torch

        n = self.N
        pb = _dev(b, (n, n), self.dtype, "b")
        x = torch.empty((n, n), dtype=self.dtype, device=b.device) if x0 is None else x0.clone()
        px = _dev(x, (n, n), self.dtype, "x")
        rep = _CGReport()
        rc = _check(lib().bsct_cg_solve(self._h, pb, px, 1 if x0 is None else 0, int(max_iter), float(rel_tol),
                                        int(check_every), ctypes.byref(rep), _stream()), "bsct_cg_solve")
        report = dict(iterations=rep.iterations, converged=bool(rep.converged), rel_residual=rep.rel_residual,
                      true_rel_residual=rep.true_rel_residual, status=rc)
        return x, report

    def solve_graph(self, b, method="pcg", max_iter=1000, rel_tol=1e-4, eps=PRECOND_EPS, out=None):
        """CG (method "cg") or circulant-preconditioned CG ("pcg") from x = 0 as one CUDA graph
        whose iterations stop on the device."""
        import torch

        n = self.N
        x = torch.empty((n, n), dtype=self.dtype, device=b.device) if out is None else out
        rep = _CGReport()
        m = {"cg": 0, "pcg": 1}[method]
        rc = _check(lib().bsct_solve_graph(self._h, m, float(eps), _dev(b, (n, n), self.dtype, "b"),
                                           _dev(x, (n, n), self.dtype, "x"), int(max_iter), float(rel_tol),
                                           ctypes.byref(rep), _stream()), "bsct_solve_graph")
        return x, dict(iterations=rep.iterations, converged=bool(rep.converged), rel_residual=rep.rel_residual,
                       true_rel_residual=rep.true_rel_residual, status=rc)

    def sd_solve(self, b, x0=None, max_iter=100, rel_tol=0.0, check_every=10):
        """Steepest descent on G x = b (the paper's reconstruction solver)."""
        import torch

        n = self.N
        pb = _dev(b, (n, n), self.dtype, "b")
        x = torch.empty((n, n), dtype=self.dtype, device=b.device) if x0 is None else x0.clone()
        rep = _CGReport()
        rc = _check(lib().bsct_sd_solve(self._h, pb, _dev(x, (n, n), self.dtype, "x"), 1 if x0 is None else 0,
                                        int(max_iter), float(rel_tol), int(check_every), ctypes.byref(rep),
                                        _stream()), "bsct_sd_solve")
        return x, dict(iterations=rep.iterations, converged=bool(rep.converged), rel_residual=rep.rel_residual,
                       true_rel_residual=rep.true_rel_residual, status=rc)

    def cg_begin(self, b, x, x0_is_zero=True):
        n = self.N
        _check(lib().bsct_cg_begin(self._h, _dev(b, (n, n), self.dtype, "b"), _dev(x, (n, n), self.dtype, "x"),
                                   1 if x0_is_zero else 0, _stream()), "bsct_cg_begin")

    def cg_iterate(self, x, n_iter):
        n = self.N
        _check(lib().bsct_cg_iterate(self._h, _dev(x, (n, n), self.dtype, "x"), int(n_iter), _stream()),
               "bsct_cg_iterate")

    def cg_residual(self):
        rr, bb = ctypes.c_double(), ctypes.c_double()
        _check(lib().bsct_cg_residual(self._h, ctypes.byref(rr), ctypes.byref(bb), _stream()), "bsct_cg_residual")
        return rr.value, bb.value


def fft_shape_candidates(N, precision=F32):
    """(forward, inverse) row-count candidates of the FFT row passes for size N (0 = not valid)."""
    f, v = (ctypes.c_int32 * 3)(), (ctypes.c_int32 * 3)()
    _check(lib().bsct_fft_shape_candidates(int(N), int(precision), f, v), "bsct_fft_shape_candidates")
    return list(f), list(v)


def fft_shape(N, precision=F32):
    """Current launch shape of the FFT apply for size N: (rows_fwd, rows_inv, cols_one_per_sm)."""
    sh = FftShape()
    _check(lib().bsct_fft_get_shape(int(N), int(precision), ctypes.byref(sh)), "bsct_fft_get_shape")
    return sh.rows_fwd, sh.rows_inv, sh.cols_one_per_sm


def set_fft_shape(N, rows_fwd, rows_inv, cols_one_per_sm=0, precision=F32):
    sh = FftShape(int(rows_fwd), int(rows_inv), int(cols_one_per_sm), 0)
    _check(lib().bsct_fft_set_shape(int(N), int(precision), ctypes.byref(sh)), "bsct_fft_set_shape")


def fft_autotune(N, precision=F32, reps=20, flush_bytes=0):
    """Time every valid launch shape for size N, keep the fastest; returns (shape, us, all_us).
    flush_bytes > 0 evicts L2 before every timed apply (bsct_fft_autotune_flushed)."""
    sh, best, allus = FftShape(), ctypes.c_double(), (ctypes.c_double * 18)()
    if flush_bytes:
        _check(lib().bsct_fft_autotune_flushed(int(N), int(precision), int(reps), int(flush_bytes), ctypes.byref(sh),
                                               ctypes.byref(best), allus, _stream()), "bsct_fft_autotune_flushed")
    else:
        _check(lib().bsct_fft_autotune(int(N), int(precision), int(reps), ctypes.byref(sh), ctypes.byref(best),
                                       allus, _stream()), "bsct_fft_autotune")
    return (sh.rows_fwd, sh.rows_inv, sh.cols_one_per_sm), best.value, list(allus)


def gram_build(geom, precision=F32):
    return GramFilter(geom, precision)


def gram_apply(gram, x, out=None):
    return gram.apply(x, out)


def backproject_workspace(geom, precision=F32):
    n = ctypes.c_size_t()
    _check(lib().bsct_backproject_workspace(geom.cptr(), precision, ctypes.byref(n)), "bsct_backproject_workspace")
    return int(n.value)


def backproject(geom, sino, precision=F32, out=None, work=None):
    """b = H^T g_hat (Sec. 5) for a device sinogram [n_angles, n_bins]."""
    import torch

    dt = _dtype(precision)
    ps = _dev(sino, (geom.n_angles, geom.n_bins), dt, "sino")
    if out is None:
        out = torch.empty((geom.N, geom.N), dtype=dt, device=sino.device)
    pb = _dev(out, (geom.N, geom.N), dt, "out")
    nbytes = backproject_workspace(geom, precision)
    if work is None or work.numel() < nbytes:
        work = torch.empty(nbytes, dtype=torch.uint8, device=sino.device)
    _check(lib().bsct_backproject(geom.cptr(), ps, pb, precision, ctypes.c_void_p(work.data_ptr()),
                                  ctypes.c_size_t(work.numel()), _stream()), "bsct_backproject")
    return out


def forward_project_workspace(geom, precision=F32):
    n = ctypes.c_size_t()
    _check(lib().bsct_forward_project_workspace(geom.cptr(), precision, ctypes.byref(n)),
           "bsct_forward_project_workspace")
    return int(n.value)


def forward_project(geom, coeffs, precision=F32, out=None, work=None):
    """g_s = S H c (Sec. 2, Eq. 3-4): the [n_angles, n_bins] detector samples of a device image [N, N]."""
    import torch

    dt = _dtype(precision)
    pc = _dev(coeffs, (geom.N, geom.N), dt, "coeffs")
    if out is None:
        out = torch.empty((geom.n_angles, geom.n_bins), dtype=dt, device=coeffs.device)
    ps = _dev(out, (geom.n_angles, geom.n_bins), dt, "out")
    nbytes = forward_project_workspace(geom, precision)
    if work is None or work.numel() < nbytes:
        work = torch.empty(nbytes, dtype=torch.uint8, device=coeffs.device)
    _check(lib().bsct_forward_project(geom.cptr(), pc, ps, precision, ctypes.c_void_p(work.data_ptr()),
                                      ctypes.c_size_t(work.numel()), _stream()), "bsct_forward_project")
    return out


def cg_solve(gram, b, x0=None, max_iter=100, rel_tol=0.0, check_every=10):
    return gram.cg_solve(b, x0, max_iter, rel_tol, check_every)


def gemm_bf16(a, b, c=None, trans_a=False, trans_b=False, alpha=1.0, beta=0.0):
    """c = alpha op(a) op(b) + beta c with BF16 a, b and FP32 c (2-D or batched 3-D tensors)."""
    import torch

    batched = a.dim() == 3
    A = a if batched else a.unsqueeze(0)
    B = b if batched else b.unsqueeze(0)
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16 or not A.is_cuda or not B.is_cuda:
        raise TypeError("a and b must be bfloat16 CUDA tensors")
    if not A.is_contiguous() or not B.is_contiguous():
        raise ValueError("a and b must be contiguous")
    M = A.shape[2] if trans_a else A.shape[1]
    K = A.shape[1] if trans_a else A.shape[2]
    N = B.shape[1] if trans_b else B.shape[2]
    if (B.shape[2] if trans_b else B.shape[1]) != K:
        raise ValueError("inner dimensions differ")
    nb = A.shape[0]
    if c is None:
        C = torch.zeros((nb, M, N), dtype=torch.float32, device=A.device)
    else:
        C = c if batched else c.unsqueeze(0)
    _dev(C, (nb, M, N), torch.float32, "c")
    _check(lib().bsct_gemm_bf16(int(trans_a), int(trans_b), M, N, K, float(alpha), ctypes.c_void_p(A.data_ptr()),
                                A.shape[2], A.shape[1] * A.shape[2], ctypes.c_void_p(B.data_ptr()), B.shape[2],
                                B.shape[1] * B.shape[2], float(beta), ctypes.c_void_p(C.data_ptr()), N, M * N, nb,
                                _stream()), "bsct_gemm_bf16")
    return C if batched else C[0]


class UNet:
    """Encoder-decoder CNN of the learned warm start (library kernels; see include/bsct.h)."""

    def __init__(self, base_channels=32, seed=0):
        self._h = ctypes.c_void_p()
        _check(lib().bsct_unet_create(int(base_channels), int(seed), ctypes.byref(self._h), _stream()),
               "bsct_unet_create")
        self.base = int(base_channels)

    def _raw(self):
        w, g, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        _check(lib().bsct_unet_params(self._h, ctypes.byref(w), ctypes.byref(g), ctypes.byref(n)), "bsct_unet_params")
        return w.value, g.value, n.value

    @property
    def n_params(self):
        return self._raw()[2]

    def _copy(self, which, to_net, t):
        _check(lib().bsct_unet_copy(self._h, which, to_net, ctypes.c_void_p(t.data_ptr()), _stream()),
               "bsct_unet_copy")

    def get_params(self):
        """Copy of the flat FP32 parameter vector (device tensor)."""
        import torch

        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        self._copy(0, 0, out)
        return out

    def get_grads(self):
        import torch

        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        self._copy(1, 0, out)
        return out

    def set_params(self, t):
        import torch

        t = t.to(device="cuda", dtype=torch.float32).contiguous()
        if t.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        self._copy(0, 1, t)

    def forward(self, x, out=None):
        """x: [n, H, W] float32 CUDA tensor (H, W multiples of 64); returns [n, H, W]."""
        import torch

        if x.dim() == 2:
            x = x.unsqueeze(0)
        nb, H, W = x.shape
        if out is None:
            out = torch.empty_like(x)
        _check(lib().bsct_unet_forward(self._h, _dev(x, (nb, H, W), torch.float32, "x"),
                                       _dev(out, (nb, H, W), torch.float32, "out"), nb, H, W, _stream()),
               "bsct_unet_forward")
        return out

    def backward(self, gout):
        import torch

        _check(lib().bsct_unet_backward(self._h, _dev(gout, tuple(gout.shape), torch.float32, "gout"), _stream()),
               "bsct_unet_backward")

    def adam_step(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().bsct_unet_adam_step(self._h, float(lr), float(beta1), float(beta2), float(eps), int(step),
                                         _stream()), "bsct_unet_adam_step")

    def close(self):
        if self._h:
            lib().bsct_unet_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mse_loss_grad(pred, target, grad, loss_acc):
    """grad = 2 (pred - target) / n ; loss_acc (1-element float64 CUDA tensor) += mean squared error."""
    import torch

    n = pred.numel()
    _check(lib().bsct_mse_loss_grad(ctypes.c_void_p(pred.data_ptr()), ctypes.c_void_p(target.data_ptr()), n,
                                    ctypes.c_void_p(grad.data_ptr()), _dev(loss_acc, (1,), torch.float64, "loss"),
                                    _stream()), "bsct_mse_loss_grad")


def gnorm_loss_grad(gram, pred, target, grad, loss_acc, weight=None):
    """G-norm loss of a batch [n, N, N]: loss_acc += (1/n) sum_i w_i <e_i, G e_i>, grad_i = (2 w_i / n) G e_i
    (e = pred - target, G the handle's Gram filter; weight: n FP64 device values or None)."""
    import torch

    n, N = pred.shape[0], gram.N
    pw = ctypes.c_void_p(0) if weight is None else _dev(weight, (n,), torch.float64, "weight")
    _check(lib().bsct_gnorm_loss_grad(gram._h, _dev(pred, (n, N, N), torch.float32, "pred"),
                                      _dev(target, (n, N, N), torch.float32, "target"), n, pw,
                                      _dev(grad, (n, N, N), torch.float32, "grad"),
                                      _dev(loss_acc, (1,), torch.float64, "loss"), _stream()), "bsct_gnorm_loss_grad")


class Batch:
    """Many independent FP32 slices (own geometry each) solved by one CUDA-graph launch."""

    def __init__(self, geoms):
        self.geoms = list(geoms)
        arr = (_Geom * len(self.geoms))(*[g._c for g in self.geoms])
        self._arr = arr
        self._h = ctypes.c_void_p()
        _check(lib().bsct_batch_create(len(self.geoms), arr, ctypes.byref(self._h), _stream()), "bsct_batch_create")

    def solve(self, sinos, xs=None, cg_iters=50):
        """Back projection + cg_iters CG iterations for every slice; returns the list of x."""
        import torch

        if xs is None:
            xs = [torch.empty((g.N, g.N), dtype=torch.float32, device=s.device) for g, s in zip(self.geoms, sinos)]
        ps = (ctypes.c_void_p * len(sinos))(*[_dev(s, (g.n_angles, g.n_bins), torch.float32, "sino").value
                                             for g, s in zip(self.geoms, sinos)])
        px = (ctypes.c_void_p * len(xs))(*[_dev(x, (g.N, g.N), torch.float32, "x").value
                                          for g, x in zip(self.geoms, xs)])
        _check(lib().bsct_batch_solve(self._h, ps, px, int(cg_iters), _stream()), "bsct_batch_solve")
        return xs

    def info(self):
        ng, nodes, kern = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().bsct_batch_info(self._h, ctypes.byref(ng), ctypes.byref(nodes), ctypes.byref(kern)),
               "bsct_batch_info")
        return {"geometries": ng.value, "graph_nodes": nodes.value, "kernels_per_launch": kern.value}

    def close(self):
        if self._h:
            lib().bsct_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
