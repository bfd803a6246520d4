"""Plain, slow, FP64 CPU oracle for the pixel-basis (box-spline) Gram-filter method.

THIS PACKAGE IS TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py``
may import it.  It shares no code with the CUDA path in
``paper_2005_13471_gb300/`` and never imports it; the only module both sides use
is ``workloads/`` (seeded synthetic inputs, none of the method's arithmetic).

Modules (each function cites the passage of Shu & Entezari, "Gram Filtering and
Sinogram Interpolation for Pixel-basis in Parallel-beam X-ray CT Reconstruction",
that it follows):

* ``geometry``   - angle table, pixel / detector coordinates, interpolation degree
                   (Sec. 2 problem statement, Sec. 5 degree rule).
* ``boxspline``  - univariate box splines (Eq. 1, Eq. 2): truncated-power formula in
                   FP64 and in mpmath, the pixel's projection as a chord length, the
                   detector-blurred footprint (one box, or a convolution of several:
                   the detector model of Sec. 2) and its autocorrelation by exact
                   piecewise Gauss-Legendre quadrature.
* ``gram``       - Gram filter taps (Sec. 4, the Gram entry with and without blur),
                   explicit Gram matrix on tiny grids, Toeplitz spectrum, Gram apply
                   (direct convolution and FFT), the circulant preconditioner
                   (the N x N section of the inverse of G's 2N-periodic circulant
                   embedding, its symbol floored; not in the paper).
* ``backproject``- correction filter (Eq. 5), B-spline sinogram interpolation and the
                   back projection H^T g (Sec. 5), forward sampling g_s = S H c.
* ``cg``         - textbook conjugate gradients on G c = H^T g (normal equations of
                   the least-squares problem of Sec. 2), its preconditioned form, and the
                   steepest descent of the paper's reconstruction study (Sec. 6).

Where the paper is silent or garbled the oracle takes one reading, the one the CUDA
path takes as well; each function's docstring states the readings it depends on.
"""
