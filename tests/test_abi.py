"""CPU checks of the C ABI: the library builds, loads, exports every declared entry
point, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bsct.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2005_13471_gb300 import _build

    _build.build()
    import paper_2005_13471_gb300 as m

    return m.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bsct_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bsct_gram_build", "bsct_backproject", "bsct_gram_apply", "bsct_cg_solve"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_supported_sizes(lib):
    import paper_2005_13471_gb300 as m

    for n in (16, 32, 64, 128, 256, 384, 512, 768, 1024, 2048):
        assert m.supported_size(n)
    for n in (0, 100, 4096, 3000):
        assert not m.supported_size(n)


def test_status_strings(lib):
    assert lib.bsct_status_string(0) == b"ok"
    assert lib.bsct_status_string(-2) == b"unsupported size"


def test_argument_validation_without_gpu(lib):
    import paper_2005_13471_gb300 as m

    h = ctypes.c_void_p()
    # rejected on the host, before any CUDA call
    bad = [
        m.Geometry(100, np.arange(4) / 4, 150),                 # unsupported N
        m.Geometry(64, np.arange(4) / 4, 90, lambda_y=0.0),      # lambda_y <= 0
        m.Geometry(64, np.arange(4) / 4, 90, zeta_blur=-1.0),    # negative blur
        m.Geometry(64, np.arange(4) / 4, 90, zeta_blur=0.1),     # short blur direction
        m.Geometry(64, np.array([0.1, np.nan]), 90),             # non-finite angle
    ]
    codes = [lib.bsct_gram_build(g.cptr(), 0, ctypes.byref(h), None) for g in bad]
    assert codes == [-2, -1, -1, -1, -1]
    assert not h
    nbytes = ctypes.c_size_t()
    assert lib.bsct_backproject_workspace(m.Geometry(64, np.arange(10) / 10, 90).cptr(), 0, ctypes.byref(nbytes)) == 0
    assert nbytes.value > 64 * 90 * 4
    assert lib.bsct_backproject_workspace(m.Geometry(64, np.arange(10) / 10, 90).cptr(), 7, ctypes.byref(nbytes)) == -1
    assert lib.bsct_gram_apply(None, None, None, 0, None) == -1


def test_new_entry_points_validate_on_the_host(lib):
    import paper_2005_13471_gb300 as m

    # forward projection: workspace size, blur and precision limits
    nbytes = ctypes.c_size_t()
    g64 = m.Geometry(64, np.arange(10) / 10, 90, 1.0, 1.0)
    assert lib.bsct_forward_project_workspace(g64.cptr(), 0, ctypes.byref(nbytes)) == 0
    assert nbytes.value >= 64 * 64 * 4 + 10 * 560 * 4
    assert lib.bsct_forward_project_workspace(m.Geometry(64, np.arange(3) / 3, 90, 1.0, 4.5).cptr(), 0,
                                              ctypes.byref(nbytes)) == -2
    assert lib.bsct_forward_project_workspace(g64.cptr(), 7, ctypes.byref(nbytes)) == -1
    assert lib.bsct_forward_project(None, None, None, 0, None, 0, None) == -1
    # solvers and applies on a missing handle
    rep = m._CGReport()
    assert lib.bsct_pcg_solve(None, 1e-4, None, None, 1, 10, 0.0, 1, ctypes.byref(rep), None) == -1
    assert lib.bsct_precond_apply(None, 1e-4, None, None, None) == -1
    assert lib.bsct_sd_solve(None, None, None, 1, 10, 0.0, 1, ctypes.byref(rep), None) == -1
    assert lib.bsct_solve_graph(None, 1, 1e-4, None, None, 10, 1e-4, ctypes.byref(rep), None) == -1
    assert lib.bsct_gram_apply_host(None, None, None, 1, None) == -1
    assert lib.bsct_pcg_solve_learned(None, None, 1e-4, None, None, 1.0, 10, 1e-4, 1, ctypes.byref(rep), None,
                                      None) == -1
    # launch shapes: candidates, the built-in default, and rejected shapes
    f, v = m.fft_shape_candidates(256)
    assert f[1] and v[1] and all(x == 0 or x >= 2 for x in f + v)
    assert m.fft_shape(256) == (f[1], v[1], 0)
    sh = m.FftShape(3, v[1], 0, 0)
    assert lib.bsct_fft_set_shape(256, 0, ctypes.byref(sh)) == -1
    assert lib.bsct_fft_get_shape(100, 0, ctypes.byref(sh)) == -2
    assert lib.bsct_fft_autotune(256, 0, 0, None, None, None, None) == -1
    assert lib.bsct_fft_autotune_flushed(256, 0, 5, -1, None, None, None, None) == -1


def test_check_finite_validates_on_the_host(lib):
    # argument errors are returned before any CUDA call
    assert lib.bsct_check_finite(None, 10, 0, None) == -1   # NULL buffer with values to check
    assert lib.bsct_check_finite(None, -1, 0, None) == -1   # negative count
    assert lib.bsct_check_finite(ctypes.c_void_p(16), 4, 7, None) == -1  # unknown precision


def test_detector_box_list_validates_on_the_host(lib):
    import paper_2005_13471_gb300 as m

    nbytes = ctypes.c_size_t()
    ang = np.arange(6) / 6
    one = m.Geometry(64, ang, 90, 1.0, 0.8)
    two = m.Geometry(64, ang, 90, 1.0, (0.8, 1.3))
    assert m.Geometry(64, ang, 90, 1.0, (0.8, 0.0)).blur_widths.tolist() == [0.8]  # zero widths dropped
    # workspaces: two boxes take the wider tables of their own path
    for f in (lib.bsct_backproject_workspace, lib.bsct_forward_project_workspace):
        assert f(one.cptr(), 0, ctypes.byref(nbytes)) == 0
        n1 = nbytes.value
        assert f(two.cptr(), 0, ctypes.byref(nbytes)) == 0
        assert nbytes.value > 0 and nbytes.value != n1
    # rejected before any CUDA call: widths outside [0.2, 4], more than two boxes, a box
    # list together with zeta_blur, n_blur > 0 without widths
    bad = [m.Geometry(64, ang, 90, 1.0, (0.8, 0.1)), m.Geometry(64, ang, 90, 1.0, (0.8, 4.5)),
           m.Geometry(64, ang, 90, 1.0, (0.5, 0.6, 0.7))]
    for g in bad:
        assert lib.bsct_backproject_workspace(g.cptr(), 0, ctypes.byref(nbytes)) == -1
    g = m.Geometry(64, ang, 90, 1.0, (0.8, 1.3))
    g._c.zeta_blur = 0.5
    assert lib.bsct_forward_project_workspace(g.cptr(), 0, ctypes.byref(nbytes)) == -1
    g = m.Geometry(64, ang, 90, 1.0, 0.0)
    g._c.n_blur = 2
    assert lib.bsct_backproject_workspace(g.cptr(), 0, ctypes.byref(nbytes)) == -1
    # two boxes too wide for the sample spacing: more samples per pixel than the tables hold
    wide = m.Geometry(64, ang, 90, 0.2, (4.0, 4.0))
    assert lib.bsct_backproject(wide.cptr(), ctypes.c_void_p(16), ctypes.c_void_p(16), 0, ctypes.c_void_p(16),
                                1 << 40, None) == -2
    # the batch takes one box
    arr = (m._Geom * 1)(two._c)
    h = ctypes.c_void_p()
    assert lib.bsct_batch_create(1, arr, ctypes.byref(h), None) == -2
    assert not h
