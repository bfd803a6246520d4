"""The accuracy study end to end on the GPU (analytic blurred ellipse sinograms, back
projection, steepest descent), small sizes.  Checks the expected behaviour of the
unregularised reconstruction: a clean sinogram at lambda_y = 1 is reconstructed well,
added noise lowers the SNR, and the metrics stay in range."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_13471_gb300 as m

    m.lib()
    return m


def test_accuracy_sweep_small(bsct):
    from paper_2005_13471_gb300 import study

    rows = study.accuracy_sweep(bsct, N=64, n_views=90, zeta=1.0, lambdas=(0.5, 1.0, 2.0), noise=(0.0, 0.05),
                                solver="sd", iters=150, n_ellipses=8)
    by = {(r["lambda_y"], r["noise"]): r for r in rows}
    assert len(rows) == 6
    assert by[(1.0, 0.0)]["snr_db"] > 15.0 and by[(1.0, 0.0)]["ssim"] > 0.8
    for lam in (0.5, 1.0, 2.0):
        assert by[(lam, 0.05)]["snr_db"] < by[(lam, 0.0)]["snr_db"]
    for r in rows:
        assert -1.0 <= r["ssim"] <= 1.0 and np.isfinite(r["snr_db"]) and r["iterations"] == 150
