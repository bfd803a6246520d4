"""Named workloads (sizes, angle counts, detector, blur, phantom, noise, iterations)."""

CONFIGS = {
    # small FP64 case the oracle finishes in seconds
    "fp64_n64": dict(N=64, n_angles=90, n_bins=92, lambda_y=1.0, zeta=0.0,
                     n_ellipses=10, seed=0, I0=None, cg_iters=20, precision="f64"),
    # FP32 GPU case with blur and Poisson noise
    "fp32_n512": dict(N=512, n_angles=720, n_bins=726, lambda_y=1.0, zeta=1.0,
                      n_ellipses=40, seed=0, I0=1e5, cg_iters=100, precision="f32"),
    # large case: 4096^2 zero-padded FFT grids
    "fp32_n2048": dict(N=2048, n_angles=1800, n_bins=2900, lambda_y=1.0, zeta=1.0,
                       n_ellipses=40, seed=0, I0=None, cg_iters=100, precision="f32"),
    # learned warm start: training and evaluation geometries
    "learned_train_n256": dict(N=256, n_angles=360, n_bins=364, lambda_y=1.0, zeta=1.0,
                               n_ellipses=40, seed=0, I0=1e5, cg_iters=200, precision="f32"),
    "learned_eval_n512": dict(N=512, n_angles=720, n_bins=726, lambda_y=1.0, zeta=1.0,
                              n_ellipses=40, seed=0, I0=1e5, cg_iters=200, precision="f32"),
}

# batched multi-slice workload: N and angle count per slice drawn from these sets
BATCH_SIZES_N = (128, 256, 384, 512, 768, 1024)
BATCH_ANGLES = (180, 360, 720, 1440)
BATCH_SLICES = 256
BATCH_CG_ITERS = 50


def batch_slices(n_slices=BATCH_SLICES, seed=0):
    """Per-slice (N, n_angles, n_bins, zeta) for the batched workload, seeded."""
    import math

    import numpy as np

    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_slices):
        N = int(rng.choice(BATCH_SIZES_N))
        na = int(rng.choice(BATCH_ANGLES))
        zeta = float(rng.choice([0.0, 1.0]))
        out.append(dict(N=N, n_angles=na, n_bins=int(math.ceil(1.42 * N)), lambda_y=1.0,
                        zeta=zeta, n_ellipses=10, seed=seed, I0=None))
    return out


def get_config(name):
    return dict(CONFIGS[name])
