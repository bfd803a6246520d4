"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Holds none of the reconstruction method's arithmetic: only phantom parameters,
analytic ellipse line integrals (the measured data), Poisson counting noise and the
named workload configurations.  Neither the oracle nor the CUDA path is imported.
"""
from .configs import CONFIGS, get_config  # noqa: F401
from .phantom import (  # noqa: F401
    ellipse_params,
    ellipse_sinogram,
    ellipse_image,
    poisson_log_sinogram,
    make_problem,
)
