"""Seeded synthetic inputs for Batch-FPM workloads.

This package generates inputs only: ground-truth objects, LED geometry, pupil
aberration coefficients, per-LED intensity factors, the random batch order and
the measurement noise. It holds none of the reconstruction arithmetic (no
forward model, no gradient, no optimiser); both the FP64 oracle and the CUDA
engine consume what it produces.
"""

from .recipes import (  # noqa: F401
    Config,
    config,
    smooth_field,
    make_object,
    led_grid,
    zernike_coeffs,
    led_gamma,
    brightfield_mask,
    add_noise,
    splitmix64,
    epoch_permutation,
    chop,
    schedule,
    CONFIG_NAMES,
)
