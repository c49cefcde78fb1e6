"""FP64 CPU oracle for the Batch-FPM mini-batch step.

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, independent
statement of what the CUDA engine computes. Only the test-suite, the package
smoke check and the CPU-baseline leg of the benchmark may import it; the
engine itself never does, and the two share no code (only the seeded input
generators in `synth` serve both).

Parity status of each function is listed in `oracle/fpm.py`'s header.
"""

from .fpm import (  # noqa: F401
    Geometry,
    Params,
    Hparams,
    Reconstruction,
    noll_nm,
    zernike,
    zernike_grad,
    pupil,
    object_spectrum,
    bilinear_upsample,
    bilinear_nodes,
    init_object,
    crop,
    forward_fields,
    forward,
    loss_and_grad,
    adam_update,
    adamw_update,
    nadam_mu,
    nadam_update,
    rmsprop_update,
)
