"""GB300-native Batch-FPM engine (arXiv 2408.13782): random mini-batch,
multi-parameter Fourier ptychographic reconstruction with hand-written sm_103a
kernels behind a C ABI (include/fpm.h)."""

from .engine import Engine, FpmError, epoch_permutation, lib, LIB_PATH, EXPORTS  # noqa: F401


def autograd_intensities(*args, **kw):
    """See paper_2408_13782_gb300.autograd.fpm_intensities (imports torch lazily)."""
    from .autograd import fpm_intensities
    return fpm_intensities(*args, **kw)
