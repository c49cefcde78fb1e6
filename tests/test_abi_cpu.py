"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every symbol include/fpm.h declares, and its schedule generator equals
the input generator's (bit-exact, Eq. 13-14)."""

import os
import re

import numpy as np
import pytest

import paper_2408_13782_gb300 as fpm
from paper_2408_13782_gb300 import build
from synth import recipes as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    try:
        build.build()
    except RuntimeError as e:  # no CUDA toolkit on this machine
        pytest.skip(str(e))
    return fpm.lib()


def test_header_declarations_are_exported(L):
    hdr = open(os.path.join(ROOT, "include", "fpm.h")).read()
    declared = set(re.findall(r"\b(fpm_[a-z_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    assert declared == set(fpm.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


@pytest.mark.parametrize("n,seed,epoch", [(49, 11, 0), (225, 22, 7), (9, 0, 3), (1, 5, 0), (121, 2**63 + 5, 2)])
def test_permutation_matches_input_generator(L, n, seed, epoch):
    got = fpm.epoch_permutation(n, seed, epoch)
    assert got.tolist() == S.epoch_permutation(n, seed, epoch).tolist()


def test_create_rejects_bad_shapes_without_gpu(L):
    # shape validation happens before any device call
    with pytest.raises(fpm.FpmError) as e:
        fpm.Engine(48, 4, np.zeros((1, 2)), 5.0, 0.532, 0.05)
    assert e.value.code == -2
    with pytest.raises(fpm.FpmError) as e:
        fpm.Engine(64, 4, np.zeros((1, 2)), 40.0, 0.532, 0.05)   # pupil box wider than the window
    assert e.value.code == -2
    with pytest.raises(fpm.FpmError) as e:
        fpm.Engine(64, 4, np.array([[200.0, 0.0]]), 10.0, 0.532, 0.05)  # crop leaves the spectrum
    assert e.value.code == -2
