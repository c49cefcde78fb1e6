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
    declared = set(re.findall(r"\b(fpm_[a-z0-9_]+)\s*\(", hdr))
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


def test_ctypes_structures_match_the_header(tmp_path):
    """Size and field offsets of every structure the Python binding mirrors, as the C
    compiler lays them out from include/fpm.h."""
    import ctypes
    import shutil
    import subprocess

    from paper_2408_13782_gb300.engine import Geometry, Hparams
    from paper_2408_13782_gb300.serve import JobDesc, JobStatus

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    mirrors = {"fpm_geometry": Geometry, "fpm_hparams": Hparams, "fpm_job_desc": JobDesc,
               "fpm_job_status": JobStatus}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fpm.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
