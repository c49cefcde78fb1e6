"""CPU checks of the engine's device helpers, emulated on the host.

The FFT pass code, the Cartesian Zernike table and the pupil function of
the CUDA engine are host-callable; a small C++ program runs them on the CPU
and the values are compared with numpy's FFT and the FP64 oracle.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_13782_gb300", "csrc")


@pytest.fixture(scope="module")
def emulated(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("emu") / "emulate")
    cuda_inc = os.environ.get("CUDA_HOME", "/usr/local/cuda") + "/include"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "native", "emulate.cpp"), "-o", exe, "-lm"],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = {}
    for line in out.splitlines():
        tag, *vals = line.split()
        rows.setdefault(tag, []).append(vals)
    return rows


def test_fft_passes_match_numpy(emulated):
    for vals in emulated["fft"]:
        M, d = int(vals[0]), int(vals[1])
        got = np.array(vals[2:], float).view(complex)
        t = np.arange(M)
        x = np.sin(0.37 * t + 0.1 * M).astype(np.float32) + 1j * (np.cos(0.91 * t).astype(np.float32) - 0.25)
        ref = np.fft.fft(x) if d < 0 else np.fft.ifft(x) * M
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 2e-6, (M, d, err)


def test_pruned_256_point_transforms_match_numpy(emulated):
    """The dataflow kernel's 256-point transforms with the pruned radix-16 passes: the
    box map of the first-pass points, an inverse transform of box-supported inputs
    (pruned first pass) and a forward transform kept on the box (pruned last pass)."""
    assert "boxmap_bad" not in emulated
    assert {int(v[0]): int(v[1]) for v in emulated["boxmap"]} == {53: 107, 63: 127, 72: 145}
    h = 53
    t = np.arange(256)
    ky = np.where(t <= 128, t, t - 256)
    box = np.abs(ky) <= h
    x = np.where(box, np.sin(0.41 * t + 0.3).astype(np.float32)
                 + 1j * (np.cos(0.77 * t).astype(np.float32) - np.float32(0.2)), 0)
    got = np.array(emulated["box256inv"][0], float).view(complex)
    ref = np.fft.ifft(x) * 256
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-6
    x = np.cos(0.23 * t + 1.1).astype(np.float32) + 1j * (np.sin(0.59 * t).astype(np.float32) + np.float32(0.1))
    got = np.array(emulated["box256fwd"][0], float).view(complex)
    ref = np.fft.fft(x)
    err = np.linalg.norm((got - ref)[box]) / np.linalg.norm(ref[box])
    assert err < 2e-6
    assert np.all(got[64:192] == 0)   # the pruned outputs (second-pass rows 4..11) are left at zero


def test_zernike_table_matches_oracle(emulated):
    for vals in emulated["zern"]:
        v = np.array(vals, float)
        x, y = v[0], v[1]
        tab = v[2:].reshape(14, 3)
        for j in range(2, 16):
            gx, gy = orc.zernike_grad(j, x, y)
            np.testing.assert_allclose(tab[j - 2], [orc.zernike(j, x, y), gx, gy], rtol=2e-6, atol=2e-6,
                                       err_msg=f"Z{j}")


def test_pupil_matches_oracle(emulated):
    zc = 0.3 * np.sin(2.1 * np.arange(14) + 0.3)
    R, lam, dk, z = 10.0, 0.532, 1.0 / (32 * 0.6), 2.5
    for vals in emulated["pupil"]:
        edge = int(vals[0])
        qy, qx, re, im = (float(v) for v in vals[1:])
        # evaluate the oracle's pupil on a 1x1 grid: p = 0, delta = -q
        g = orc.Geometry(2, 2, np.zeros((1, 2)), R, "hard" if edge else "aa", lam, dk)
        g.m = 1
        P = orc.pupil(g, zc, z, [-qy, -qx])
        ref = P["M"][0, 0]
        assert abs(complex(re, im) - ref) < 2e-5, (edge, qy, qx, complex(re, im), ref)


def test_monomial_basis_matches_oracle(emulated):
    c = 0.3 * np.cos(1.7 * np.arange(14) + 0.4)
    for vals in emulated["theta"]:
        v = np.array(vals, float)
        x, y, th, gx, gy = v[:5]
        zs = v[5:]
        ref_th = sum(cj * orc.zernike(j, x, y) for j, cj in zip(range(2, 16), c))
        ref_g = [sum(cj * orc.zernike_grad(j, x, y)[a] for j, cj in zip(range(2, 16), c)) for a in (0, 1)]
        np.testing.assert_allclose([th, gx, gy], [ref_th, *ref_g], rtol=3e-6, atol=3e-6)
        np.testing.assert_allclose(zs, [orc.zernike(j, x, y) for j in range(2, 16)], rtol=3e-6, atol=3e-6)


def test_column_form_matches_oracle(emulated):
    """theta, d theta/dx and d theta/dy from the per-column polynomials in y (the form the
    per-LED kernel evaluates) against the Zernike sums of the oracle."""
    c = 0.3 * np.cos(1.7 * np.arange(14) + 0.4)
    rows = emulated["colform"]
    assert len(rows) == 30
    for vals in rows:
        x, y, th, gx, gy = (float(v) for v in vals)
        ref_th = sum(cj * orc.zernike(j, x, y) for j, cj in zip(range(2, 16), c))
        ref_g = [sum(cj * orc.zernike_grad(j, x, y)[a] for j, cj in zip(range(2, 16), c)) for a in (0, 1)]
        np.testing.assert_allclose([th, gx, gy], [ref_th, *ref_g], rtol=3e-6, atol=3e-6)


def test_optimiser_coefficients_match_oracle(emulated):
    """The host's per-step coefficients (handed to the update kernel) against the oracle's
    definitions: Adam's bias corrections and NAdam's momentum schedule and running product."""
    b1, b2, psi = 0.9, 0.999, 0.004
    prod = 1.0
    rows = {(int(v[0]), int(v[1])): [float(x) for x in v[2:]] for v in emulated["coef"]}
    assert len(rows) == 48
    for t in range(1, 13):
        bc2 = 1.0 / np.sqrt(1 - b2 ** t)
        for opt in (0, 1):   # Adam, AdamW
            np.testing.assert_allclose(rows[(opt, t)][:4], [1 / (1 - b1 ** t), bc2, 0, 0], rtol=1e-7)
        mu, mu_next = orc.nadam_mu(t, b1, psi), orc.nadam_mu(t + 1, b1, psi)
        prod *= mu
        got = rows[(2, t)]
        np.testing.assert_allclose(got[:4], [mu_next / (1 - prod * mu_next), bc2, (1 - mu) / (1 - prod), 0],
                                   rtol=1e-7)
        assert got[4] == pytest.approx(prod, rel=1e-15)
        assert rows[(3, t)][:4] == [0.0, 1.0, 0.0, 0.0]
    assert float(emulated["nadam_advance"][0][0]) == pytest.approx(prod, rel=1e-15)


def test_parallel_polynomial_entries_equal_serial(emulated):
    assert float(emulated["polyentry"][0][0]) <= 1e-6
