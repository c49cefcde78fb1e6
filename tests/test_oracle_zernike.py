"""Pins for the oracle's Zernike polynomials: Noll's table, orthonormality and derivatives."""

import math

import numpy as np
import pytest

import oracle as orc


def _noll_table(golden_dir):
    rows = []
    with open(f"{golden_dir}/zernike_noll1976.txt") as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            j, n, m, expr = line.split(None, 3)
            rows.append((int(j), int(n), int(m), expr.strip()))
    return rows


def test_noll_index_and_values(golden_dir):
    rng = np.random.default_rng(0)
    rho = rng.random(200) * 1.1
    t = rng.random(200) * 2 * math.pi
    x, y = rho * np.cos(t), rho * np.sin(t)
    env = dict(np=np, sqrt=np.sqrt, sin=np.sin, cos=np.cos, rho=rho, t=t)
    rows = _noll_table(golden_dir)
    assert [r[0] for r in rows] == list(range(2, 16))
    for j, n, m, expr in rows:
        assert orc.noll_nm(j) == (n, m)
        ref = eval(expr, {"__builtins__": {}}, env)
        np.testing.assert_allclose(orc.zernike(j, x, y), ref, atol=1e-12, err_msg=f"Z{j}")


def test_orthonormal_on_unit_disk():
    # Gauss-Legendre in rho (exact for these polynomial degrees) times a
    # uniform rule in angle.
    xr, wr = np.polynomial.legendre.leggauss(16)
    rho = 0.5 * (xr + 1)
    wr = 0.5 * wr * rho
    nt = 32
    t = 2 * math.pi * np.arange(nt) / nt
    R, T = np.meshgrid(rho, t, indexing="ij")
    W = wr[:, None] * (2 * math.pi / nt) * np.ones_like(T)
    x, y = R * np.cos(T), R * np.sin(T)
    Z = np.stack([orc.zernike(j, x, y) for j in range(1, 16)])
    G = np.einsum("aij,bij,ij->ab", Z, Z, W) / math.pi
    np.testing.assert_allclose(G, np.eye(15), atol=1e-12)


@pytest.mark.parametrize("j", list(range(2, 16)))
def test_gradients_match_differences(j):
    rng = np.random.default_rng(j)
    x, y = rng.uniform(-1, 1, 50), rng.uniform(-1, 1, 50)
    h = 1e-6
    gx, gy = orc.zernike_grad(j, x, y)
    np.testing.assert_allclose(gx, (orc.zernike(j, x + h, y) - orc.zernike(j, x - h, y)) / (2 * h), atol=1e-7)
    np.testing.assert_allclose(gy, (orc.zernike(j, x, y + h) - orc.zernike(j, x, y - h)) / (2 * h), atol=1e-7)
