"""Pins of the oracle's free-form pupil (the pupil-recovery reading of Section 2.2):
a complex field P on the integer nodes of the crop grid multiplying the
parametric pupil, evaluated at q = p - delta by bilinear interpolation.

* The interpolation against scipy's regular-grid linear interpolator, and its
  derivatives against finite differences.
* P = 1 reproduces the parametric model; a constant P = c scales every
  intensity by |c|^2.
* The gradients with respect to Re and Im of the nodes and the offsets (which
  gain a term from P~ moving with q) against central finite differences.
* Reconstruction.step with the field learned against torch autograd and
  torch.optim.Adam (the interpolation written with torch ops).
"""

import math

import numpy as np
import pytest

import oracle as orc
from tests.helpers import generic_params, tiny_geometry
from tests.test_oracle_physics_pins import _zernike_torch


def _ff(m, seed, amp=0.2):
    rng = np.random.default_rng(seed)
    return (1 + amp * rng.normal(size=(m, m))) * np.exp(1j * amp * rng.normal(size=(m, m)))


def test_bilinear_matches_scipy_and_finite_differences():
    from scipy.interpolate import RegularGridInterpolator
    m = 16
    P = _ff(m, 1, amp=0.5)
    n = np.arange(m) - m // 2
    rng = np.random.default_rng(2)
    qy, qx = rng.uniform(-6, 6, 200), rng.uniform(-6, 6, 200)
    val, dy, dx, _ = orc.bilinear_nodes(P, qy, qx)
    for part in (np.real, np.imag):
        ref = RegularGridInterpolator((n, n), part(P), method="linear")(np.stack([qy, qx], -1))
        np.testing.assert_allclose(part(val), ref, atol=1e-13)
    h = 1e-7
    fd_y = (orc.bilinear_nodes(P, qy + h, qx)[0] - orc.bilinear_nodes(P, qy - h, qx)[0]) / (2 * h)
    fd_x = (orc.bilinear_nodes(P, qy, qx + h)[0] - orc.bilinear_nodes(P, qy, qx - h)[0]) / (2 * h)
    np.testing.assert_allclose(dy, fd_y, atol=1e-7)
    np.testing.assert_allclose(dx, fd_x, atol=1e-7)


def _tiny():
    g, _, _ = tiny_geometry(N=32, m=16, grid=3, pitch=3.0, R=5.0, edge="aa", seed=7)
    prm = generic_params(g, seed=4, z=2.0, off=0.3)
    rng = np.random.default_rng(8)
    O = rng.normal(size=(g.N, g.N)) + 1j * rng.normal(size=(g.N, g.N))
    I = orc.forward(O * (1 + 0.2 * rng.normal(size=O.shape)), generic_params(g, seed=9, z=1.0, off=0.2), g,
                    range(g.n_leds))
    return g, prm, O, I


def test_unit_field_is_the_parametric_model_and_constant_scales_intensities():
    g, prm, O, I = _tiny()
    idx = [0, 4, 8]
    ref = orc.forward(O, prm, g, idx)
    p1 = prm.copy()
    p1.pupil_ff = np.ones((g.m, g.m), np.complex128)
    np.testing.assert_allclose(orc.forward(O, p1, g, idx), ref, rtol=1e-13, atol=1e-13)
    L0, g0, _ = orc.loss_and_grad(O, prm, g, idx, I)
    L1, g1, _ = orc.loss_and_grad(O, p1, g, idx, I)
    assert L1 == pytest.approx(L0, rel=1e-13)
    for k in ("object", "zernike", "gamma", "offset"):
        np.testing.assert_allclose(g1[k], g0[k], rtol=1e-11, atol=1e-13)
    c = 0.7 * np.exp(0.4j)
    p1.pupil_ff = np.full((g.m, g.m), c)
    np.testing.assert_allclose(orc.forward(O, p1, g, idx), abs(c) ** 2 * ref, rtol=1e-12, atol=1e-13)


def test_node_and_offset_gradients_match_finite_differences():
    g, prm, O, I = _tiny()
    prm.pupil_ff = _ff(g.m, 3)
    idx = [0, 4, 8]
    L, gr, _ = orc.loss_and_grad(O, prm, g, idx, I)
    h = 1e-6

    def L_at(p):
        return orc.loss_and_grad(O, p, g, idx, I)[0]

    # nodes inside the supports (|n| < R), Re and Im
    for (ny, nx) in ((0, 0), (2, -3), (-4, 1), (3, 3)):
        for part, unit in (("re", 1.0), ("im", 1j)):
            p = prm.copy()
            p.pupil_ff[ny + g.m // 2, nx + g.m // 2] += unit * h
            Lp = L_at(p)
            p.pupil_ff[ny + g.m // 2, nx + g.m // 2] -= 2 * unit * h
            Lm = L_at(p)
            fd = (Lp - Lm) / (2 * h)
            got = gr["pupil"][ny + g.m // 2, nx + g.m // 2]
            got = got.real if part == "re" else got.imag
            assert got == pytest.approx(fd, rel=1e-5, abs=1e-9), (ny, nx, part)
    # offsets: the bilinear factor is piecewise linear in q, so the difference
    # step stays inside one cell (no node crossing within +-h)
    for i in idx:
        for ax in (0, 1):
            p = prm.copy()
            p.offset[i, ax] += h
            Lp = L_at(p)
            p.offset[i, ax] -= 2 * h
            Lm = L_at(p)
            assert gr["offset"][i, ax] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5, abs=1e-9), (i, ax)


def _torch_loss_ff(torch, g, I, O, zern, z, gamma, delta, Pff, idx):
    """The amplitude batch loss with the free-form pupil, written with torch ops."""
    m, N, R = g.m, g.N, float(g.R)
    p = torch.arange(m, dtype=torch.float64) - m // 2
    py, px = torch.meshgrid(p, p, indexing="ij")
    L = 0.0
    for i in idx:
        i = int(i)
        qy, qx = py - delta[i, 0], px - delta[i, 1]
        r = torch.sqrt(qy * qy + qx * qx)
        A = torch.clamp(R + 0.5 - r, 0.0, 1.0)
        theta = torch.tensordot(zern, _zernike_torch(torch, qx / R, qy / R), dims=1)
        k2 = (r * g.dk_per_um) ** 2
        inside = A > 0
        root = torch.sqrt(torch.where(inside, 1.0 / g.lambda_um ** 2 - k2, torch.ones_like(k2)))
        kappa = torch.where(inside, 2 * math.pi * (root - 1.0 / g.lambda_um), torch.zeros_like(k2))
        fy0, fx0 = torch.floor(qy), torch.floor(qx)
        fy, fx = qy - fy0, qx - fx0
        iy = torch.clamp(fy0.long() + m // 2, 0, m - 2)
        ix = torch.clamp(fx0.long() + m // 2, 0, m - 2)
        Pt = ((1 - fy) * ((1 - fx) * Pff[iy, ix] + fx * Pff[iy, ix + 1])
              + fy * ((1 - fx) * Pff[iy + 1, ix] + fx * Pff[iy + 1, ix + 1]))
        M = A * torch.exp(1j * (theta + z[0] * kappa)) * Pt
        r0 = N // 2 + int(g.n_int[i, 0]) - m // 2
        c0 = N // 2 + int(g.n_int[i, 1]) - m // 2
        psi = torch.fft.ifft2(torch.fft.ifftshift(O[r0:r0 + m, c0:c0 + m] * M))
        a = torch.sqrt(torch.clamp(torch.tensor(np.asarray(I[i], np.float64)), min=0.0))
        L = L + torch.sum((torch.sqrt(gamma[i]) * torch.abs(psi) - a) ** 2)
    return L


def test_reconstruction_with_free_form_pupil_matches_torch():
    torch = pytest.importorskip("torch")
    g, prm, O, I = _tiny()
    lr = dict(object=0.05, zernike=0.02, defocus=0.1, gamma=0.03, offset=0.05, pupil=0.02)
    hp = orc.Hparams(lr=lr, learn=("object", "zernike", "defocus", "gamma", "offset", "pupil"), offset_bound=0.35)
    rec = orc.Reconstruction(g, I, hp, O0=O, prm=prm)
    f64 = torch.float64
    t = dict(object=torch.tensor(O, dtype=torch.complex128, requires_grad=True),
             zernike=torch.tensor(prm.zernike, dtype=f64, requires_grad=True),
             defocus=torch.tensor([prm.defocus], dtype=f64, requires_grad=True),
             gamma=torch.tensor(prm.gamma, dtype=f64, requires_grad=True),
             offset=torch.tensor(prm.offset, dtype=f64, requires_grad=True),
             pupil=torch.ones((g.m, g.m), dtype=torch.complex128, requires_grad=True))
    opt = torch.optim.Adam([{"params": [t[k]], "lr": lr[k]} for k in t], betas=(0.9, 0.999), eps=1e-8)
    for b in ([0, 4, 8], [2, 5], [1, 7, 3, 6], [8, 0]):
        L_ref = rec.step(b)
        opt.zero_grad()
        L = _torch_loss_ff(torch, g, I, t["object"], t["zernike"], t["defocus"], t["gamma"], t["offset"],
                           t["pupil"], b)
        L.backward()
        opt.step()
        with torch.no_grad():
            t["offset"].clamp_(-hp.offset_bound, hp.offset_bound)
            t["gamma"].clamp_(min=hp.gamma_floor)
        assert float(L.detach()) == pytest.approx(L_ref, rel=1e-11)
    np.testing.assert_allclose(rec.prm.pupil_ff, t["pupil"].detach().numpy(), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(rec.O, t["object"].detach().numpy(), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(rec.prm.offset, t["offset"].detach().numpy(), rtol=1e-10, atol=1e-12)
    assert np.max(np.abs(rec.prm.pupil_ff - 1)) > 1e-3   # the field did move
