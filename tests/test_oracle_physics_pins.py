"""Pins of the oracle against results fixed independently of its own formulas.

* The defocus phase kappa (Section 2.1, Eq. 3: H = exp(i z kappa)) against the
  paraxial (Fresnel) propagator exp(-i pi lambda z |k|^2): their ratio is
  1 + (lambda k)^2 / 4 + O((lambda k)^4), which a wrong 2 pi, a misplaced
  lambda, a wrong spectral bin or a flipped sign all break.
* The forward model under defocus against the Talbot self-imaging law: a weak
  cosine grating of period d imaged in focus, at z_T / 4, z_T / 2 and z_T
  (z_T = 2 d^2 / lambda, the paraxial Talbot length) has its first-harmonic
  contrast multiplied by cos(2 pi z / z_T): 0, -1 and +1, up to the
  non-paraxial correction.
* Reconstruction.step (Section 2.3, Eq. 13: the random-batch update with an
  Adam-family optimiser) against an independent PyTorch reconstruction: the
  forward model written with torch complex ops and torch.fft, the gradients
  from torch.autograd, the update from torch.optim.Adam with one parameter
  group per parameter and its own learning rate, the offsets clamped after
  each step() - compared over several steps with every group learned, FP64.
"""

import math

import numpy as np
import pytest

import oracle as orc
from tests.helpers import generic_params, tiny_geometry


def test_defocus_phase_has_the_fresnel_limit():
    g = orc.Geometry(64, 64, np.zeros((1, 2)), 20.0, "hard", 0.532, 1.0 / (64 * 0.6))
    P = orc.pupil(g, np.zeros(14), 1.0, [0.0, 0.0])
    p = np.arange(g.m) - g.m // 2
    qy, qx = np.meshgrid(p, p, indexing="ij")
    k = np.hypot(qy, qx) * g.dk_per_um          # spatial frequency, 1/um
    lam = g.lambda_um
    inside = (P["A"] > 0) & (k > 0)
    fresnel = -math.pi * lam * k ** 2           # phase per um of defocus, paraxial
    ratio = P["kappa"][inside] / fresnel[inside]
    lk2 = (lam * k[inside]) ** 2
    # kappa / kappa_F = 2 (1 - sqrt(1 - u)) / u with u = (lambda k)^2
    #                 = 1 + u/4 + u^2/8 + ...: the remainder after 1 + u/4 is below u^2/4
    assert np.all(np.abs(ratio - 1 - lk2 / 4) <= lk2 ** 2 / 4 + 1e-12)
    # small |k|: the Fresnel limit itself, to second order in lambda k
    small = lk2 < 4e-3
    assert small.sum() > 40
    assert np.all(np.abs(ratio[small] - 1) <= lk2[small] / 4 + lk2[small] ** 2 / 4)
    assert np.all(np.abs(ratio[small] - 1) <= 1.1e-3)


@pytest.mark.parametrize("period_px", [8, 16])
def test_defocused_grating_follows_the_talbot_law(period_px):
    """Weak cosine grating on the central LED's crop: the image contrast at z is the
    in-focus contrast times cos(2 pi z / z_T), z_T = 2 d^2 / lambda (paraxial)."""
    N = m = 64
    g = orc.Geometry(N, m, np.zeros((1, 2)), 20.0, "hard", 0.532, 1.0 / (m * 0.6))
    dx = 1.0 / (m * g.dk_per_um)                 # low-res pixel, um
    d = period_px * dx                           # grating period, um
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    eps = 1e-3
    o = 1.0 + eps * np.cos(2 * math.pi * xx / period_px)
    O = orc.object_spectrum(o.astype(np.complex128), g.s)
    zt = 2 * d ** 2 / g.lambda_um

    def contrast(z):
        prm = orc.Params(np.zeros(14), z, np.ones(1), np.zeros((1, 2)))
        I = orc.forward(O, prm, g, [0])[0]
        h = np.fft.fft(I.mean(axis=0))[m // period_px]
        return h.real / (m / 2)

    c0 = contrast(0.0)
    assert abs(c0 - 2 * eps) < 1e-6              # in focus: I = 1 + 2 eps cos + O(eps^2)
    u = (g.lambda_um / d) ** 2                   # non-paraxial correction of the phase: 2 pi z/zT * u/4
    for frac, want in ((0.25, 0.0), (0.5, -1.0), (1.0, 1.0)):
        got = contrast(frac * zt) / c0
        slack = 2 * math.pi * frac * u / 4 + 1e-3
        assert abs(got - want) <= slack, (frac, got, want)


# ----------------------------------------------------------------------------
# Reconstruction.step against torch autograd + torch.optim
# ----------------------------------------------------------------------------

def _zernike_torch(torch, x, y):
    """Noll j = 2..15 on the unit disk, written out in Cartesian form."""
    s3, s5, s6, s8, s10 = (math.sqrt(v) for v in (3, 5, 6, 8, 10))
    r2 = x * x + y * y
    return torch.stack([
        2 * x, 2 * y, s3 * (2 * r2 - 1), 2 * s6 * x * y, s6 * (x * x - y * y),
        s8 * (3 * r2 - 2) * y, s8 * (3 * r2 - 2) * x, s8 * (3 * x * x * y - y ** 3), s8 * (x ** 3 - 3 * x * y * y),
        s5 * (6 * r2 * r2 - 6 * r2 + 1), s10 * (4 * r2 - 3) * (x * x - y * y), s10 * (4 * r2 - 3) * 2 * x * y,
        s10 * (x ** 4 - 6 * x * x * y * y + y ** 4), s10 * (4 * x ** 3 * y - 4 * x * y ** 3)])


def _torch_batch_loss(torch, g, I, O, zern, z, gamma, delta, idx):
    """Amplitude loss of the batch (Eq. 5 summed, Eq. 13) with the pupil of Eq. 3."""
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
        M = A * torch.exp(1j * (theta + z[0] * kappa))
        r0 = N // 2 + int(g.n_int[i, 0]) - m // 2
        c0 = N // 2 + int(g.n_int[i, 1]) - m // 2
        psi = torch.fft.ifft2(torch.fft.ifftshift(O[r0:r0 + m, c0:c0 + m] * M))
        a = torch.sqrt(torch.clamp(torch.tensor(np.asarray(I[i], np.float64)), min=0.0))
        L = L + torch.sum((torch.sqrt(gamma[i]) * torch.abs(psi) - a) ** 2)
    return L


def test_reconstruction_step_matches_torch_autograd_and_optim():
    torch = pytest.importorskip("torch")
    g, _, _ = tiny_geometry(N=32, m=16, grid=3, pitch=3.0, R=5.0, edge="aa", seed=7)
    prm = generic_params(g, seed=4, z=2.0, off=0.3)
    rng = np.random.default_rng(8)
    O0 = rng.normal(size=(g.N, g.N)) + 1j * rng.normal(size=(g.N, g.N))
    # measured stack from a different object and parameters (a non-trivial loss)
    prm_t = generic_params(g, seed=9, z=1.0, off=0.2)
    I = orc.forward(O0 * (1 + 0.2 * rng.normal(size=O0.shape)), prm_t, g, range(g.n_leds))
    lr = dict(object=0.05, zernike=0.02, defocus=0.1, gamma=0.03, offset=0.05)
    hp = orc.Hparams(lr=lr, learn=("object", "zernike", "defocus", "gamma", "offset"), offset_bound=0.35)
    rec = orc.Reconstruction(g, I, hp, O0=O0, prm=prm)

    f64 = torch.float64
    t = dict(object=torch.tensor(O0, dtype=torch.complex128, requires_grad=True),
             zernike=torch.tensor(prm.zernike, dtype=f64, requires_grad=True),
             defocus=torch.tensor([prm.defocus], dtype=f64, requires_grad=True),
             gamma=torch.tensor(prm.gamma, dtype=f64, requires_grad=True),
             offset=torch.tensor(prm.offset, dtype=f64, requires_grad=True))
    opt = torch.optim.Adam([{"params": [t[k]], "lr": lr[k]} for k in t], betas=(0.9, 0.999), eps=1e-8)
    batches = [[0, 4, 8], [2, 5], [1, 7, 3, 6], [8, 0], [4, 2, 7]]
    for b in batches:
        L_ref = rec.step(b)
        opt.zero_grad()
        L = _torch_batch_loss(torch, g, I, t["object"], t["zernike"], t["defocus"], t["gamma"], t["offset"], b)
        L.backward()
        opt.step()
        with torch.no_grad():
            t["offset"].clamp_(-hp.offset_bound, hp.offset_bound)
            t["gamma"].clamp_(min=hp.gamma_floor)
        assert float(L.detach()) == pytest.approx(L_ref, rel=1e-11)
    np.testing.assert_allclose(rec.O, t["object"].detach().numpy(), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(rec.prm.zernike, t["zernike"].detach().numpy(), rtol=1e-10, atol=1e-12)
    assert rec.prm.defocus == pytest.approx(float(t["defocus"][0]), rel=1e-10)
    np.testing.assert_allclose(rec.prm.gamma, t["gamma"].detach().numpy(), rtol=1e-10)
    np.testing.assert_allclose(rec.prm.offset, t["offset"].detach().numpy(), rtol=1e-10, atol=1e-12)
    # the clamp was active: some offset sits on the bound after the steps
    assert np.any(np.isclose(np.abs(rec.prm.offset), hp.offset_bound))
