"""Pins for the oracle's forward model (Section 2.1, Eq. 1-3).

Each test fixes the oracle against something other than itself: direct
O(n^4) sums, Parseval, closed forms for constant and cosine-grating objects,
scipy's periodic linear interpolation, and the global-phase symmetry of |.|^2.
"""

import math

import numpy as np
import pytest

import oracle as orc
from synth import recipes as S
from tests.helpers import generic_params, tiny_geometry


def _brute_ifft2_centred(Phi):
    """psi(y, x) = (1/m^2) sum_p Phi(p) exp(+2 pi i (p_y y + p_x x)/m), p centred."""
    m = Phi.shape[0]
    p = np.arange(m) - m // 2
    r = np.arange(m)
    E = np.exp(2j * math.pi * np.outer(r, p) / m)       # [r, p]
    return E @ Phi @ E.T / (m * m)


def test_forward_field_matches_direct_sum():
    g, _, _ = tiny_geometry()
    prm = generic_params(g)
    rng = np.random.default_rng(0)
    O = rng.normal(size=(g.N, g.N)) + 1j * rng.normal(size=(g.N, g.N))
    for i in range(g.n_leds):
        Phi, psi, P = orc.forward_fields(O, prm, g, i)
        np.testing.assert_allclose(psi, _brute_ifft2_centred(Phi), rtol=0, atol=1e-12)
        # Parseval for the normalised inverse transform
        assert abs(np.sum(np.abs(psi) ** 2) - np.sum(np.abs(Phi) ** 2) / g.m ** 2) < 1e-10


def test_object_spectrum_matches_direct_sum():
    N, s = 16, 4
    rng = np.random.default_rng(1)
    o = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    k = np.arange(N) - N // 2
    r = np.arange(N)
    E = np.exp(-2j * math.pi * np.outer(k, r) / N)
    direct = E @ o @ E.T / s ** 2
    np.testing.assert_allclose(orc.object_spectrum(o, s), direct, atol=1e-11)


def test_constant_object_closed_form():
    # o = c everywhere: only the DC of O is non-zero (= c m^2), so LED i sees
    # |psi|^2 = |c|^2 A(-n_i - delta_i)^2 everywhere: bright field constant,
    # dark field zero.
    g, _, _ = tiny_geometry(edge="aa")
    prm = generic_params(g)
    c = 0.7 * np.exp(0.3j)
    O = orc.object_spectrum(np.full((g.N, g.N), c), g.s)
    I = orc.forward(O, prm, g, range(g.n_leds))
    for i in range(g.n_leds):
        q = -g.n_int[i] - prm.offset[i]
        A = float(np.clip(g.R + 0.5 - np.hypot(*q), 0.0, 1.0))
        np.testing.assert_allclose(I[i], prm.gamma[i] * abs(c) ** 2 * A ** 2, atol=1e-12)


def test_cosine_grating_closed_form():
    # o = 1 + eps cos(2 pi f.r / N): O has DC m^2 and two peaks eps m^2 / 2 at
    # +-f. With a hard aberration-free pupil and integer LED offsets, psi is
    # the sum of the admitted peaks, each a plane wave on the low-res grid.
    N, m, R, eps = 64, 16, 4.0, 0.4
    f = np.array([2, 5])
    nominal = np.array([[0, 0], [0, 3], [2, -4], [-3, 3], [5, 0], [1, 6]], float)
    g = orc.Geometry(N, m, nominal, R, "hard", 0.532, 1.0 / (m * 0.6))
    prm = orc.Params(np.zeros(14), 0.0, np.linspace(0.9, 1.1, len(nominal)), np.zeros_like(nominal))
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    o = 1 + eps * np.cos(2 * math.pi * (f[0] * yy + f[1] * xx) / N)
    I = orc.forward(orc.object_spectrum(o, g.s), prm, g, range(len(nominal)))
    ry, rx = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    for i, n in enumerate(g.n_int):
        psi = np.zeros((m, m), complex)
        for amp, k in ((1.0, np.zeros(2)), (eps / 2, f), (eps / 2, -f)):
            p = k - n                                    # position in the crop
            if np.hypot(*p) <= R and np.all(p >= -m // 2) and np.all(p < m // 2):
                psi += amp * np.exp(2j * math.pi * (p[0] * ry + p[1] * rx) / m)
        np.testing.assert_allclose(I[i], prm.gamma[i] * np.abs(psi) ** 2, atol=1e-12)


def test_global_phase_leaves_intensity_unchanged():
    g, _, _ = tiny_geometry()
    prm = generic_params(g)
    rng = np.random.default_rng(2)
    O = rng.normal(size=(g.N, g.N)) + 1j * rng.normal(size=(g.N, g.N))
    I1 = orc.forward(O, prm, g, range(g.n_leds))
    I2 = orc.forward(O * np.exp(0.83j), prm, g, range(g.n_leds))
    np.testing.assert_allclose(I1, I2, rtol=1e-12, atol=1e-12)


def test_pupil_pieces_closed_form():
    # Aberration-free, in-focus AA pupil: M = A exactly; defocus alone: the
    # phase is z * 2 pi (sqrt(lambda^-2 - |q dk|^2) - 1/lambda).
    g, _, _ = tiny_geometry(edge="aa")
    P = orc.pupil(g, np.zeros(14), 0.0, [0.2, -0.3])
    np.testing.assert_allclose(P["M"], P["A"], atol=0)
    assert P["A"].max() == 1.0 and P["A"].min() == 0.0
    z = 3.0
    P = orc.pupil(g, np.zeros(14), z, [0.0, 0.0])
    m = g.m
    p = np.arange(m) - m // 2
    qy, qx = np.meshgrid(p, p, indexing="ij")
    k = np.hypot(qy, qx) * g.dk_per_um
    inside = P["A"] > 0
    expect = z * 2 * math.pi * (np.sqrt(1 / g.lambda_um ** 2 - k ** 2) - 1 / g.lambda_um)
    np.testing.assert_allclose(P["chi"][inside], expect[inside], atol=1e-12)
    # piston removed: zero phase at the pupil centre
    assert abs(P["chi"][m // 2, m // 2]) < 1e-12


def test_bilinear_matches_scipy_periodic_linear_interpolation():
    # scipy's order-1 spline interpolation with periodic ('grid-wrap')
    # boundary, sampled at source coordinates Y/s.
    from scipy import ndimage
    rng = np.random.default_rng(3)
    a = rng.random((16, 12))
    for s in (2, 4):
        yy, xx = np.meshgrid(np.arange(16 * s) / s, np.arange(12 * s) / s, indexing="ij")
        ref = ndimage.map_coordinates(a, [yy, xx], order=1, mode="grid-wrap")
        np.testing.assert_allclose(orc.bilinear_upsample(a, s), ref, atol=1e-13)


def test_init_object_brightfield_consistency():
    # Initialising from a noise-free centre image of a pure-amplitude object
    # whose spectrum fits inside the pupil reproduces that image.
    N, m, s = 64, 16, 4
    g = orc.Geometry(N, m, np.zeros((1, 2)), 7.0, "hard", 0.532, 1.0 / (m * 0.6))
    prm = orc.Params.initial(g)
    yy, xx = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    amp_lr = 0.8 + 0.1 * np.cos(2 * math.pi * (yy + 2 * xx) / m)
    O0 = orc.init_object(amp_lr ** 2, s)
    assert np.isclose(O0[N // 2, N // 2].real, m * m * np.mean(orc.bilinear_upsample(amp_lr, s)))
    I = orc.forward(O0, prm, g, [0])[0]
    assert np.max(np.abs(np.sqrt(I) - amp_lr)) < 0.02


def test_recipes_shapes_and_ranges():
    o = S.make_object(64, 5)
    assert o.shape == (64, 64)
    assert np.abs(o).min() >= 0.5 - 1e-12 and np.abs(o).max() <= 1 + 1e-12
    assert np.abs(np.angle(o)).max() <= math.pi / 2 + 1e-12
    nom, tru = S.led_grid(15, 12, 0.5, 1)
    assert nom.shape == (225, 2) and np.all(nom[0] == 0)
    assert np.all(np.abs(tru - nom) <= 0.5)


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4_x4"])
def test_config_crops_fit(name):
    c = S.config(name)
    nom, tru = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
    n = np.rint(tru)
    assert np.all(np.abs(n) <= (c.N - c.m) // 2)
