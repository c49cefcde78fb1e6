"""Pins for the oracle's gradients (the adjoint of Eq. 3 under the loss of Eq. 5).

Central finite differences in FP64 on every gradient, the global-phase
invariance, the zero gradient at the truth and the closed-form optimum of the
intensity factor.
"""

import math

import numpy as np
import pytest

import oracle as orc
from synth import recipes as S
from tests.helpers import generic_params, simulate, tiny_geometry


def _problem(edge="aa", loss="amplitude", seed=0):
    g, _, _ = tiny_geometry(edge=edge, seed=seed + 7)
    prm = generic_params(g, seed=seed + 3)
    rng = np.random.default_rng(seed)
    O = orc.object_spectrum(S.make_object(g.N, seed + 9), g.s)
    # measurements from a perturbed state so residuals are far from zero
    prm_m = generic_params(g, seed=seed + 30)
    I_meas = orc.forward(O * (1 + 0.3 * rng.normal(size=O.shape)), prm_m, g, range(g.n_leds))
    I_meas += 0.01 * rng.normal(size=I_meas.shape)
    idx = [0, 4, 7, 2]
    return g, prm, O, I_meas, idx, loss


def _L(O, prm, g, idx, I, loss):
    return orc.loss_and_grad(O, prm, g, idx, I, loss)[0]


def _fd(f, x0, h):
    return (f(x0 + h) - f(x0 - h)) / (2 * h)


def _check(num, ana, what, rtol=1e-6, scale=1.0):
    assert abs(num - ana) <= rtol * max(abs(ana), scale), f"{what}: fd {num} vs analytic {ana}"


@pytest.mark.parametrize("loss", ["amplitude", "intensity", "linear"])
def test_gradients_match_central_differences(loss):
    g, prm, O, I, idx, loss = _problem(loss=loss)
    L0, gr, _ = orc.loss_and_grad(O, prm, g, idx, I, loss)
    h = 1e-6
    sc = L0 * 1e-6
    rng = np.random.default_rng(5)
    # object entries on the union of the batch's supports
    sup = np.zeros(O.shape, bool)
    for i in idx:
        P = orc.pupil(g, prm.zernike, prm.defocus, prm.offset[i])
        orc.crop(sup, g, i)[...] |= P["A"] > 0
    cand = np.argwhere(sup)
    for (r, c) in cand[rng.choice(len(cand), 12, replace=False)]:
        for part, unit in (("re", 1.0), ("im", 1j)):
            def f(x, r=r, c=c, unit=unit):
                O2 = O.copy()
                O2[r, c] += unit * x
                return _L(O2, prm, g, idx, I, loss)
            ana = gr["object"][r, c].real if part == "re" else gr["object"][r, c].imag
            _check(_fd(f, 0.0, h * max(1.0, abs(O[r, c]))), ana, f"O[{r},{c}].{part}", scale=sc / h)
    for j in range(14):
        def f(x, j=j):
            p2 = prm.copy(); p2.zernike[j] = x
            return _L(O, p2, g, idx, I, loss)
        _check(_fd(f, prm.zernike[j], h), gr["zernike"][j], f"c{j + 2}", scale=sc)

    def fz(x):
        p2 = prm.copy(); p2.defocus = x
        return _L(O, p2, g, idx, I, loss)
    _check(_fd(fz, prm.defocus, h), gr["defocus"], "z", scale=sc)
    for i in range(g.n_leds):
        def fg(x, i=i):
            p2 = prm.copy(); p2.gamma[i] = x
            return _L(O, p2, g, idx, I, loss)
        _check(_fd(fg, prm.gamma[i], h), gr["gamma"][i], f"gamma{i}", scale=sc)
        for ax in (0, 1):
            def fo(x, i=i, ax=ax):
                p2 = prm.copy(); p2.offset[i, ax] = x
                return _L(O, p2, g, idx, I, loss)
            _check(_fd(fo, prm.offset[i, ax], h), gr["offset"][i, ax], f"delta{i},{ax}", scale=sc)
    # LEDs outside the batch get exactly zero gradient
    out = [i for i in range(g.n_leds) if i not in idx]
    assert np.all(gr["gamma"][out] == 0) and np.all(gr["offset"][out] == 0)


def test_hard_edge_object_gradient():
    g, prm, O, I, idx, loss = _problem(edge="hard")
    L0, gr, _ = orc.loss_and_grad(O, prm, g, idx, I, loss)
    r, c = g.N // 2 + int(g.n_int[idx[1], 0]) + 1, g.N // 2 + int(g.n_int[idx[1], 1]) - 2
    h = 1e-6 * abs(O[r, c])
    for unit, ana in ((1.0, gr["object"][r, c].real), (1j, gr["object"][r, c].imag)):
        def f(x):
            O2 = O.copy(); O2[r, c] += unit * x
            return _L(O2, prm, g, idx, I, loss)
        _check(_fd(f, 0.0, h), ana, "O hard", scale=L0 * 1e-6 / h)


def test_global_phase_direction_has_zero_gradient():
    # L(exp(i a) O) = L(O) for all a, so Re sum conj(grad_O) * (i O) = 0.
    g, prm, O, I, idx, loss = _problem()
    _, gr, _ = orc.loss_and_grad(O, prm, g, idx, I, loss)
    d = np.real(np.sum(np.conj(gr["object"]) * 1j * O))
    norm = np.linalg.norm(gr["object"]) * np.linalg.norm(O)
    assert abs(d) <= 1e-12 * norm


def test_zero_loss_and_gradient_at_truth():
    c = S.config("c1").with_(N=64, m=16, grid=5, pitch=2, R=4, edge="aa",
                              zernike_sigma=0.3, z_um=3.0, jitter=0.3,
                              gamma_range=(0.8, 1.2))
    I, o, g_n, g_t, prm_t = simulate(c, dtype=np.float64)
    O_t = orc.object_spectrum(o, c.s)
    L, gr, per = orc.loss_and_grad(O_t, prm_t, g_t, range(g_t.n_leds), I)
    assert L < 1e-20
    for k, v in gr.items():
        if v is not None:   # (no free-form pupil here: its gradient is None)
            assert np.max(np.abs(v)) < 1e-8, k


def test_gamma_optimum_closed_form():
    # For fixed psi the amplitude loss in gamma is minimised at
    # sqrt(gamma*) = sum(a |psi|) / sum(|psi|^2), where its gradient vanishes.
    g, prm, O, I, idx, loss = _problem()
    for i in idx:
        _, psi, _ = orc.forward_fields(O, prm, g, i)
        a = np.sqrt(np.maximum(I[i], 0))
        prm.gamma[i] = (np.sum(a * np.abs(psi)) / np.sum(np.abs(psi) ** 2)) ** 2
    _, gr, _ = orc.loss_and_grad(O, prm, g, idx, I, loss)
    L = _L(O, prm, g, idx, I, loss)
    assert np.max(np.abs(gr["gamma"][idx])) < 1e-9 * L


@pytest.mark.slow
def test_c3_gradients_central_difference_h1e3():
    # The differentiation workload at its full size (512^2 / 128^2, 9x9 LEDs,
    # batch 4), FP64 central differences with h = 1e-3 on sampled entries.
    c = S.config("c3")
    I, o, g_n, g_t, prm_t = simulate(c, dtype=np.float64)
    rng = np.random.default_rng(1)
    prm = prm_t.copy()
    prm.zernike += rng.normal(0, 0.05, 14)
    prm.defocus += 0.5
    prm.offset += rng.uniform(-0.1, 0.1, prm.offset.shape)
    O = orc.object_spectrum(o, c.s) * (1 + 0.05 * rng.normal(size=(c.N, c.N)))
    idx = [3, 17, 40, 66]
    L0, gr, _ = orc.loss_and_grad(O, prm, g_t, idx, I)
    h = 1e-3
    for j in (0, 5, 13):
        def f(x, j=j):
            p2 = prm.copy(); p2.zernike[j] = x
            return _L(O, p2, g_t, idx, I, "amplitude")
        _check(_fd(f, prm.zernike[j], h), gr["zernike"][j], f"c{j + 2}", rtol=1e-4, scale=L0 * 1e-7)

    def fz(x):
        p2 = prm.copy(); p2.defocus = x
        return _L(O, p2, g_t, idx, I, "amplitude")
    _check(_fd(fz, prm.defocus, h), gr["defocus"], "z", rtol=1e-4, scale=L0 * 1e-7)
    i = idx[2]
    for ax in (0, 1):
        def fo(x, ax=ax):
            p2 = prm.copy(); p2.offset[i, ax] = x
            return _L(O, p2, g_t, idx, I, "amplitude")
        _check(_fd(fo, prm.offset[i, ax], h), gr["offset"][i, ax], "delta", rtol=1e-3, scale=L0 * 1e-7)
    r, cc = c.N // 2 + int(g_t.n_int[i, 0]) + 3, c.N // 2 + int(g_t.n_int[i, 1]) - 5
    hO = h * abs(O[r, cc])

    def fO(x):
        O2 = O.copy(); O2[r, cc] += x
        return _L(O2, prm, g_t, idx, I, "amplitude")
    _check(_fd(fO, 0.0, hO), gr["object"][r, cc].real, "O", rtol=1e-4, scale=L0 * 1e-7 / hO)
