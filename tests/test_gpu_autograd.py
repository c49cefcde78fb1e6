"""The torch.autograd.Function over the hand-written adjoint (differentiation workload:
512^2 / 128^2, 9x9 LEDs, batch 4), against the FP64 oracle and against FP64
central differences (h = 1e-3) of the oracle's loss."""

import numpy as np
import pytest

import oracle as orc
from synth import recipes as S
from tests.gpu_common import engine_for, record, rel_l2, simulate

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_G = 1e-4


@pytest.fixture(scope="module")
def c3():
    c = S.config("c3")
    I, o, g_n, g_t, prm_t = simulate(c)
    rng = np.random.default_rng(7)
    prm = prm_t.copy()
    prm.zernike = prm.zernike + rng.normal(0, 0.05, 14)
    prm.defocus += 0.5
    prm.offset = np.clip(prm.offset + rng.uniform(-0.1, 0.1, prm.offset.shape), -0.9, 0.9)
    O = orc.object_spectrum(o, c.s) * (1 + 0.05 * rng.normal(size=(c.N, c.N)))
    return c, I, g_t, prm, O


def _leaves(O, prm, dev):
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device=dev, requires_grad=True)
    Ot = torch.tensor(O.astype(np.complex64), device=dev, requires_grad=True)
    return Ot, t(prm.zernike), t([prm.defocus]), t(prm.gamma), t(prm.offset)


def _grads(leaves):
    Ot, z, d, g, o = leaves
    return dict(object=Ot.grad.cpu().numpy().astype(np.complex128), zernike=z.grad.cpu().numpy(),
                defocus=float(d.grad.cpu().numpy()[0]), gamma=g.grad.cpu().numpy(), offset=o.grad.cpu().numpy())


def _compare(tag, got, ref):
    for k in ("object", "zernike", "gamma", "offset"):
        e = rel_l2(got[k], ref[k])
        record(f"autograd.{tag}.{k}", e)
        assert e <= TOL_G, (tag, k, e)
    e = abs(got["defocus"] - ref["defocus"]) / max(abs(ref["defocus"]), 1e-30)
    record(f"autograd.{tag}.defocus", e)
    assert e <= TOL_G


def test_function_linear_functional_matches_oracle(c3):
    from paper_2408_13782_gb300.autograd import fpm_intensities
    c, I, g, prm, O = c3
    dev = torch.device("cuda", 0)
    eng = engine_for(g)
    idx = [3, 17, 40, 66]
    rng = np.random.default_rng(1)
    w = rng.normal(size=(len(idx), g.m, g.m))
    leaves = _leaves(O, prm, dev)
    Ipred = fpm_intensities(eng, idx, *leaves)
    assert Ipred.shape == (4, g.m, g.m) and Ipred.device == dev
    ref_I = orc.forward(O, prm, g, idx)
    record("autograd.forward", rel_l2(Ipred.detach().cpu().numpy(), ref_I))
    assert rel_l2(Ipred.detach().cpu().numpy(), ref_I) <= 1e-5
    (Ipred * torch.tensor(w, dtype=torch.float32, device=dev)).sum().backward()
    Iw = np.zeros((g.n_leds, g.m, g.m))
    Iw[idx] = w
    _, ref, _ = orc.loss_and_grad(O, prm, g, idx, Iw, "linear")
    _compare("linear", _grads(leaves), ref)


def test_function_under_a_torch_amplitude_loss(c3):
    # L = sum (sqrt(I_pred) - sqrt(max(I_meas, 0)))^2 written with torch ops on the
    # Function's output: autograd feeds dL/dI into the adjoint; the result must be
    # the oracle's amplitude-loss gradient.
    from paper_2408_13782_gb300.autograd import fpm_intensities
    c, I, g, prm, O = c3
    dev = torch.device("cuda", 0)
    eng = engine_for(g)
    idx = [5, 12, 70, 33]
    leaves = _leaves(O, prm, dev)
    Ipred = fpm_intensities(eng, idx, *leaves)
    a = torch.tensor(np.sqrt(np.maximum(I[idx], 0)), dtype=torch.float32, device=dev)
    L = ((torch.sqrt(Ipred) - a) ** 2).sum()
    L.backward()
    Lref, ref, _ = orc.loss_and_grad(O, prm, g, idx, I.astype(np.float64), "amplitude")
    assert abs(float(L) - Lref) <= 1e-5 * Lref
    _compare("amplitude", _grads(leaves), ref)


def test_function_against_central_differences(c3):
    from paper_2408_13782_gb300.autograd import fpm_intensities
    c, I, g, prm, O = c3
    dev = torch.device("cuda", 0)
    eng = engine_for(g)
    idx = [3, 17, 40, 66]
    rng = np.random.default_rng(2)
    w = rng.normal(size=(len(idx), g.m, g.m))
    leaves = _leaves(O, prm, dev)
    (fpm_intensities(eng, idx, *leaves) * torch.tensor(w, dtype=torch.float32, device=dev)).sum().backward()
    got = _grads(leaves)
    Iw = np.zeros((g.n_leds, g.m, g.m))
    Iw[idx] = w
    L = lambda O_, p_: orc.loss_and_grad(O_, p_, g, idx, Iw, "linear")[0]
    h = 1e-3
    L0 = abs(L(O, prm))
    for j in (0, 6, 13):
        p1, p2 = prm.copy(), prm.copy()
        p1.zernike[j] += h; p2.zernike[j] -= h
        fd = (L(O, p1) - L(O, p2)) / (2 * h)
        assert abs(got["zernike"][j] - fd) <= 1e-3 * abs(fd) + 1e-7 * L0, (j, got["zernike"][j], fd)
    p1, p2 = prm.copy(), prm.copy()
    p1.defocus += h; p2.defocus -= h
    fd = (L(O, p1) - L(O, p2)) / (2 * h)
    assert abs(got["defocus"] - fd) <= 1e-3 * abs(fd) + 1e-7 * L0
    i = idx[1]
    for ax in (0, 1):
        p1, p2 = prm.copy(), prm.copy()
        p1.offset[i, ax] += h; p2.offset[i, ax] -= h
        fd = (L(O, p1) - L(O, p2)) / (2 * h)
        assert abs(got["offset"][i, ax] - fd) <= 1e-2 * abs(fd) + 1e-7 * L0, (ax, got["offset"][i, ax], fd)
    p1, p2 = prm.copy(), prm.copy()
    p1.gamma[i] += h; p2.gamma[i] -= h
    fd = (L(O, p1) - L(O, p2)) / (2 * h)
    assert abs(got["gamma"][i] - fd) <= 1e-3 * abs(fd) + 1e-7 * L0
    r, col = c.N // 2 + int(g.n_int[i, 0]) + 2, c.N // 2 + int(g.n_int[i, 1]) - 3
    hO = h * abs(O[r, col])
    for unit, part in ((1.0, "re"), (1j, "im")):
        O1, O2 = O.copy(), O.copy()
        O1[r, col] += unit * hO; O2[r, col] -= unit * hO
        fd = (L(O1, prm) - L(O2, prm)) / (2 * hO)
        ana = got["object"][r, col].real if part == "re" else got["object"][r, col].imag
        assert abs(ana - fd) <= 1e-3 * abs(fd) + 1e-7 * L0 / hO, (part, ana, fd)


@pytest.mark.parametrize("m", [128, 512])
def test_stored_fields_equal_recomputed_bitwise(m):
    """Keeping psi between the passes gives the recompute path's gradients bit for bit
    (same kernels up to where psi is formed)."""
    from paper_2408_13782_gb300.autograd import fpm_intensities
    from tests.gpu_common import multiparam_problem
    c, I, g, prm, O = multiparam_problem(m=m, grid=5 if m < 512 else 3, seed=12)
    dev = torch.device("cuda", 0)
    eng = engine_for(g)
    idx = [4, 0, 7, 2] if g.n_leds > 7 else [4, 0, 2]
    w = torch.tensor(np.random.default_rng(2).normal(size=(len(idx), g.m, g.m)).astype(np.float32), device=dev)
    out = {}
    for store in (False, True):
        leaves = _leaves(O, prm, dev)
        I_pred = fpm_intensities(eng, idx, *leaves, store_fields=store)
        (I_pred * w).sum().backward()
        out[store] = (I_pred.detach().cpu().numpy(), _grads(leaves))
    assert np.array_equal(out[False][0], out[True][0])
    for k in ("object", "zernike", "gamma", "offset"):
        assert np.array_equal(out[False][1][k], out[True][1][k]), k
    assert out[False][1]["defocus"] == out[True][1]["defocus"]
