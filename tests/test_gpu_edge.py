"""Degenerate and boundary cases of the method on the GPU, against the FP64 oracle:
a single LED, an all-zero object (psi = 0 everywhere, where the amplitude
residual's psi/|psi| is defined as 0), LED offsets at the +-1 px bound of the
crop box, and an LED whose support touches the edge of the m x m window."""

import numpy as np
import pytest

import oracle as orc
from tests.gpu_common import engine_for, push, record, rel_l2
from tests.helpers import generic_params

pytestmark = pytest.mark.gpu

TOL_I, TOL_G = 1e-5, 1e-4


def _geom(nominal, m=64, s=4, R=14.0, edge="aa"):
    return orc.Geometry(m * s, m, np.asarray(nominal, np.float64).reshape(-1, 2), R, edge, 0.532, 1.0 / (m * 0.6))


def _object(g, seed):
    rng = np.random.default_rng(seed)
    o = (0.75 + 0.25 * rng.uniform(size=(g.N, g.N))) * np.exp(1j * rng.uniform(-1, 1, (g.N, g.N)))
    return orc.object_spectrum(o, g.s)


def _measured(I, seed):
    """Intensities that differ from the prediction by a random field (a uniform
    factor would make every phase gradient vanish: residual parallel to psi)."""
    rng = np.random.default_rng(seed)
    return (I * (1.0 + 0.2 * rng.standard_normal(I.shape))).astype(np.float32)


def _check_grad(tag, got, ref, idx):
    for k in ("object", "zernike", "gamma", "offset"):
        a, b = got[k], ref[k]
        if k in ("gamma", "offset"):
            a, b = np.asarray(a)[idx], np.asarray(b)[idx]
        e = rel_l2(a, b)
        record(f"edge.{tag}.{k}", e)
        assert np.all(np.isfinite(a)) and e <= TOL_G, (k, e)


def test_single_led():
    g = _geom([[0.3, -0.2]])
    prm = generic_params(g, seed=4)
    O = _object(g, 1)
    eng = engine_for(g)
    push(eng, O, prm)
    I = orc.forward(O, prm, g, [0])
    got = eng.forward([0])
    record("edge.single.forward", rel_l2(got, I))
    assert rel_l2(got, I) <= TOL_I
    meas = _measured(I, 11)
    eng.load(meas, init=False)
    push(eng, O, prm)
    out = eng.backward([0])
    L, ref, _ = orc.loss_and_grad(O, prm, g, [0], meas.astype(np.float64), "amplitude")
    assert abs(out["loss"] - L) <= TOL_I * L
    _check_grad("single", out, ref, [0])


def test_zero_object_gives_zero_field_and_finite_gradients():
    g = _geom([[0, 0], [0, 8], [8, -8]])
    prm = generic_params(g, seed=5)
    O = np.zeros((g.N, g.N), np.complex128)
    eng = engine_for(g)
    push(eng, O, prm)
    assert np.array_equal(eng.forward([0, 1, 2]), np.zeros((3, g.m, g.m), np.float32))
    meas = np.random.default_rng(2).uniform(0, 2, (g.n_leds, g.m, g.m)).astype(np.float32)
    eng.load(meas, init=False)
    push(eng, O, prm)
    out = eng.backward([0, 1, 2])
    L, ref, _ = orc.loss_and_grad(O, prm, g, [0, 1, 2], meas.astype(np.float64), "amplitude")
    assert abs(out["loss"] - L) <= TOL_I * L           # = sum of the measured intensities
    # psi = 0: every gradient is exactly 0 (psi/|psi| := 0), on both sides
    for k in ("object", "zernike", "gamma", "offset"):
        assert not np.any(np.asarray(ref[k])), k
        assert not np.any(np.asarray(out[k])), k


@pytest.mark.parametrize("edge", ["aa", "hard"])
def test_offsets_at_the_bound(edge):
    g = _geom([[0, 0], [0, 8], [8, 0], [-8, -8]], edge=edge)
    prm = generic_params(g, seed=6)
    prm.offset = np.array([[1.0, -1.0], [-1.0, 1.0], [1.0, 1.0], [-1.0, -1.0]])   # the clamp bound
    O = _object(g, 3)
    eng = engine_for(g)
    push(eng, O, prm)
    idx = np.arange(g.n_leds)
    I = orc.forward(O, prm, g, idx)
    got = eng.forward(idx)
    record(f"edge.bound.{edge}.forward", rel_l2(got, I))
    assert rel_l2(got, I) <= TOL_I
    meas = _measured(I, 12)
    eng.load(meas, init=False)
    push(eng, O, prm)
    out = eng.backward(idx)
    L, ref, _ = orc.loss_and_grad(O, prm, g, idx, meas.astype(np.float64), "amplitude")
    _check_grad(f"bound.{edge}", out, ref, idx)


def test_support_at_the_window_edge():
    """The widest box the m x m window holds: R so that 2h + 1 = m - 1 (h = 31 at m = 64)."""
    m = 64
    R = 28.5   # h = floor(R + 1/2 + sqrt 2) + 1 = 31
    g = _geom([[0, 0], [1, -1]], m=m, R=R)
    prm = generic_params(g, seed=8, off=0.3)
    O = _object(g, 4)
    eng = engine_for(g)
    push(eng, O, prm)
    idx = [0, 1]
    I = orc.forward(O, prm, g, idx)
    got = eng.forward(idx)
    record("edge.window.forward", rel_l2(got, I))
    assert rel_l2(got, I) <= TOL_I
    meas = _measured(I, 13)
    eng.load(meas, init=False)
    push(eng, O, prm)
    out = eng.backward(idx)
    L, ref, _ = orc.loss_and_grad(O, prm, g, idx, meas.astype(np.float64), "amplitude")
    _check_grad("window", out, ref, idx)
