"""Degenerate and boundary cases of the method on the GPU, against the FP64 oracle:
a single LED, an all-zero object (psi = 0 everywhere, where the amplitude
residual's psi/|psi| is defined as 0), LED offsets at the +-1 px bound of the
crop box, and an LED whose support touches the edge of the m x m window."""

import numpy as np
import pytest

import oracle as orc
from paper_2408_13782_gb300 import FpmError
from tests.gpu_common import engine_for, multiparam_problem, push, record, rel_l2
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


def test_memory_limit_refuses_growth_and_keeps_the_handle_usable():
    """Failure injection on the host: a device-memory limit below what a larger
    batch needs makes that step fail with FPM_ERR_OOM before any buffer is
    touched; the handle then runs smaller batches, and after the limit is lifted
    the larger one, with the same results as a handle that never failed."""
    c, I, g, prm, O = multiparam_problem(m=64, grid=5, seed=81)
    sched = [[0, 5, 9], [3, 1, 12, 7, 20, 24, 2, 8, 15, 11, 6, 4], [2, 22]]
    ref = engine_for(g)
    ref.load(I, init=True)
    for b in sched:
        ref.step(b)
    eng = engine_for(g)
    eng.load(I, init=True)
    eng.step(sched[0])
    used = eng.memory_used()
    assert used > 0
    eng.set_memory_limit(used + 1024)          # room for nothing larger than the 3-LED batch buffers
    with pytest.raises(FpmError) as e:
        eng.step(sched[1])
    assert e.value.code == -4 and "limit" in str(e.value)
    assert eng.memory_used() == used            # nothing was freed or allocated
    eng.set_memory_limit(0)                     # lifted: the same step now runs
    eng.step(sched[1])
    eng.step(sched[2])
    assert np.array_equal(eng.get_state(), ref.get_state())


def test_intensity_factors_held_at_the_floor_like_the_oracle():
    c, I, g, prm, O = multiparam_problem(m=64, grid=5, seed=83)
    prm.gamma[:] = 0.5
    I_dark = (orc.forward(O, prm, g, range(g.n_leds)) * 0.2).astype(np.float32)
    hp = orc.Hparams(lr=dict(object=0.0, zernike=0.0, defocus=0.0, gamma=2.0, offset=0.0), learn=("gamma",))
    rec = orc.Reconstruction(g, I_dark, hp, O0=O, prm=prm)
    rec.step([0, 1, 2])
    eng = engine_for(g)
    eng.set_hparams(lr=dict(object=0.0, zernike=0.0, defocus=0.0, gamma=2.0, offset=0.0), learn=("gamma",))
    eng.load(I_dark, init=False)
    push(eng, O, prm)
    eng.step([0, 1, 2])
    got = eng.get()["gamma"]
    assert np.all(got[[0, 1, 2]] == np.float32(1e-3))
    np.testing.assert_allclose(got, rec.prm.gamma, rtol=1e-6)
