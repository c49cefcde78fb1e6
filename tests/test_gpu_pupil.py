"""The free-form pupil field (the pupil-recovery reading of Section 2.2) on the
GPU against the FP64 oracle, through the C ABI: forward intensities, every
gradient including the field's, steps with the field learned, in the per-LED
cluster form (m = 64, 128) and the dataflow form (m = 256); the unit field
reproduces the parametric model; the field travels with checkpoints.

The engine's field holds the W x W box nodes (|n| <= h); the oracle's holds
the m x m crop grid, so the engine's field is embedded in a field of ones.
"""

import numpy as np
import pytest

import oracle as orc
from paper_2408_13782_gb300 import FpmError
from tests.gpu_common import engine_for, hparams_to_engine, multiparam_problem, push, record, rel_l2

pytestmark = pytest.mark.gpu

TOL_I, TOL_G = 1e-5, 1e-4
ALL = ("object", "zernike", "defocus", "gamma", "offset", "pupil")


def _field(W, seed, amp=0.15):
    rng = np.random.default_rng(seed)
    return (1 + amp * rng.normal(size=(W, W))) * np.exp(1j * amp * rng.normal(size=(W, W)))


def _embed(P, m):
    W = P.shape[0]
    h = W // 2
    out = np.ones((m, m), np.complex128)
    out[m // 2 - h:m // 2 + h + 1, m // 2 - h:m // 2 + h + 1] = P
    return out


def _setup(m, form="auto", seed=91, grid=5):
    c, I, g, prm, O = multiparam_problem(m=m, grid=grid if m < 256 else 3, pitch=None if m < 256 else 32.0,
                                         R=None if m < 256 else 50.0, seed=seed)
    eng = engine_for(g)
    eng.set_step_form(form)
    P = _field(eng.box, seed + 1).astype(np.complex64).astype(np.complex128)
    prm.pupil_ff = _embed(P, g.m)
    return c, I, g, prm, O, eng, P


@pytest.mark.parametrize("m,form", [(64, "auto"), (128, "auto"), (256, "dataflow"), (256, "cluster")])
def test_forward_and_gradients_with_a_field(m, form):
    c, I, g, prm, O, eng, P = _setup(m, form)
    eng.load(I, init=False)
    push(eng, O, prm)
    eng.set_pupil(P)
    got_P, on = eng.get_pupil()
    assert on and np.array_equal(got_P, P)
    idx = np.arange(g.n_leds)
    err = rel_l2(eng.forward(idx), orc.forward(O, prm, g, idx))
    record(f"pupil.forward.m{m}.{form}", err)
    assert err <= TOL_I
    b = [i for i in (3, 0, 7, 1) if i < g.n_leds]
    got = eng.backward(b)
    L, ref, _ = orc.loss_and_grad(O, prm, g, b, I.astype(np.float64), "amplitude")
    assert abs(got["loss"] - L) <= TOL_I * L
    h = eng.box // 2
    ref_P = ref["pupil"][g.m // 2 - h:g.m // 2 + h + 1, g.m // 2 - h:g.m // 2 + h + 1]
    errs = {"object": rel_l2(got["object"], ref["object"]), "zernike": rel_l2(got["zernike"], ref["zernike"]),
            "defocus": rel_l2([got["defocus"]], [ref["defocus"]]), "gamma": rel_l2(got["gamma"], ref["gamma"]),
            "offset": rel_l2(got["offset"], ref["offset"]), "pupil": rel_l2(eng.pupil_gradient(), ref_P)}
    for k, v in errs.items():
        record(f"pupil.grad.m{m}.{form}.{k}", v)
        assert v <= TOL_G, (k, v)


def test_unit_field_is_the_parametric_model():
    c, I, g, prm, O, eng, P = _setup(64)
    eng.load(I, init=False)
    push(eng, O, prm)
    idx = np.arange(g.n_leds)
    I0 = eng.forward(idx)
    g0 = eng.backward([4, 1])
    eng.set_pupil(np.ones((eng.box, eng.box), np.complex128))
    assert rel_l2(eng.forward(idx), I0) <= 1e-6
    g1 = eng.backward([4, 1])
    for k in ("object", "zernike", "gamma", "offset"):
        assert rel_l2(g1[k], g0[k]) <= 1e-5, k
    eng.set_pupil(None)
    assert not eng.get_pupil()[1]
    assert np.array_equal(eng.forward(idx), I0)   # out of the model again: the parametric arithmetic


@pytest.mark.parametrize("m,form", [(64, "auto"), (256, "dataflow")])
def test_steps_with_the_field_learned(m, form):
    c, I, g, prm, O, eng, P = _setup(m, form, seed=93)
    hp = orc.Hparams(lr=dict(object=0.5, zernike=0.01, defocus=0.1, gamma=0.01, offset=0.01, pupil=0.02), learn=ALL)
    rec = orc.Reconstruction(g, I, hp, O0=O, prm=prm)
    hparams_to_engine(eng, hp)
    eng.load(I, init=False)
    push(eng, O, prm)
    eng.set_pupil(P)
    h = eng.box // 2
    sl = slice(g.m // 2 - h, g.m // 2 + h + 1)
    batches = [[3, 1, 8, 0], [5, 2], [7, 4, 6]] if g.n_leds > 8 else [[3, 1, 8, 0], [5], [2, 7, 6, 4]]
    for k, b in enumerate(batches):
        L_ref = rec.step(b)
        L_got = eng.step(b)
        assert abs(L_got - L_ref) <= 1e-5 * L_ref, (k, L_got, L_ref)
        st = eng.get()
        eo, ep = rel_l2(st["object"], rec.O), rel_l2(eng.get_pupil()[0], rec.prm.pupil_ff[sl, sl])
        record(f"pupil.steps.m{m}.k{k}.object", eo)
        record(f"pupil.steps.m{m}.k{k}.field", ep)
        assert eo <= 1e-4 and ep <= 1e-4, (k, eo, ep)
        for name, ref in (("zernike", rec.prm.zernike), ("gamma", rec.prm.gamma), ("offset", rec.prm.offset)):
            assert rel_l2(st[name], ref) <= 1e-4, (k, name)


def test_field_checkpoint_and_refusals():
    c, I, g, prm, O, eng, P = _setup(64, seed=95)
    eng.set_hparams(learn=("object", "pupil"), lr=dict(pupil=0.02))
    eng.load(I, init=True)
    got, on = eng.get_pupil()
    assert on and np.array_equal(got, np.ones_like(got))   # a learned field starts at 1
    sched = [[0, 1, 2, 3], [4, 5, 6], [7, 8, 9, 10]]
    eng.step(sched[0])
    state = eng.get_state()
    eng.step(sched[1])
    eng.step(sched[2])
    ref = eng.get_state()
    eng2 = engine_for(g)
    eng2.set_hparams(learn=("object", "pupil"), lr=dict(pupil=0.02))
    eng2.load(I, init=True)
    eng2.set_state(state)
    eng2.step(sched[1])
    eng2.step(sched[2])
    assert np.array_equal(eng2.get_state(), ref)
    with pytest.raises(FpmError):                  # learned: cannot be taken out
        eng.set_pupil(None)
    with pytest.raises(FpmError):                  # the tensor-core forms have no free-form factor
        eng.set_hparams(learn=("object", "pupil"), precision="bf16x3")
