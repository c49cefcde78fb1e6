"""Tensor-core DFT forms of the per-LED kernel vs the FP64 oracle and the FP32 FFT path.

The m-point DFTs of the forward model (Section 2.1, Eq. 3) and of its adjoint
run as tcgen05 contractions with BF16 or TF32 operands and FP32 accumulation;
the X3 forms split each operand into hi + lo and sum three products.

Error bounds per form follow from the operand rounding: a BF16 operand keeps
8 significant bits (unit roundoff u = 2^-9), TF32 11 (u = 2^-11); a depth-K
contraction of rounded operands has relative error of order u, and the
intensity |psi|^2 doubles it. The split forms drop only the lo*lo product and
the rounding of lo, so their error is of order u^2 (BF16: ~4e-6, TF32: ~2e-7)
plus the accumulation: the tensor cores add each MMA's products into the FP32
accumulator with truncation, and the DFT sums cancel, which leaves a floor of
a few 1e-6 on intensities at m = 256 for both split forms. The bounds below
sit a few times above those orders; TF32X3 is held to the FP32 path's own
tolerances (1e-5 forward, 1e-4 gradients, 1e-3 object after the fixed epoch
count).
"""

import numpy as np
import pytest

import oracle as orc
from paper_2408_13782_gb300 import FpmError
from synth import recipes as S
from tests.gpu_common import engine_for, multiparam_problem, push, record, rel_l2, simulate

pytestmark = pytest.mark.gpu

MODES = ("bf16", "bf16x3", "tf32", "tf32x3")
# the split forms are held to the FP32 path's tolerances (1e-5 / 1e-4)
TOL_I = {"bf16": 2e-2, "bf16x3": 1e-5, "tf32": 5e-3, "tf32x3": 1e-5}
TOL_G = {"bf16": 5e-2, "bf16x3": 1e-4, "tf32": 1e-2, "tf32x3": 1e-4}
TOL_O = {"bf16": 0.5, "bf16x3": 2e-2, "tf32": 0.2, "tf32x3": 1e-3}


def _grid(m):
    return 5 if m < 256 else 3


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m", [64, 128, 256])
def test_forward(m, mode):
    c, I, g, prm, O = multiparam_problem(m=m, grid=_grid(m))
    eng = engine_for(g)
    push(eng, O, prm)
    idx = np.arange(g.n_leds)
    fft = eng.forward(idx)
    eng.set_hparams(precision=mode)
    got = eng.forward(idx)
    ref = orc.forward(O, prm, g, idx)
    err = rel_l2(got, ref)
    record(f"gemm.forward.m{m}.{mode}", err)
    record(f"gemm.forward_vs_fft.m{m}.{mode}", rel_l2(got, fft))
    assert err <= TOL_I[mode]
    for i in idx:   # per image, dark field included
        assert rel_l2(got[i], ref[i]) <= 10 * TOL_I[mode]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m", [64, 256])
def test_gradients_builtin_loss(m, mode):
    c, I, g, prm, O = multiparam_problem(m=m, grid=_grid(m))
    eng = engine_for(g)
    eng.set_hparams(precision=mode)
    eng.load(I, init=False)
    push(eng, O, prm)
    idx = [i for i in (3, 0, 8, 7) if i < g.n_leds]
    got = eng.backward(idx)
    L, ref, _ = orc.loss_and_grad(O, prm, g, idx, I.astype(np.float64), "amplitude")
    errs = {"loss": abs(got["loss"] - L) / L}
    for k in ("object", "zernike", "defocus", "gamma", "offset"):
        a = [got[k]] if k == "defocus" else got[k]
        b = [ref[k]] if k == "defocus" else ref[k]
        if k in ("gamma", "offset"):
            a, b = np.asarray(a)[idx], np.asarray(b)[idx]
        errs[k] = rel_l2(a, b)
    for k, e in errs.items():
        record(f"gemm.grad.m{m}.{mode}.{k}", e)
    # the loss, a sum of squared amplitude residuals, is held to the gradient bound
    for k, e in errs.items():
        assert e <= TOL_G[mode], (k, e)


def test_gradients_upstream_tf32x3():
    c, I, g, prm, O = multiparam_problem(m=64, seed=9)
    eng = engine_for(g)
    eng.set_hparams(precision="tf32x3")
    push(eng, O, prm)
    idx = [1, 6, 2]
    w = np.random.default_rng(3).normal(size=(len(idx), g.m, g.m)).astype(np.float32)
    got = eng.backward(idx, dL_dI=w)
    Iw = np.zeros((g.n_leds, g.m, g.m))
    Iw[idx] = w
    _, ref, _ = orc.loss_and_grad(O, prm, g, idx, Iw, "linear")
    for k in ("object", "zernike", "gamma", "offset"):
        a, b = got[k], ref[k]
        if k in ("gamma", "offset"):
            a, b = np.asarray(a)[idx], np.asarray(b)[idx]
        e = rel_l2(a, b)
        record(f"gemm.upstream.tf32x3.{k}", e)
        assert e <= TOL_G["tf32x3"], (k, e)


@pytest.fixture(scope="module")
def c1_oracle_20():
    """Config 1 (noise-free, m = 64, 7 x 7 LEDs), batch 8, 20 epochs on the oracle."""
    c = S.config("c1").with_(epochs=20)
    I, o, g_n, g_t, prm_t = simulate(c)
    hp = orc.Hparams(lr=dict(c.lr), learn=c.learn)
    rec = orc.Reconstruction(g_n, I, hp)
    sched = S.schedule(g_n.n_leds, c.B, c.epochs, c.seed)
    rec.run(sched)
    return c, I, g_n, hp, sched, rec, o


def _run_engine(c, I, g, hp, sched, precision):
    eng = engine_for(g)
    eng.set_hparams(lr=dict(hp.lr), betas=(hp.beta1, hp.beta2), eps=hp.eps, loss=hp.loss, learn=hp.learn,
                    precision=precision)
    eng.load(I, init=True)
    nb = -(-g.n_leds // c.B)
    for e in range(c.epochs):
        ep = sched[e * nb:(e + 1) * nb]
        full = np.stack([b for b in ep if len(b) == c.B])
        eng.run(full)
        for b in ep:
            if len(b) != c.B:
                eng.step(b)
    return eng


@pytest.mark.parametrize("mode", MODES)
def test_trajectory_config1_20_epochs(mode, c1_oracle_20):
    c, I, g, hp, sched, rec, o = c1_oracle_20
    eng = _run_engine(c, I, g, hp, sched, mode)
    got = eng.get()["object"]
    eo = rel_l2(got, rec.O)
    record(f"gemm.trajectory.c1.{mode}.object", eo)
    # reconstruction quality against the truth (up to the global phase)
    O_t = orc.object_spectrum(o, c.s)
    ph = np.vdot(got, O_t)
    record(f"gemm.trajectory.c1.{mode}.vs_truth", rel_l2(got * ph / abs(ph), O_t))
    assert eo <= TOL_O[mode]


def test_precision_switch_and_rejections():
    c, I, g, prm, O = multiparam_problem(m=64)
    eng = engine_for(g)
    push(eng, O, prm)
    idx = np.arange(g.n_leds)
    a = eng.forward(idx)
    eng.set_hparams(precision="bf16")
    eng.set_hparams(precision="fp32_fft")
    assert np.array_equal(eng.forward(idx), a)   # back on the FFT path, bit for bit
    for m in (32, 512):
        c2, I2, g2, prm2, O2 = multiparam_problem(m=m, grid=3)
        e2 = engine_for(g2)
        with pytest.raises(FpmError):
            e2.set_hparams(precision="tf32")
        push(e2, O2, prm2)   # the handle stays usable on the FFT path
        e2.forward([0])
