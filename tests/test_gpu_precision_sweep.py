"""Precision sweep of the transform arithmetic on the noise-free plain recipe.

The 64-point recipe (256^2 / 64^2, 7 x 7 LEDs) and the same recipe scaled x4
(1024^2 / 256^2, pitch 32, R = 56) so that the low-res DFTs are 256-point.
Every form (FP32 FFTs; BF16, BF16X3, TF32, TF32X3 tensor-core DFTs) runs the
same 20-epoch reconstruction (object only, Adam lr 0.1, seeded batch order)
at batch sizes 8, 16 and 32 and is compared with the FP64 oracle run on the
same schedule: per-LED forward intensities at the truth, the object gradient
at the initial point, and the object after 20 epochs (relative L2). All
figures go to the parity report; the assertions hold the FP32 path and both
split forms (BF16X3, TF32X3) to the FP32 tolerances on intensities and
gradients, and every form to a finite, bounded trajectory error.
"""

import numpy as np
import pytest

import oracle as orc
from synth import recipes as S
from tests.gpu_common import engine_for, record, rel_l2, simulate

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FORMS = ("fp32_fft", "bf16", "bf16x3", "tf32", "tf32x3")
BATCHES = (8, 16, 32)
EPOCHS = 20
TOL_FP32 = dict(forward=1e-5, grad=1e-4, object=1e-3)
# bounds on the 20-epoch object error against the oracle: Adam turns rounding
# differences on elements with near-zero gradients into lr-sized steps, so the
# FP32 path itself drifts from the FP64 trajectory by ~1e-3 at some batch
# sizes (1.2e-3 measured at batch 16 on the 64-point recipe); the 1e-3 object
# tolerance is defined on the batch-8, 30-epoch run of the parity tests
BOUND = {"bf16": 0.5, "bf16x3": 0.05, "tf32": 0.5, "tf32x3": 5e-3, "fp32_fft": 5e-3}


def _engine(g, c, form):
    eng = engine_for(g)
    eng.set_hparams(lr=dict(c.lr), learn=c.learn, precision=form)
    return eng


def _reconstruct(eng, c, I, B, sched):
    eng.load(I, init=True)
    nb = -(-c.n_leds // B)
    for e in range(EPOCHS):
        ep = sched[e * nb:(e + 1) * nb]
        full = [b for b in ep if len(b) == B]
        if full:
            eng.run(np.stack(full))
        for b in ep:
            if len(b) != B:
                eng.step(b)
    return eng.get()["object"]


@pytest.mark.parametrize("name", ["c1", "c4_x4"])
def test_precision_sweep(name):
    c = S.config(name).with_(epochs=EPOCHS)
    I, o, g_n, g_t, prm_t = simulate(c)
    tag = f"sweep.{name}"
    # forward intensities at the truth and the object gradient at the initial point
    O_t = orc.object_spectrum(o, c.s)
    idx = np.arange(c.n_leds)
    ref_I = orc.forward(O_t, prm_t, g_t, idx)
    hp = orc.Hparams(lr=dict(c.lr), learn=c.learn)
    rec0 = orc.Reconstruction(g_n, I, hp)
    gidx = list(range(0, c.n_leds, 3))[:8]
    _, ref_g, _ = orc.loss_and_grad(rec0.O, rec0.prm, g_n, gidx, I.astype(np.float64), "amplitude")
    for form in FORMS:
        eng = engine_for(g_t)
        eng.set_hparams(precision=form)
        eng.set(object=O_t, zernike=prm_t.zernike, defocus=prm_t.defocus, gamma=prm_t.gamma, offset=prm_t.offset)
        got = eng.forward(idx)
        per_led = max(rel_l2(got[i], ref_I[i]) for i in idx if np.linalg.norm(ref_I[i]) > 0)
        record(f"{tag}.{form}.forward", rel_l2(got, ref_I))
        record(f"{tag}.{form}.forward_worst_led", per_led)
        eng.close()
        eng = _engine(g_n, c, form)
        eng.load(I, init=True)
        gg = eng.backward(gidx)["object"]
        record(f"{tag}.{form}.grad_object", rel_l2(gg, ref_g["object"]))
        eng.close()
        if form in ("fp32_fft", "bf16x3", "tf32x3"):
            assert rel_l2(got, ref_I) <= TOL_FP32["forward"]
            assert rel_l2(gg, ref_g["object"]) <= TOL_FP32["grad"]
    # 20-epoch reconstructions per batch size
    for B in BATCHES:
        sched = S.schedule(c.n_leds, B, EPOCHS, c.seed)
        rec = orc.Reconstruction(g_n, I, hp)
        rec.run(sched)
        for form in FORMS:
            eng = _engine(g_n, c, form)
            O = _reconstruct(eng, c, I, B, sched)
            eng.close()
            e = rel_l2(O, rec.O)
            ph = np.vdot(O, O_t)
            record(f"{tag}.B{B}.{form}.object", e)
            record(f"{tag}.B{B}.{form}.object_vs_truth", rel_l2(O * ph / abs(ph), O_t))
            assert np.isfinite(e) and e <= BOUND[form], (B, form, e)
        ph = np.vdot(rec.O, O_t)
        record(f"{tag}.B{B}.oracle.object_vs_truth", rel_l2(rec.O * ph / abs(ph), O_t))
