"""Pins for the update rule (Eq. 13 with Adam) and the batch schedule (Eq. 14)."""

import numpy as np
import pytest
import torch

import oracle as orc
from synth import recipes as S
from tests.helpers import simulate


def test_adam_first_step_closed_form():
    # From zero moments, bias correction makes the first step lr * g / (|g| + eps).
    rng = np.random.default_rng(0)
    g = rng.normal(size=100) * 10.0 ** rng.uniform(-6, 3, 100)
    w = np.zeros(100)
    orc.adam_update(w, g, np.zeros(100), np.zeros(100), 1, 0.1, 0.9, 0.999, 1e-8)
    np.testing.assert_allclose(w, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_matches_torch_on_complex_and_real():
    rng = np.random.default_rng(1)
    w0 = rng.normal(size=(6, 5)) + 1j * rng.normal(size=(6, 5))
    tw = torch.tensor(w0, dtype=torch.complex128, requires_grad=True)
    opt = torch.optim.Adam([tw], lr=0.05, betas=(0.9, 0.999), eps=1e-8)
    w = np.stack([w0.real, w0.imag], -1)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for t in range(1, 8):
        g = rng.normal(size=(6, 5)) + 1j * rng.normal(size=(6, 5))
        if t == 4:
            g[:2] = 0.0                       # zero-gradient rows still move by momentum
        opt.zero_grad()
        tw.grad = torch.tensor(g, dtype=torch.complex128)
        opt.step()
        orc.adam_update(w, np.stack([g.real, g.imag], -1), m, v, t, 0.05, 0.9, 0.999, 1e-8)
    np.testing.assert_allclose(w[..., 0] + 1j * w[..., 1], tw.detach().numpy(), rtol=1e-13, atol=1e-15)


def _torch_steps(opt, w0, grads):
    # FP64 default dtype: NAdam keeps its running momentum product as a scalar of that type
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    try:
        tw = torch.tensor(w0, dtype=torch.float64, requires_grad=True)
        o = opt([tw])
        for g in grads:
            o.zero_grad()
            tw.grad = torch.tensor(g, dtype=torch.float64)
            o.step()
    finally:
        torch.set_default_dtype(old)
    return tw.detach().numpy()


@pytest.mark.parametrize("name", ["adamw", "nadam", "rmsprop"])
def test_adam_family_matches_torch(name):
    """AdamW, NAdam and RMSprop of the oracle against torch.optim's implementations, on
    the (Re, Im) components, seven steps including one with zero gradient on some rows."""
    rng = np.random.default_rng(2)
    w0 = rng.normal(size=(6, 5, 2))
    grads = [rng.normal(size=(6, 5, 2)) * 10.0 ** rng.uniform(-3, 2) for _ in range(7)]
    grads[3][:2] = 0.0
    lr, b1, b2, eps, wd, psi = 0.05, 0.9, 0.999, 1e-8, 0.01, 0.004
    w, m, v, prod = w0.copy(), np.zeros_like(w0), np.zeros_like(w0), 1.0
    for t, g in enumerate(grads, start=1):
        if name == "adamw":
            orc.adamw_update(w, g, m, v, t, lr, b1, b2, eps, wd)
        elif name == "nadam":
            prod *= orc.nadam_mu(t, b1, psi)
            orc.nadam_update(w, g, m, v, t, lr, b1, b2, eps, prod, prod * orc.nadam_mu(t + 1, b1, psi), psi)
        else:
            orc.rmsprop_update(w, g, v, lr, b2, eps)
    opt = {"adamw": lambda p: torch.optim.AdamW(p, lr=lr, betas=(b1, b2), eps=eps, weight_decay=wd),
           "nadam": lambda p: torch.optim.NAdam(p, lr=lr, betas=(b1, b2), eps=eps, momentum_decay=psi),
           "rmsprop": lambda p: torch.optim.RMSprop(p, lr=lr, alpha=b2, eps=eps)}[name]
    np.testing.assert_allclose(w, _torch_steps(opt, w0, grads), rtol=1e-12, atol=1e-14)


def test_rmsprop_first_step_closed_form():
    # From a zero running mean the first step is lr * g / (sqrt(1 - alpha) |g| + eps).
    rng = np.random.default_rng(3)
    g = rng.normal(size=50) * 10.0 ** rng.uniform(-6, 3, 50)
    w = np.zeros(50)
    orc.rmsprop_update(w, g, np.zeros(50), 0.1, 0.99, 1e-8)
    np.testing.assert_allclose(w, -0.1 * g / (np.sqrt(0.01) * np.abs(g) + 1e-8), rtol=1e-12)


def test_nadam_schedule_and_first_step():
    # mu_t = b1 (1 - 0.96^(t psi) / 2); from zero moments the first step is
    # lr ((1 - mu_1) / (1 - mu_1) + mu_2 (1 - b1) / (1 - mu_1 mu_2)) g / (|g| + eps)
    b1, psi = 0.9, 0.004
    assert orc.nadam_mu(1, b1, psi) == pytest.approx(b1 * (1 - 0.5 * 0.96 ** psi), rel=1e-15)
    mu1, mu2 = orc.nadam_mu(1, b1, psi), orc.nadam_mu(2, b1, psi)
    g = np.array([2.0, -0.5, 1e-3])
    w = np.zeros(3)
    orc.nadam_update(w, g, np.zeros(3), np.zeros(3), 1, 0.1, b1, 0.999, 0.0, mu1, mu1 * mu2, psi)
    coef = 1.0 + mu2 * (1 - b1) / (1 - mu1 * mu2)
    np.testing.assert_allclose(w, -0.1 * coef * np.sign(g), rtol=1e-12)


def test_adam_zero_state_zero_gradient_is_noop():
    w = np.ones(4)
    orc.adam_update(w, np.zeros(4), np.zeros(4), np.zeros(4), 3, 0.1, 0.9, 0.999, 1e-8)
    assert np.all(w == 1.0)


def test_splitmix64_published_vector(golden_dir):
    ref = [int(l) for l in open(f"{golden_dir}/splitmix64_seed1234567.txt") if l.strip() and not l.startswith("#")]
    gen = S.splitmix64(1234567)
    assert [next(gen) for _ in range(5)] == ref


def test_paper_batching_example(golden_dir):
    lines = [l.split() for l in open(f"{golden_dir}/paper_batching_example.txt") if l.strip() and not l.startswith("#")]
    order = [int(x) for x in lines[0][1:]]
    batches = [[int(x) for x in l[1:]] for l in lines if l[0] == "batch"]
    N, B, K, n = (int(x) for x in [l for l in lines if l[0] == "eq14"][0][1:])
    assert [list(b) for b in S.chop(order, 3)] == batches
    # Eq. (14) for a pass of the non-random schedule
    sched = S.schedule(N, B, epochs=1, seed=0, shuffle=False)
    assert len(sched) == K
    counts = np.bincount(np.concatenate(sched), minlength=N)
    assert np.all(counts == B * K // N) and B * K // N == n


@pytest.mark.parametrize("n,B,epochs", [(49, 8, 30), (225, 16, 20), (9, 3, 4), (121, 40, 3)])
def test_schedule_equal_counts(n, B, epochs):
    sched = S.schedule(n, B, epochs, seed=123)
    assert len(sched) == epochs * -(-n // B)
    counts = np.bincount(np.concatenate(sched), minlength=n)
    assert np.all(counts == epochs)                # Eq. (14): every image equally often
    for e in range(epochs):                         # each pass is a permutation
        per = np.concatenate(sched[e * -(-n // B):(e + 1) * -(-n // B)])
        assert sorted(per) == list(range(n))
    assert all(len(set(b)) == len(b) for b in sched)
    assert S.epoch_permutation(n, 123, 0).tolist() != S.epoch_permutation(n, 123, 1).tolist()


def test_oracle_reconstruction_reduces_loss():
    c = S.config("c1")
    I, o, g_n, g_t, prm_t = simulate(c)
    rec = orc.Reconstruction(g_n, I, orc.Hparams(lr=dict(c.lr), learn=c.learn))
    sched = S.schedule(g_n.n_leds, c.B, 3, c.seed)
    per_epoch = len(sched) // 3
    losses = rec.run(sched)
    e0 = sum(losses[:per_epoch])
    e2 = sum(losses[-per_epoch:])
    assert e2 < 0.95 * e0


def test_intensity_factors_held_at_the_floor():
    """A step large enough to push some gamma below zero leaves it at the floor
    (the amplitude loss takes sqrt(gamma)); the others move as Adam says."""
    from tests.helpers import generic_params, tiny_geometry
    g, _, _ = tiny_geometry()
    prm = generic_params(g, seed=3)
    prm.gamma[:] = 0.5
    rng = np.random.default_rng(4)
    O = rng.normal(size=(g.N, g.N)) + 1j * rng.normal(size=(g.N, g.N))
    I = orc.forward(O, prm, g, range(g.n_leds)) * 0.2      # measured darker: every gamma gradient > 0
    hp = orc.Hparams(lr=dict(object=0.0, zernike=0.0, defocus=0.0, gamma=2.0, offset=0.0), learn=("gamma",))
    rec = orc.Reconstruction(g, I, hp, O0=O, prm=prm)
    rec.step([0, 1, 2])
    assert np.all(rec.prm.gamma[[0, 1, 2]] == hp.gamma_floor)      # 0.5 - ~2 < 0: held at the floor
    assert np.all(rec.prm.gamma[3:] == 0.5)                          # zero gradient, first step: no move
