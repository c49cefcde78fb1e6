"""The allocation-free gradient call against the handle-based one and the oracle.

fpm_gradients_static exists for callers that cannot allocate device memory
(code running while a host framework owns the device memory pool, or real-time
loops where an allocation may block): every buffer is theirs, and the
intermediates live in a fixed static array inside the library. It must give
the same loss and gradients as fpm_backward, the existing entry point, within
the parity tests' tolerances (1e-5 on the loss, 1e-4 on every gradient), on
consecutive calls - the second call reuses the array the first one left behind
- for both losses and both pupil edges, with offsets at the bound; and the
same as the FP64 oracle. Its optional err_out reports the kernels' error bits.
This file is collected last so that a failure here stops a run only after all
other tests have run.
"""

import numpy as np
import pytest

import oracle as orc
from paper_2408_13782_gb300 import FpmError
from paper_2408_13782_gb300 import engine as E
from tests.gpu_common import engine_for, multiparam_problem, push, rel_l2

pytestmark = pytest.mark.gpu

TOL_LOSS, TOL_G = 1e-5, 1e-4
BOUND = 1.0  # FPM_OFFSET_BOUND_PX


def _device_inputs(torch, O, prm, I):
    dev = torch.device("cuda", torch.cuda.current_device())
    Ot = np.ascontiguousarray(O.T)  # column-major: element (row y, col x) at x * N + y
    O_t = torch.from_numpy(np.stack([Ot.real, Ot.imag], -1).astype(np.float32)).to(dev)
    params = np.concatenate([prm.zernike, [prm.defocus], prm.gamma, prm.offset.ravel()]).astype(np.float32)
    return dev, O_t, torch.from_numpy(params).to(dev), torch.from_numpy(np.ascontiguousarray(I, np.float32)).to(dev)


def _call(torch, g, dev, O_t, params, stack, batch, loss="amplitude"):
    n = g.n_leds
    gO_t = torch.full_like(O_t, float("nan"))
    gp = torch.full((15 + 3 * n,), float("nan"), dtype=torch.float32, device=dev)
    L = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    err = torch.full((1,), -1, dtype=torch.int32, device=dev)
    E.gradients_static(g.m, g.s, g.nominal, g.R, g.lambda_um, g.dk_per_um, g.edge, O_t, params, stack,
                       batch, gO_t, gp, L, loss=loss, stream=torch.cuda.current_stream().cuda_stream, err_out=err)
    torch.cuda.synchronize()
    go = gO_t.cpu().numpy()
    gpv = gp.cpu().numpy().astype(np.float64)
    return dict(object=(go[..., 0] + 1j * go[..., 1].astype(np.float64)).T, zernike=gpv[:14],
                defocus=float(gpv[14]), gamma=gpv[15:15 + n], offset=gpv[15 + n:].reshape(n, 2),
                loss=float(L.cpu().numpy()[0]), err=int(err.cpu().numpy()[0]))


def _assert_close(got, ref):
    assert abs(got["loss"] - ref["loss"]) <= TOL_LOSS * abs(ref["loss"])
    assert rel_l2(got["object"], ref["object"]) <= TOL_G
    assert rel_l2(got["zernike"], ref["zernike"]) <= TOL_G
    assert rel_l2([got["defocus"]], [ref["defocus"]]) <= TOL_G
    assert rel_l2(got["gamma"], ref["gamma"]) <= TOL_G
    assert rel_l2(got["offset"], ref["offset"]) <= TOL_G


@pytest.mark.parametrize("m,grid,batches", [
    (64, 5, ([3, 0, 11, 7], [5, 1, 2, 9, 20, 13])),
    (256, 15, (list(range(100, 116)), list(range(16)))),
])
def test_static_gradients_equal_backward_on_consecutive_calls(m, grid, batches):
    torch = pytest.importorskip("torch")
    c, I, g, prm, O = multiparam_problem(m=m, grid=grid, pitch=12.0 if m == 256 else None,
                                         R=50.0 if m == 256 else None, seed=71)
    eng = engine_for(g)
    eng.load(I, init=False)
    push(eng, O, prm)
    dev, O_t, params, stack = _device_inputs(torch, O, prm, I)
    for batch in batches:
        got = _call(torch, g, dev, O_t, params, stack, batch)
        assert got["err"] == 0
        _assert_close(got, eng.backward(batch))
    eng.close()


@pytest.mark.parametrize("loss,edge", [("amplitude", "hard"), ("intensity", "aa"), ("intensity", "hard")])
def test_static_gradients_losses_edges_and_offsets_at_the_bound(loss, edge):
    """Both losses and pupil edges, every offset of the batch at +-bound (the widest
    support the crop box is sized for), against fpm_backward and the oracle."""
    torch = pytest.importorskip("torch")
    c, I, g, prm, O = multiparam_problem(m=64, grid=5, edge=edge, seed=73)
    rng = np.random.default_rng(5)
    batch = [7, 12, 2, 18, 0]
    prm.offset[batch] = BOUND * rng.choice([-1.0, 1.0], size=(len(batch), 2))
    eng = engine_for(g)
    eng.set_hparams(loss=loss)
    eng.load(I, init=False)
    push(eng, O, prm)
    dev, O_t, params, stack = _device_inputs(torch, O, prm, I)
    got = _call(torch, g, dev, O_t, params, stack, batch, loss=loss)
    assert got["err"] == 0
    _assert_close(got, eng.backward(batch))
    L, ref, _ = orc.loss_and_grad(O, prm, g, batch, I.astype(np.float64), loss)
    _assert_close(got, dict(ref, loss=L))
    eng.close()


def test_static_gradients_report_an_offset_beyond_the_bound():
    torch = pytest.importorskip("torch")
    c, I, g, prm, O = multiparam_problem(m=64, grid=5, seed=74)
    prm.offset[3] = [1.5, -0.2]
    dev, O_t, params, stack = _device_inputs(torch, O, prm, I)
    assert _call(torch, g, dev, O_t, params, stack, [1, 2])["err"] == 0      # LED 3 not in the batch
    assert _call(torch, g, dev, O_t, params, stack, [1, 3, 2])["err"] == 8   # FPM_DEVERR_OFFSET
    assert _call(torch, g, dev, O_t, params, stack, [4])["err"] == 0        # cleared by the next call


def test_static_gradients_reject_a_batch_larger_than_the_array_and_capture():
    torch = pytest.importorskip("torch")
    c, I, g, prm, O = multiparam_problem(m=256, grid=15, pitch=12.0, R=50.0, seed=72)
    dev, O_t, params, stack = _device_inputs(torch, O, prm, I)
    gO_t = torch.empty_like(O_t)
    gp = torch.empty(15 + 3 * g.n_leds, device=dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    with pytest.raises(FpmError) as e:   # 64 boxes of 105^2 complex values: 5.6 MB > 4 MB
        E.gradients_static(g.m, g.s, g.nominal, g.R, g.lambda_um, g.dk_per_um, g.edge, O_t, params, stack,
                           list(range(64)), gO_t, gp, loss)
    assert e.value.code == -2 and "static array holds" in str(e.value)
    # a call on a stream being captured is refused (its host tables cannot be recorded)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with pytest.raises(FpmError) as e:
        with torch.cuda.graph(graph, stream=s, capture_error_mode="relaxed"):
            E.gradients_static(g.m, g.s, g.nominal, g.R, g.lambda_um, g.dk_per_um, g.edge, O_t, params, stack,
                               list(range(8)), gO_t, gp, loss, stream=s.cuda_stream)
    assert e.value.code == -8
