"""The allocation-free gradient call against the handle-based one.

fpm_gradients_static exists for callers that cannot allocate device memory
(code running while a host framework owns the device memory pool, or real-time
loops where an allocation may block): every buffer is theirs, and the
intermediates live in a fixed static array inside the library. It must give
the same loss and gradients as fpm_backward, the existing entry point, within
the parity tests' tolerances (1e-5 on the loss, 1e-4 on every gradient), on
consecutive calls - the second call reuses the array the first one left behind.
This file is collected last so that a failure here stops a run only after all
other tests have run.
"""

import numpy as np
import pytest

from paper_2408_13782_gb300 import FpmError
from paper_2408_13782_gb300 import engine as E
from tests.gpu_common import engine_for, multiparam_problem, push, rel_l2

pytestmark = pytest.mark.gpu

TOL_LOSS, TOL_G = 1e-5, 1e-4


def _device_inputs(torch, O, prm, I):
    dev = torch.device("cuda", torch.cuda.current_device())
    Ot = np.ascontiguousarray(O.T)  # column-major: element (row y, col x) at x * N + y
    O_t = torch.from_numpy(np.stack([Ot.real, Ot.imag], -1).astype(np.float32)).to(dev)
    params = np.concatenate([prm.zernike, [prm.defocus], prm.gamma, prm.offset.ravel()]).astype(np.float32)
    return dev, O_t, torch.from_numpy(params).to(dev), torch.from_numpy(np.ascontiguousarray(I, np.float32)).to(dev)


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
    n = g.n_leds
    for batch in batches:
        ref = eng.backward(batch)
        gO_t = torch.full_like(O_t, float("nan"))
        gp = torch.full((15 + 3 * n,), float("nan"), dtype=torch.float32, device=dev)
        loss = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        E.gradients_static(g.m, g.s, g.nominal, g.R, g.lambda_um, g.dk_per_um, g.edge, O_t, params, stack,
                           batch, gO_t, gp, loss, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        go = gO_t.cpu().numpy()
        g_obj = (go[..., 0] + 1j * go[..., 1].astype(np.float64)).T
        gpv = gp.cpu().numpy().astype(np.float64)
        L = float(loss.cpu().numpy()[0])
        assert abs(L - ref["loss"]) <= TOL_LOSS * abs(ref["loss"])
        assert rel_l2(g_obj, ref["object"]) <= TOL_G
        assert rel_l2(gpv[:14], ref["zernike"]) <= TOL_G
        assert rel_l2([gpv[14]], [ref["defocus"]]) <= TOL_G
        assert rel_l2(gpv[15:15 + n], ref["gamma"]) <= TOL_G
        assert rel_l2(gpv[15 + n:].reshape(n, 2), ref["offset"]) <= TOL_G
    eng.close()


def test_static_gradients_reject_a_batch_larger_than_the_array():
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
