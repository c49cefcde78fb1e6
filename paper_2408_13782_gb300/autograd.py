"""torch.autograd.Function over the engine's forward model and hand-written adjoint.

    I = FpmForward.apply(engine, idx, O, zernike, defocus, gamma, offset)

computes the predicted intensities I[b] = gamma_i |psi_i|^2 for the LEDs
idx[b] (Section 2.1, Eq. 3) with fpm_forward, saving nothing but its inputs.
Backward receives dL/dI and calls fpm_backward, which recomputes the
low-res fields psi_i on the GPU (no field is stored between the passes) and
returns the gradients (with store_fields=True the fields are kept instead:
fpm_forward_fields / fpm_backward_fields, for the memory comparison) of O, the Zernike coefficients, z, gamma and the LED
offsets (convention for complex O: dL/dRe O + i dL/dIm O, which is what
PyTorch uses for complex leaves).

Argument marshalling only; every computation runs in the CUDA engine.
Tensors live on the engine's device: O is complex64 [N, N] (or float32
[N, N, 2]), zernike float32 [14], defocus float32 [1], gamma float32
[n_leds], offset float32 [n_leds, 2]; the result is float32 [B, m, m].
"""

from __future__ import annotations

import numpy as np
import torch

from .engine import Engine, _ptr, lib


def _as_pairs(O: torch.Tensor) -> torch.Tensor:
    if O.is_complex():
        return torch.view_as_real(O.to(torch.complex64).contiguous()).contiguous()
    return O.to(torch.float32).contiguous()


class FpmForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, engine: Engine, idx, O, zernike, defocus, gamma, offset, store_fields=False):
        idx = np.ascontiguousarray(np.asarray(idx, np.int32))
        Op = _as_pairs(O.detach())
        z = zernike.detach().to(torch.float32).contiguous()
        d = defocus.detach().to(torch.float32).reshape(1).contiguous()
        g = gamma.detach().to(torch.float32).contiguous()
        o = offset.detach().to(torch.float32).contiguous()
        engine._check(lib().fpm_set(engine.handle, _ptr(Op), _ptr(z), _ptr(d), _ptr(g), _ptr(o)))
        out = torch.empty((idx.size, engine.m, engine.m), dtype=torch.float32, device=Op.device)
        if store_fields:   # keep psi [B, m, m] (complex64) for the backward pass
            psi = torch.empty((idx.size, engine.m, engine.m, 2), dtype=torch.float32, device=Op.device)
            engine._check(lib().fpm_forward_fields(engine.handle, idx.ctypes.data, idx.size, _ptr(out), _ptr(psi)))
            ctx.save_for_backward(Op, z, d, g, o, psi)
        else:
            engine._check(lib().fpm_forward(engine.handle, idx.ctypes.data, idx.size, _ptr(out)))
            ctx.save_for_backward(Op, z, d, g, o)
        ctx.engine = engine
        ctx.idx = idx
        ctx.o_complex = O.is_complex()
        ctx.defocus_shape = defocus.shape
        ctx.store_fields = store_fields
        return out

    @staticmethod
    def backward(ctx, grad_I):
        engine, idx = ctx.engine, ctx.idx
        Op, z, d, g, o = ctx.saved_tensors[:5]
        # the engine holds the state of the last call; restore this call's inputs
        engine._check(lib().fpm_set(engine.handle, _ptr(Op), _ptr(z), _ptr(d), _ptr(g), _ptr(o)))
        dev = Op.device
        up = grad_I.to(torch.float32).contiguous()
        gO = torch.empty_like(Op)
        gz = torch.empty(14, dtype=torch.float32, device=dev)
        gd = torch.empty(1, dtype=torch.float32, device=dev)
        gg = torch.empty(engine.n_leds, dtype=torch.float32, device=dev)
        go = torch.empty((engine.n_leds, 2), dtype=torch.float32, device=dev)
        if ctx.store_fields:
            psi = ctx.saved_tensors[5]
            engine._check(lib().fpm_backward_fields(engine.handle, idx.ctypes.data, idx.size, _ptr(psi), _ptr(up),
                                                    _ptr(gO), _ptr(gz), _ptr(gd), _ptr(gg), _ptr(go)))
        else:
            engine._check(lib().fpm_backward(engine.handle, idx.ctypes.data, idx.size, _ptr(up), _ptr(gO),
                                             _ptr(gz), _ptr(gd), _ptr(gg), _ptr(go), None))
        gO_out = torch.view_as_complex(gO) if ctx.o_complex else gO
        return None, None, gO_out, gz, gd.reshape(ctx.defocus_shape), gg, go, None


def fpm_intensities(engine: Engine, idx, O, zernike, defocus, gamma, offset, store_fields=False) -> torch.Tensor:
    """Differentiable predicted intensities [B, m, m] for the LEDs idx.

    store_fields=False (default) recomputes the fields psi in the backward
    pass; True keeps them (B * m * m * 8 bytes) between the passes."""
    return FpmForward.apply(engine, idx, O, zernike, defocus, gamma, offset, store_fields)
