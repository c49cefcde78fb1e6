"""ctypes binding of the GB300 Batch-FPM engine (include/fpm.h).

Argument marshalling only: every computation runs in the CUDA library. Arrays
may be numpy arrays (host) or torch tensors (host or CUDA); the library infers
the copy direction from unified addressing. Importing works without a GPU;
creating an engine needs the built library and a CUDA device, and fails with
FpmError otherwise (there is no fallback path).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfpm_gb300.so")

FPM_OK = 0
ERRORS = {-1: "FPM_ERR_ARG", -2: "FPM_ERR_SHAPE", -3: "FPM_ERR_RANGE", -4: "FPM_ERR_OOM",
          -5: "FPM_ERR_NONFINITE", -6: "FPM_ERR_TIMEOUT", -7: "FPM_ERR_CUDA", -8: "FPM_ERR_STATE"}
EDGE = {"aa": 0, "hard": 1}
LOSS = {"amplitude": 0, "intensity": 1}
LEARN = {"object": 1, "zernike": 2, "defocus": 4, "gamma": 8, "offset": 16, "pupil": 32}
# transform arithmetic: FP32 shared-memory FFTs, or the DFT as tensor-core
# contractions with BF16 / TF32 operands (x3: hi + lo split, three products)
PRECISION = {"fp32_fft": 0, "bf16": 1, "bf16x3": 2, "tf32": 3, "tf32x3": 4}
OPTIMIZER = {"adam": 0, "adamw": 1, "nadam": 2, "rmsprop": 3}
# kernels of a step: the per-LED cluster form, or the dataflow form (m = 256)
STEP_FORM = {"auto": 0, "cluster": 1, "dataflow": 2}
LOAD_INIT = 1

# every symbol include/fpm.h declares
EXPORTS = ("fpm_create", "fpm_set_hparams", "fpm_get_hparams", "fpm_load", "fpm_step", "fpm_run",
           "fpm_epoch_loss", "fpm_profile_run", "fpm_forward", "fpm_backward",
           "fpm_forward_fields", "fpm_backward_fields", "fpm_get", "fpm_set", "fpm_set_object_field",
           "fpm_state_size", "fpm_get_state", "fpm_set_state", "fpm_dims", "fpm_epoch_permutation",
           "fpm_gradients_static", "fpm_job_footprint", "fpm_server_create", "fpm_server_submit",
           "fpm_server_tick", "fpm_server_status", "fpm_server_result", "fpm_server_clock", "fpm_server_stats",
           "fpm_server_error", "fpm_server_destroy", "fpm_destroy", "fpm_last_error",
           "fpm_set_step_form", "fpm_get_step_form", "fpm_check_wait_timeout", "fpm_probe_fp32_fma",
           "fpm_set_memory_limit", "fpm_memory_used", "fpm_server_set_admission", "fpm_server_set_grouping",
           "fpm_set_pupil", "fpm_get_pupil", "fpm_pupil_gradient")


class FpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n_leds", ctypes.c_int32), ("led_offset", ctypes.c_void_p),
                ("lambda_um", ctypes.c_float), ("dk_per_um", ctypes.c_float), ("pupil_edge", ctypes.c_int32)]


class Hparams(ctypes.Structure):
    _fields_ = [("lr_object", ctypes.c_float), ("lr_zernike", ctypes.c_float), ("lr_defocus", ctypes.c_float),
                ("lr_gamma", ctypes.c_float), ("lr_offset", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("loss", ctypes.c_int32),
                ("learn_mask", ctypes.c_uint32), ("precision", ctypes.c_int32), ("optimizer", ctypes.c_int32),
                ("weight_decay", ctypes.c_float), ("lr_pupil", ctypes.c_float)]


_lib = None


def lib():
    """Load the engine library (raises FpmError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FpmError(-7, f"engine library missing at {LIB_PATH}; build it with "
                           "paper_2408_13782_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, f32p, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p
    sig = {
        "fpm_create": ([ctypes.POINTER(Geometry), ctypes.c_float, i32, vp, ctypes.POINTER(vp)], i32),
        "fpm_set_hparams": ([vp, ctypes.POINTER(Hparams)], i32),
        "fpm_get_hparams": ([vp, ctypes.POINTER(Hparams)], i32),
        "fpm_load": ([vp, f32p, i32], i32),
        "fpm_step": ([vp, vp, i32, dp], i32),
        "fpm_run": ([vp, vp, i32, i32, dp], i32),
        "fpm_epoch_loss": ([vp, dp, i32], i32),
        "fpm_profile_run": ([vp, vp, i32, i32, vp, ctypes.c_int64, vp, vp, vp], i32),
        "fpm_forward": ([vp, vp, i32, f32p], i32),
        "fpm_backward": ([vp, vp, i32, f32p, f32p, f32p, f32p, f32p, f32p, dp], i32),
        "fpm_forward_fields": ([vp, vp, i32, f32p, f32p], i32),
        "fpm_backward_fields": ([vp, vp, i32, f32p, f32p, f32p, f32p, f32p, f32p, f32p], i32),
        "fpm_get": ([vp, f32p, f32p, f32p, f32p, f32p], i32),
        "fpm_set": ([vp, f32p, f32p, f32p, f32p, f32p], i32),
        "fpm_set_object_field": ([vp, f32p], i32),
        "fpm_state_size": ([vp], ctypes.c_int64),
        "fpm_get_state": ([vp, f32p], i32),
        "fpm_set_state": ([vp, f32p], i32),
        "fpm_dims": ([vp, vp, vp, vp, vp], i32),
        "fpm_epoch_permutation": ([i32, ctypes.c_uint64, i32, vp], i32),
        "fpm_gradients_static": ([ctypes.POINTER(Geometry), ctypes.c_float, i32, vp, vp, vp, vp, i32, i32,
                                  vp, vp, vp, vp, vp], i32),
        "fpm_set_step_form": ([vp, i32], i32),
        "fpm_get_step_form": ([vp, vp, vp], i32),
        "fpm_check_wait_timeout": ([vp, vp, i32, ctypes.c_double], i32),
        "fpm_probe_fp32_fma": ([i32, i32, vp, vp], i32),
        "fpm_set_memory_limit": ([vp, ctypes.c_int64], i32),
        "fpm_set_pupil": ([vp, f32p], i32),
        "fpm_get_pupil": ([vp, f32p, vp], i32),
        "fpm_pupil_gradient": ([vp, f32p], i32),
        "fpm_memory_used": ([vp], ctypes.c_int64),
        "fpm_destroy": ([vp], None),
        "fpm_last_error": ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _ptr(x):
    """Address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous, "array must be C-contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr()
    raise TypeError(type(x))


def epoch_permutation(n: int, seed: int, epoch: int) -> np.ndarray:
    out = np.empty(n, np.int32)
    rc = lib().fpm_epoch_permutation(n, seed & ((1 << 64) - 1), epoch, out.ctypes.data)
    if rc:
        raise FpmError(rc, "bad arguments")
    return out


def probe_fp32_fma(iters: int = 4096, reps: int = 5):
    """fpm_probe_fp32_fma: measured FP32 FMA throughput of the current device, TFLOP/s."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib().fpm_probe_fp32_fma(iters, reps, ctypes.byref(t), ctypes.byref(ms))
    if rc:
        raise FpmError(rc, "FP32 FMA probe failed")
    return t.value, ms.value


def gradients_static(m, upsample, led_offset, pupil_radius, lambda_um, dk_per_um, edge, O_t, params, stack,
                     idx, g_object_t, g_params, loss_out, loss="amplitude", stream=0, err_out=None):
    """fpm_gradients_static: loss and gradients with caller-owned device buffers only.

    For callers that cannot allocate device memory (see include/fpm.h). O_t,
    params, stack, g_object_t, g_params, loss_out (and err_out, an int32 [1]
    tensor, optional) are CUDA tensors of the current device (column-major O and
    gradient: element (row y, col x) at x * N + y); idx is a host sequence."""
    import torch
    off = np.ascontiguousarray(np.asarray(led_offset, np.float32).reshape(-1, 2))
    n, N = off.shape[0], m * upsample
    dev = torch.cuda.current_device()
    want = {"O_t": (O_t, torch.float32, N * N * 2), "params": (params, torch.float32, 15 + 3 * n),
            "stack": (stack, torch.float32, n * m * m), "g_object_t": (g_object_t, torch.float32, N * N * 2),
            "g_params": (g_params, torch.float32, 15 + 3 * n), "loss_out": (loss_out, torch.float64, 1)}
    if err_out is not None:
        want["err_out"] = (err_out, torch.int32, 1)
    for name, (t, dt, numel) in want.items():
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev and t.dtype == dt
                and t.numel() == numel and t.is_contiguous()):
            raise FpmError(-1, f"{name}: want a contiguous {dt} CUDA tensor of {numel} elements on device {dev}")
    g = Geometry(m, n, off.ctypes.data, lambda_um, dk_per_um, EDGE[edge])
    b = np.ascontiguousarray(np.asarray(idx, np.int32))
    rc = lib().fpm_gradients_static(ctypes.byref(g), pupil_radius, upsample, _ptr(O_t), _ptr(params), _ptr(stack),
                                    b.ctypes.data, b.size, LOSS[loss], _ptr(g_object_t), _ptr(g_params),
                                    _ptr(loss_out), _ptr(err_out), ctypes.c_void_p(stream))
    if rc:
        raise FpmError(rc, lib().fpm_last_error(None).decode())


class Engine:
    """One reconstruction job (object, pupil, defocus, LED parameters, Adam state) on the GPU."""

    def __init__(self, m: int, upsample: int, led_offset, pupil_radius: float, lambda_um: float,
                 dk_per_um: float, edge: str = "aa", stream=None):
        L = lib()
        self._off = np.ascontiguousarray(np.asarray(led_offset, np.float32).reshape(-1, 2))
        g = Geometry(m, self._off.shape[0], self._off.ctypes.data, lambda_um, dk_per_um, EDGE[edge])
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        h = ctypes.c_void_p()
        rc = L.fpm_create(ctypes.byref(g), pupil_radius, upsample, ctypes.c_void_p(stream), ctypes.byref(h))
        if rc:
            raise FpmError(rc, L.fpm_last_error(None).decode())
        self._h = h
        self.m, self.s, self.N, self.n_leds = m, upsample, m * upsample, self._off.shape[0]
        dims = [ctypes.c_int32() for _ in range(4)]
        L.fpm_dims(h, *(ctypes.byref(d) for d in dims))
        self.box = dims[3].value

    # -- plumbing --------------------------------------------------------
    def _check(self, rc):
        if rc:
            raise FpmError(rc, lib().fpm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().fpm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- API ---------------------------------------------------------------
    def set_hparams(self, lr=None, betas=(0.9, 0.999), eps=1e-8, loss="amplitude", learn=("object",),
                    precision="fp32_fft", optimizer="adam", weight_decay=0.0):
        rates = dict(object=0.1, zernike=0.01, defocus=0.1, gamma=0.01, offset=0.01, pupil=0.01)
        rates.update(lr or {})
        lr = rates
        mask = 0
        for k in learn:
            mask |= LEARN[k]
        hp = Hparams(lr["object"], lr["zernike"], lr["defocus"], lr["gamma"], lr["offset"],
                     betas[0], betas[1], eps, LOSS[loss], mask, PRECISION[precision], OPTIMIZER[optimizer],
                     weight_decay, lr["pupil"])
        self._check(lib().fpm_set_hparams(self._h, ctypes.byref(hp)))

    def set_memory_limit(self, nbytes: int):
        """Limit on the handle's device memory (bytes; <= 0: none)."""
        self._check(lib().fpm_set_memory_limit(self._h, int(nbytes)))

    def memory_used(self) -> int:
        return int(lib().fpm_memory_used(self._h))

    def set_step_form(self, form: str = "auto"):
        """Kernels of a step: 'auto' / 'cluster' (per-LED clusters) or 'dataflow' (m = 256)."""
        self._check(lib().fpm_set_step_form(self._h, STEP_FORM[form]))

    def step_form(self):
        """(form asked for, whether the dataflow form is in use)."""
        f, d = ctypes.c_int32(), ctypes.c_int32()
        self._check(lib().fpm_get_step_form(self._h, ctypes.byref(f), ctypes.byref(d)))
        return {v: k for k, v in STEP_FORM.items()}[f.value], bool(d.value)

    def check_wait_timeout(self, idx, limit_s: float):
        """fpm_check_wait_timeout: one step whose waits cannot be satisfied, bounded by
        limit_s. Returns (code, message); FPM_ERR_TIMEOUT (-6) is the expected code."""
        b = np.ascontiguousarray(np.asarray(idx, np.int32))
        rc = lib().fpm_check_wait_timeout(self._h, b.ctypes.data, b.size, float(limit_s))
        return rc, lib().fpm_last_error(self._h).decode()

    def load(self, stack, init: bool = True):
        stack = _f32(stack)
        self._check(lib().fpm_load(self._h, _ptr(stack), LOAD_INIT if init else 0))

    def step(self, batch, loss: bool = True) -> float | None:
        b = np.ascontiguousarray(np.asarray(batch, np.int32))
        out = ctypes.c_double() if loss else None
        self._check(lib().fpm_step(self._h, b.ctypes.data, b.size, ctypes.byref(out) if loss else None))
        return out.value if loss else None

    def run(self, schedule, losses=True):
        """schedule: [n_steps, B] int32 (host). losses: True -> numpy array,
        a CUDA tensor [n_steps] float64 -> filled asynchronously, False -> none."""
        s = np.ascontiguousarray(np.asarray(schedule, np.int32))
        assert s.ndim == 2
        if losses is True:
            out = np.empty(s.shape[0], np.float64)
            self._check(lib().fpm_run(self._h, s.ctypes.data, s.shape[0], s.shape[1], out.ctypes.data))
            return out
        dst = _ptr(losses) if losses is not False and losses is not None else None
        self._check(lib().fpm_run(self._h, s.ctypes.data, s.shape[0], s.shape[1], dst))
        return losses if dst else None

    def profile_run(self, schedule, flush=None, per_kernel=True):
        """Timed steps (see fpm_profile_run). flush: a CUDA tensor cleared before every
        step, or None. per_kernel=True returns per-step ms of (per-LED kernel, update
        kernel, step), the kernels run back to back; per_kernel=False times only the
        step, with the update kernel launched early as inside run(), and returns
        (None, None, step)."""
        s = np.ascontiguousarray(np.asarray(schedule, np.int32))
        n = s.shape[0]
        led, upd, stp = (np.empty(n, np.float32) for _ in range(3))
        fb = flush.numel() * flush.element_size() if flush is not None else 0
        self._check(lib().fpm_profile_run(self._h, s.ctypes.data, n, s.shape[1], _ptr(flush), fb,
                                          led.ctypes.data if per_kernel else None,
                                          upd.ctypes.data if per_kernel else None, stp.ctypes.data))
        return (led, upd, stp) if per_kernel else (None, None, stp)

    def epoch_loss(self, reset=False) -> float:
        out = ctypes.c_double()
        self._check(lib().fpm_epoch_loss(self._h, ctypes.byref(out), int(reset)))
        return out.value

    def forward(self, idx, out=None):
        b = np.ascontiguousarray(np.asarray(idx, np.int32))
        if out is None:
            out = np.empty((b.size, self.m, self.m), np.float32)
        self._check(lib().fpm_forward(self._h, b.ctypes.data, b.size, _ptr(out)))
        return out

    def backward(self, idx, dL_dI=None, want_object=True):
        b = np.ascontiguousarray(np.asarray(idx, np.int32))
        gO = np.empty((self.N, self.N, 2), np.float32) if want_object else None
        gz = np.empty(14, np.float32)
        gd = np.empty(1, np.float32)
        gg = np.empty(self.n_leds, np.float32)
        go = np.empty((self.n_leds, 2), np.float32)
        loss = ctypes.c_double()
        up = _f32(dL_dI) if dL_dI is not None and isinstance(dL_dI, np.ndarray) else dL_dI
        self._check(lib().fpm_backward(self._h, b.ctypes.data, b.size, _ptr(up), _ptr(gO), _ptr(gz),
                                       _ptr(gd), _ptr(gg), _ptr(go), ctypes.byref(loss)))
        return dict(object=None if gO is None else gO[..., 0] + 1j * gO[..., 1].astype(np.float64),
                    zernike=gz, defocus=float(gd[0]), gamma=gg, offset=go, loss=loss.value)

    def get(self, object=True, out=None):
        """The current state. out (optional): caller-owned host buffers to copy into
        (e.g. pinned tensors reused across calls), a dict with float32 'object'
        [N, N, 2], 'zernike' [14], 'defocus' [1], 'gamma' [n_leds], 'offset'
        [n_leds, 2]; they are returned as they are (no complex conversion)."""
        if out is not None:
            self._check(lib().fpm_get(self._h, _ptr(out["object"]) if object else None, _ptr(out["zernike"]),
                                      _ptr(out["defocus"]), _ptr(out["gamma"]), _ptr(out["offset"])))
            return out
        O = np.empty((self.N, self.N, 2), np.float32) if object else None
        z = np.empty(14, np.float32)
        d = np.empty(1, np.float32)
        g = np.empty(self.n_leds, np.float32)
        o = np.empty((self.n_leds, 2), np.float32)
        self._check(lib().fpm_get(self._h, _ptr(O), _ptr(z), _ptr(d), _ptr(g), _ptr(o)))
        return dict(object=None if O is None else O[..., 0] + 1j * O[..., 1].astype(np.float64),
                    zernike=z, defocus=float(d[0]), gamma=g, offset=o)

    def get_object_into(self, tensor):
        """Copy O into a CUDA tensor [N, N, 2] float32 without a host round trip."""
        self._check(lib().fpm_get(self._h, _ptr(tensor), None, None, None, None))

    def set(self, object=None, zernike=None, defocus=None, gamma=None, offset=None):
        O = None
        if object is not None:
            O = _f32(np.stack([np.real(object), np.imag(object)], -1)) if np.iscomplexobj(object) else _f32(object)
        z = None if zernike is None else _f32(zernike)
        d = None if defocus is None else _f32(np.array([defocus]))
        g = None if gamma is None else _f32(gamma)
        o = None if offset is None else _f32(offset)
        self._check(lib().fpm_set(self._h, _ptr(O), _ptr(z), _ptr(d), _ptr(g), _ptr(o)))

    def set_pupil(self, P):
        """Free-form pupil field ([W, W] complex, node (ny, nx) at [ny + h, nx + h]); None removes it."""
        if P is None:
            self._check(lib().fpm_set_pupil(self._h, None))
            return
        arr = _f32(np.stack([np.real(P), np.imag(P)], -1)) if np.iscomplexobj(P) else _f32(P)
        self._check(lib().fpm_set_pupil(self._h, _ptr(arr)))

    def get_pupil(self):
        """(field [W, W] complex, whether it is in the model)."""
        out = np.empty((self.box, self.box, 2), np.float32)
        on = ctypes.c_int32()
        self._check(lib().fpm_get_pupil(self._h, out.ctypes.data, ctypes.byref(on)))
        return out[..., 0] + 1j * out[..., 1].astype(np.float64), bool(on.value)

    def pupil_gradient(self):
        """Gradient of the field from the last backward ([W, W] complex)."""
        out = np.empty((self.box, self.box, 2), np.float32)
        self._check(lib().fpm_pupil_gradient(self._h, out.ctypes.data))
        return out[..., 0] + 1j * out[..., 1].astype(np.float64)

    def set_object_field(self, o):
        arr = _f32(np.stack([np.real(o), np.imag(o)], -1))
        self._check(lib().fpm_set_object_field(self._h, _ptr(arr)))

    def state_size(self) -> int:
        return int(lib().fpm_state_size(self._h))

    def get_state(self) -> np.ndarray:
        st = np.empty(self.state_size(), np.float32)
        self._check(lib().fpm_get_state(self._h, st.ctypes.data))
        return st

    def set_state(self, st):
        st = _f32(st)
        self._check(lib().fpm_set_state(self._h, st.ctypes.data))


def _f32(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.contiguous()
    return np.ascontiguousarray(np.asarray(x, np.float32))
