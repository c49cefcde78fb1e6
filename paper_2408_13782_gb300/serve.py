"""Binding of the engine's continuous-batching server (fpm_server_* in include/fpm.h).

Argument marshalling plus a small driver that submits jobs at their arrival
times and calls fpm_server_tick until every job is finished; all scheduling,
admission and GPU work happen in the library.
"""

from __future__ import annotations

import ctypes
import time

import numpy as np

from .engine import EDGE, LEARN, LOSS, OPTIMIZER, PRECISION, FpmError, Geometry, Hparams, lib

JOB_QUEUED, JOB_ACTIVE, JOB_DONE, JOB_FAILED = 0, 1, 2, 3


class JobDesc(ctypes.Structure):
    _fields_ = [("geometry", Geometry), ("pupil_radius_px", ctypes.c_float), ("upsample", ctypes.c_int32),
                ("hparams", Hparams), ("batch", ctypes.c_int32), ("max_epochs", ctypes.c_int32),
                ("rel_tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


class JobStatus(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("epochs", ctypes.c_int32), ("loss", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("led_updates", ctypes.c_int64), ("footprint", ctypes.c_int64)]


def _declare(L):
    if getattr(L, "_fpm_server_declared", False):
        return
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "fpm_job_footprint": ([ctypes.POINTER(JobDesc)], i64),
        "fpm_server_create": ([i64, i32, ctypes.POINTER(vp)], i32),
        "fpm_server_submit": ([vp, ctypes.POINTER(JobDesc), vp, ctypes.POINTER(i64)], i32),
        "fpm_server_tick": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "fpm_server_status": ([vp, i64, ctypes.POINTER(JobStatus)], i32),
        "fpm_server_result": ([vp, i64, vp, vp, vp, vp, vp], i32),
        "fpm_server_clock": ([vp], ctypes.c_double),
        "fpm_server_stats": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
                             i32),
        "fpm_server_error": ([vp], ctypes.c_char_p),
        "fpm_server_set_admission": ([vp, i32], i32),
        "fpm_server_set_grouping": ([vp, i32], i32),
        "fpm_server_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    L._fpm_server_declared = True


def job_desc(m, upsample, led_offset, pupil_radius, lambda_um, dk_per_um, edge="aa", batch=8, max_epochs=40,
             rel_tol=1e-4, seed=0, lr=None, learn=("object",), loss="amplitude", precision="fp32_fft",
             optimizer="adam", weight_decay=0.0):
    """A job description; keep the returned tuple alive until it has been submitted."""
    off = np.ascontiguousarray(np.asarray(led_offset, np.float32).reshape(-1, 2))
    rates = dict(object=0.1, zernike=0.01, defocus=0.1, gamma=0.01, offset=0.01, pupil=0.01)
    rates.update(lr or {})
    mask = 0
    for k in learn:
        mask |= LEARN[k]
    hp = Hparams(rates["object"], rates["zernike"], rates["defocus"], rates["gamma"], rates["offset"],
                 0.9, 0.999, 1e-8, LOSS[loss], mask, PRECISION[precision], OPTIMIZER[optimizer], weight_decay,
                 rates["pupil"])
    g = Geometry(m, off.shape[0], off.ctypes.data, lambda_um, dk_per_um, EDGE[edge])
    return JobDesc(g, pupil_radius, upsample, hp, batch, max_epochs, rel_tol, seed & ((1 << 64) - 1)), off


def footprint(desc) -> int:
    L = lib()
    _declare(L)
    return int(L.fpm_job_footprint(ctypes.byref(desc[0])))


ADMISSION = {"arrival": 0, "smallest": 1}
GROUPING = {"config": 0, "size": 1, "mixed": 2}


class Server:
    def __init__(self, hbm_budget_bytes: int, max_active: int = 64, admission: str = "arrival",
                 grouping: str = "config"):
        L = lib()
        _declare(L)
        h = ctypes.c_void_p()
        rc = L.fpm_server_create(int(hbm_budget_bytes), int(max_active), ctypes.byref(h))
        if rc:
            raise FpmError(rc, "server creation failed")
        self._h = h
        self._check(L.fpm_server_set_admission(h, ADMISSION[admission]))
        self.set_grouping(grouping)

    def set_grouping(self, grouping: str):
        """Which resident jobs share a round: "config", "size" or "mixed" (fpm.h)."""
        self._check(lib().fpm_server_set_grouping(self._h, GROUPING[grouping]))

    def _check(self, rc):
        if rc:
            raise FpmError(rc, lib().fpm_server_error(self._h).decode())

    def submit(self, desc, stack) -> int:
        st = np.ascontiguousarray(np.asarray(stack, np.float32))
        jid = ctypes.c_int64()
        self._check(lib().fpm_server_submit(self._h, ctypes.byref(desc[0]), st.ctypes.data, ctypes.byref(jid)))
        return jid.value

    def tick(self):
        a, q = ctypes.c_int32(), ctypes.c_int32()
        self._check(lib().fpm_server_tick(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def status(self, jid) -> dict:
        s = JobStatus()
        self._check(lib().fpm_server_status(self._h, jid, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in JobStatus._fields_}

    def result(self, jid, N, n_leds) -> dict:
        O = np.empty((N, N, 2), np.float32)
        z = np.empty(14, np.float32)
        d = np.empty(1, np.float32)
        g = np.empty(n_leds, np.float32)
        o = np.empty((n_leds, 2), np.float32)
        self._check(lib().fpm_server_result(self._h, jid, O.ctypes.data, z.ctypes.data, d.ctypes.data,
                                            g.ctypes.data, o.ctypes.data))
        return dict(object=O[..., 0] + 1j * O[..., 1].astype(np.float64), zernike=z, defocus=float(d[0]),
                    gamma=g, offset=o)

    def clock(self) -> float:
        return lib().fpm_server_clock(self._h)

    def stats(self) -> dict:
        """Rounds launched, job epochs they ran, most jobs in one round, kernel launches."""
        v = [ctypes.c_int64() for _ in range(4)]
        self._check(lib().fpm_server_stats(self._h, *[ctypes.byref(x) for x in v]))
        return dict(rounds=v[0].value, round_epochs=v[1].value, max_jobs_per_round=v[2].value,
                    launches=v[3].value)

    def close(self):
        if getattr(self, "_h", None):
            lib().fpm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_arrivals(server: Server, jobs, poll_s: float = 0.0002):
    """Submit jobs [(desc, stack, arrival_s)] at their arrival times (server clock)
    and tick until all have finished. Returns (ids, statuses, wall seconds)."""
    order = sorted(range(len(jobs)), key=lambda i: jobs[i][2])
    ids = [None] * len(jobs)
    k = 0
    t_start = server.clock()
    while True:
        t = server.clock() - t_start
        while k < len(order) and jobs[order[k]][2] <= t:
            i = order[k]
            ids[i] = server.submit(jobs[i][0], jobs[i][1])
            k += 1
        active, queued = server.tick()
        if k == len(order) and active == 0 and queued == 0:
            break
        if active == 0 and queued == 0 and k < len(order):
            time.sleep(max(0.0, min(poll_s, jobs[order[k]][2] - t)))
    statuses = [server.status(j) for j in ids]
    return ids, statuses, server.clock() - t_start
