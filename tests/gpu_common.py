"""Shared setup for the GPU parity tests: the same problem on the engine and the oracle."""

from __future__ import annotations

import json
import os

import numpy as np

import oracle as orc
from paper_2408_13782_gb300 import Engine
from synth import recipes as S
from tests.helpers import generic_params, rel_l2, simulate

REPORT = {}


def record(name, value):
    """Keep an error figure for the parity report (written if FPM_PARITY_REPORT is set)."""
    REPORT[name] = float(value)
    path = os.environ.get("FPM_PARITY_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(REPORT, fh, indent=1, sort_keys=True)


def engine_for(geom: orc.Geometry) -> Engine:
    return Engine(geom.m, geom.s, geom.nominal, geom.R, geom.lambda_um, geom.dk_per_um, geom.edge)


def push(eng: Engine, O, prm: orc.Params):
    eng.set(object=O, zernike=prm.zernike, defocus=prm.defocus, gamma=prm.gamma, offset=prm.offset)


def hparams_to_engine(eng: Engine, hp: orc.Hparams):
    eng.set_hparams(lr=dict(hp.lr), betas=(hp.beta1, hp.beta2), eps=hp.eps, loss=hp.loss, learn=hp.learn,
                    optimizer=hp.optimizer, weight_decay=hp.weight_decay)


def multiparam_problem(m=64, s=4, grid=5, pitch=None, R=None, edge="aa", seed=5, z=3.0):
    """A generic multi-parameter problem (aberrations, defocus, gamma, offsets)."""
    R = R if R is not None else 14.0 * m / 64
    pitch = pitch if pitch is not None else 8.0 * m / 64
    c = S.Config(f"mp{m}", N=m * s, m=m, grid=grid, pitch=pitch, R=R, edge=edge, jitter=0.4, z_um=z,
                 zernike_sigma=0.3, gamma_range=(0.8, 1.2),
                 noise=dict(bf_mean=2000.0, df_mean=20.0, read_sigma=2.0), B=4, epochs=2,
                 learn=("object", "zernike", "defocus", "gamma", "offset"), seed=seed)
    I, o, g_n, g_t, prm_t = simulate(c)
    # evaluate away from the truth so every gradient is non-trivial
    rng = np.random.default_rng(seed + 100)
    prm = prm_t.copy()
    prm.zernike = prm.zernike + rng.normal(0, 0.1, 14)
    prm.defocus += 0.7
    prm.gamma = prm.gamma * rng.uniform(0.9, 1.1, prm.gamma.shape)
    prm.offset = np.clip(prm.offset + rng.uniform(-0.2, 0.2, prm.offset.shape), -0.9, 0.9)
    O = orc.object_spectrum(o, c.s) * (1 + 0.1 * rng.normal(size=(c.N, c.N)))
    return c, I, g_t, prm, O


__all__ = ["REPORT", "record", "engine_for", "push", "hparams_to_engine", "multiparam_problem",
           "generic_params", "rel_l2", "simulate"]
