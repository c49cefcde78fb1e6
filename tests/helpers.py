"""Problem builders shared by the tests (inputs from `synth`, truth from `oracle`)."""

from __future__ import annotations

import numpy as np

import oracle as orc
from synth import recipes as S


def tiny_geometry(N=32, m=16, grid=3, pitch=3.0, R=5.0, edge="aa", seed=7,
                  jitter=0.4, lambda_um=0.532, dx_lr_um=0.6):
    nominal, truth = S.led_grid(grid, pitch, jitter, seed)
    g = orc.Geometry(N, m, truth, R, edge, lambda_um, 1.0 / (m * dx_lr_um))
    return g, nominal, truth


def generic_params(geom: orc.Geometry, seed=3, zsig=0.3, z=2.0, off=0.4):
    rng = np.random.default_rng(seed)
    return orc.Params(
        zernike=rng.normal(0, zsig, 14),
        defocus=float(z),
        gamma=rng.uniform(0.8, 1.2, geom.n_leds),
        offset=rng.uniform(-off, off, (geom.n_leds, 2)),
    )


def geometry_from_config(c, positions="truth"):
    nominal, truth = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
    pos = truth if positions == "truth" else nominal
    return orc.Geometry(c.N, c.m, pos, c.R, c.edge, c.lambda_um, c.dk_per_um), nominal, truth


def truth_params(c, geom_truth: orc.Geometry, truth):
    """Ground-truth parameters in the truth geometry (offsets = sub-pixel part)."""
    return orc.Params(
        zernike=S.zernike_coeffs(c.zernike_sigma, c.seed),
        defocus=float(c.z_um),
        gamma=S.led_gamma(c.n_leds, *c.gamma_range, c.seed),
        offset=truth - geom_truth.n_int,
    )


def simulate(c, dtype=np.float32):
    """Measured stack for config c, computed with the oracle at the truth.

    Returns (stack [n, m, m], o_truth, geometry with nominal positions,
    ground-truth geometry, truth params).
    """
    g_t, nominal, truth = geometry_from_config(c, "truth")
    prm_t = truth_params(c, g_t, truth)
    o = S.make_object(c.N, c.seed)
    O_t = orc.object_spectrum(o, c.s)
    I = orc.forward(O_t, prm_t, g_t, range(g_t.n_leds))
    if c.noise:
        bright = S.brightfield_mask(nominal, c.R)
        I = S.add_noise(I, bright, c.noise["bf_mean"], c.noise["df_mean"],
                        c.noise["read_sigma"], c.seed)
    g_n = orc.Geometry(c.N, c.m, nominal, c.R, c.edge, c.lambda_um, c.dk_per_um)
    return I.astype(dtype), o, g_n, g_t, prm_t


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))
