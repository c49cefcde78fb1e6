"""Seeded recipes for the synthetic Batch-FPM workloads.

The paper's own simulation (Section 3.1) uses ground-truth images that are not
available, so every workload here is synthetic with the paper's shapes: a
1024x1024 high-resolution object imaged through a 4x-upsampled 256x256
low-resolution camera by a square LED grid, Gaussian-filtered random
amplitude/phase fields standing in for the sample, and Poisson plus read noise
standing in for the camera (Sections 3.1-3.2 describe low-exposure dark-field
images as the noisy ones).

Nothing here evaluates the imaging model: noisy stacks are made by passing the
clean intensities (computed by the caller with whichever implementation it is
testing) through :func:`add_noise`.

LED indexing follows the paper's illumination sequence (Section 3.2): index 0
is the centre LED, then the 3x3 ring, the 5x5 ring and so on (Chebyshev rings,
counter-clockwise by angle within a ring), so the identity order is the
classic centre-to-periphery sequential order of Eq. (7).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

_M64 = (1 << 64) - 1


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Config:
    name: str
    N: int                      # high-res side
    m: int                      # low-res side
    grid: int                   # LEDs per side of the square grid
    pitch: float                # spectral px between neighbouring LEDs
    R: float                    # pupil radius, spectral px
    edge: str = "aa"            # 'aa' (anti-aliased ramp) or 'hard'
    jitter: float = 0.0         # ground-truth sub-pixel LED jitter, U(-j, j)
    z_um: float = 0.0           # ground-truth defocus
    lambda_um: float = 0.532
    dx_lr_um: float = 0.6       # low-res pixel at the sample plane
    zernike_sigma: float = 0.0  # ground-truth Noll 2..15 coefficient std, rad
    gamma_range: tuple = (1.0, 1.0)
    noise: dict | None = None   # {'bf_mean', 'df_mean', 'read_sigma'}
    B: int = 8
    epochs: int = 30
    lr: dict = field(default_factory=lambda: dict(
        object=0.1, zernike=0.01, defocus=0.1, gamma=0.01, offset=0.01))
    learn: tuple = ("object",)
    seed: int = 2408

    @property
    def s(self) -> int:
        return self.N // self.m

    @property
    def n_leds(self) -> int:
        return self.grid * self.grid

    @property
    def dk_per_um(self) -> float:
        """Spectral bin of both grids, 1/um (low-res field is m * dx_lr wide)."""
        return 1.0 / (self.m * self.dx_lr_um)

    def with_(self, **kw) -> "Config":
        return replace(self, **kw)


_ALL = ("object", "zernike", "defocus", "gamma", "offset")


def _c1() -> Config:
    # 256^2 object, 7x7 LEDs spaced 8 px, 64^2 images, hard circular pupil
    # r=14, z=0, unit intensities, noise-free; batch 8, Adam lr 0.1, 30 epochs.
    return Config("c1_plain_256", N=256, m=64, grid=7, pitch=8, R=14,
                  edge="hard", B=8, epochs=30, seed=11)


def _c2() -> Config:
    # Paper-scale ROI (Section 3.1 shapes: 1024^2 object, 256^2 images),
    # 15x15 LEDs spaced 12 px with +-0.5 px jitter, pupil r=50 with Noll
    # 2..15 aberrations ~N(0, 0.3 rad), z=+15 um at 532 nm, intensities
    # U(0.8, 1.2), Poisson (bright 2000 / dark 20 photons) + read sigma 2.
    return Config("c2_multiparam_1024", N=1024, m=256, grid=15, pitch=12,
                  R=50, edge="aa", jitter=0.5, z_um=15.0, zernike_sigma=0.3,
                  gamma_range=(0.8, 1.2),
                  noise=dict(bf_mean=2000.0, df_mean=20.0, read_sigma=2.0),
                  B=16, epochs=20,
                  lr=dict(object=1.0, zernike=0.01, defocus=0.1, gamma=0.01,
                          offset=0.01),
                  learn=_ALL, seed=22)


def _c3() -> Config:
    # Differentiation check: 512^2 / 128^2, 9x9 LEDs, batch 4; the pupil
    # radius and pitch scale with m from the 64-px case (r = 14 m/64,
    # pitch = 8 m/64). Aberrations, defocus, intensities and jitter are on so
    # that every gradient is exercised at a generic point.
    return Config("c3_grad_512", N=512, m=128, grid=9, pitch=16, R=28,
                  edge="aa", jitter=0.5, z_um=5.0, zernike_sigma=0.3,
                  gamma_range=(0.8, 1.2), B=4, epochs=1, learn=_ALL, seed=33)


def _c3_mem() -> Config:
    # Memory run: 2048^2 / 512^2, 15x15 LEDs, batch 64.
    return Config("c3_mem_2048", N=2048, m=512, grid=15, pitch=64, R=112,
                  edge="aa", jitter=0.5, z_um=5.0, zernike_sigma=0.3,
                  gamma_range=(0.8, 1.2), B=64, epochs=1, learn=_ALL, seed=34)


def _c4_x4() -> Config:
    # The 64-px recipe scaled x4 (1024^2 / 256^2, 7x7, pitch 32, r=56) so the
    # low-res DFTs are 256-point; noise-free; 20 epochs.
    return Config("c4_plain_x4_1024", N=1024, m=256, grid=7, pitch=32, R=56,
                  edge="hard", B=16, epochs=20, seed=44)


CONFIG_NAMES = ("c1", "c2", "c3", "c3_mem", "c4_x4")


def config(name: str) -> Config:
    return {"c1": _c1, "c2": _c2, "c3": _c3, "c3_mem": _c3_mem,
            "c4_x4": _c4_x4}[name]()


RGB_WAVELENGTHS_UM = (0.470, 0.523, 0.623)   # the three LED colours of Section 3.3


def rgb_job_configs(N: int, grid: int, seed: int, wavelengths=RGB_WAVELENGTHS_UM) -> list:
    """The three colour channels of one field of view (Section 3.3) as serving jobs:
    the 64-px recipe scaled to high-res side N at 0.532 um, then, per wavelength,
    the pupil radius and the LED pitch in spectral px scaled by 0.532 / lambda (a
    fixed numerical aperture and LED geometry on a fixed spectral grid). Same
    stack shape for every channel; the same sample (object seed)."""
    base = serving_job_config(N, grid, seed)
    return [base.with_(name=f"{base.name}_{int(round(lam * 1000))}nm", lambda_um=lam,
                       R=base.R * 0.532 / lam, pitch=base.pitch * 0.532 / lam)
            for lam in wavelengths]


def serving_job_config(N: int, grid: int, seed: int) -> Config:
    """One serving request: the 64-px recipe scaled to high-res side N."""
    m = N // 4
    return Config(f"serve_{N}_{grid}x{grid}", N=N, m=m, grid=grid,
                  pitch=8 * m / 64, R=14 * m / 64, edge="hard", B=8,
                  epochs=40, seed=seed)


# --------------------------------------------------------------------------
# ground truth
# --------------------------------------------------------------------------

def smooth_field(N: int, sigma_px: float, rng: np.random.Generator) -> np.ndarray:
    """iid N(0,1) noise, periodically Gaussian-filtered (sigma in px), scaled to [0, 1]."""
    w = rng.standard_normal((N, N))
    f = np.fft.fftfreq(N)
    f2 = f[:, None] ** 2 + f[None, :] ** 2
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * np.exp(-2.0 * math.pi ** 2 * sigma_px ** 2 * f2)))
    g -= g.min()
    return g / g.max()


def make_object(N: int, seed: int, sigma_px: float = 4.0) -> np.ndarray:
    """Complex transmission: amplitude in [0.5, 1], phase in [-pi/2, pi/2]."""
    rng = np.random.default_rng([seed, 1])
    amp = 0.5 + 0.5 * smooth_field(N, sigma_px, rng)
    ph = -0.5 * math.pi + math.pi * smooth_field(N, sigma_px, rng)
    return amp * np.exp(1j * ph)


def led_grid(grid: int, pitch: float, jitter: float, seed: int):
    """Nominal and ground-truth spectral LED centres, px (row, col) from DC.

    Returns (nominal [n,2], truth [n,2]); truth = nominal + U(-jitter, jitter).
    Ordered centre first, then square rings outward (the paper's LED
    numbering), counter-clockwise by angle within a ring.
    """
    h = (grid - 1) // 2
    cells = []
    for iy in range(-h, h + 1):
        for ix in range(-h, h + 1):
            ring = max(abs(iy), abs(ix))
            ang = math.atan2(iy, ix) % (2 * math.pi)
            cells.append((ring, ang, iy, ix))
    cells.sort()
    nominal = np.array([[c[2] * pitch, c[3] * pitch] for c in cells], dtype=np.float64)
    rng = np.random.default_rng([seed, 2])
    truth = nominal + rng.uniform(-jitter, jitter, size=nominal.shape) if jitter > 0 else nominal.copy()
    return nominal, truth


def zernike_coeffs(sigma: float, seed: int) -> np.ndarray:
    """Noll j = 2..15 coefficients (14 values, rad), ~N(0, sigma)."""
    if sigma <= 0:
        return np.zeros(14)
    return np.random.default_rng([seed, 3]).normal(0.0, sigma, size=14)


def led_gamma(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    if lo == hi:
        return np.full(n, float(lo))
    return np.random.default_rng([seed, 4]).uniform(lo, hi, size=n)


def brightfield_mask(nominal: np.ndarray, R: float) -> np.ndarray:
    """Exposure class used by the noise model: bright field iff |offset| <= R."""
    return np.hypot(nominal[:, 0], nominal[:, 1]) <= R


def add_noise(I_clean: np.ndarray, bright: np.ndarray, bf_mean: float,
              df_mean: float, read_sigma: float, seed: int) -> np.ndarray:
    """Camera model for a stack [n, m, m] of clean intensities.

    Each exposure class is scaled so its mean photon count is bf_mean (bright
    field) or df_mean (dark field), Poisson-sampled, read noise N(0, sigma^2)
    added, and the result divided back by the class scale so the stack stays
    in the clean stack's units.
    """
    rng = np.random.default_rng([seed, 5])
    out = np.empty_like(I_clean, dtype=np.float64)
    for cls, mean in ((True, bf_mean), (False, df_mean)):
        sel = np.nonzero(bright == cls)[0]
        if sel.size == 0:
            continue
        mu = float(np.mean(I_clean[sel]))
        scale = mean / mu if mu > 0 else 1.0
        lam = np.clip(I_clean[sel] * scale, 0.0, None)
        photons = rng.poisson(lam).astype(np.float64)
        photons += rng.normal(0.0, read_sigma, size=photons.shape)
        out[sel] = photons / scale
    return out


# --------------------------------------------------------------------------
# random batch order (Eq. 13-14): the draw is an input to both implementations
# --------------------------------------------------------------------------

def splitmix64(state: int):
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): yields 64-bit outputs."""
    s = state & _M64
    while True:
        s = (s + 0x9E3779B97F4A7C15) & _M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        yield z ^ (z >> 31)


def epoch_permutation(n: int, seed: int, epoch: int) -> np.ndarray:
    """Permutation of range(n) for one epoch.

    SplitMix64 seeded with seed XOR ((epoch + 1) * 0xA0761D6478BD642F mod 2^64)
    drives a Durstenfeld Fisher-Yates shuffle of the identity: for i = n-1
    down to 1, j = next() mod (i + 1), swap a[i], a[j].
    """
    state = (seed ^ (((epoch + 1) * 0xA0761D6478BD642F) & _M64)) & _M64
    g = splitmix64(state)
    a = list(range(n))
    for i in range(n - 1, 0, -1):
        j = next(g) % (i + 1)
        a[i], a[j] = a[j], a[i]
    return np.array(a, dtype=np.int32)


def chop(order, B: int) -> list:
    """Consecutive batches of size B; the last one is short if B does not divide."""
    order = list(order)
    return [np.array(order[k:k + B], dtype=np.int32) for k in range(0, len(order), B)]


def schedule(n: int, B: int, epochs: int, seed: int, shuffle: bool = True) -> list:
    """Batches for `epochs` passes; each LED appears exactly once per pass.

    shuffle=False gives the fixed sequential order of Eq. (7) (B=1) or the
    paper's non-random batching example (Section 2.3).
    """
    out = []
    for e in range(epochs):
        order = epoch_permutation(n, seed, e) if shuffle else np.arange(n, dtype=np.int32)
        out.extend(chop(order, B))
    return out
