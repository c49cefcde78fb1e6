"""Plain FP64 restatement of Batch-FPM (arXiv 2408.13782), step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring): used by tests, the
package smoke check and the benchmark's CPU baseline; never by the engine.

What it computes, with the passage each part follows:

* thin object o(r) = exp(i phi - mu) and its centred spectrum
  O = fftshift(fft2(o)) / s^2 .................... Section 2.1, Eq. (1)
* per-LED low-res field and intensity
  I_i = gamma_i |F^-1( O(k - k_mi) P(k) H(k, z) )|^2 ... Section 2.1, Eq. (2)-(3)
* loss summed over the images of a batch ............ Section 2.2, Eq. (4)-(5)
* its gradient (the paper differentiates automatically; here the adjoint is
  written out with the convention grad_w = dL/dRe w + i dL/dIm w)
* the random batch update with Adam ................. Section 2.3, Eq. (13)
* each image used once per pass (batch order given as input) .. Eq. (14)
* initial object: bilinear-interpolated centre-LED image ...... Section 2.3

Readings where the paper is silent or garbled:

* defocus kernel: the paper's sqrt(1 - kx^2 - ky^2) mixes units; it is read
  as kappa(k) = 2 pi (sqrt(lambda^-2 - |k|^2) - lambda^-1), the angular
  spectrum phase per unit z minus its (intensity-invariant) piston;
* pupil: circle of radius R (spectral px) times exp(i sum_j c_j Z_j(q/R)),
  Noll j = 2..15, orthonormal on the unit disk; edge either hard
  (A = [|q| <= R]) or anti-aliased (A = clamp(R + 1/2 - |q|, 0, 1));
* LED geometry: crop at the integer part n_i of the spectral offset, pupil,
  aberration and defocus evaluated at q = p - delta_i (sub-pixel part);
* loss: amplitude form sum (sqrt(gamma)|psi| - sqrt(max(I_meas, 0)))^2 by
  default, the intensity form of Eq. (4) as an option; plain sums; a
  'linear' form sum w I_pred (w given in place of I_meas) states the
  gradient for an arbitrary upstream dL/dI;
* psi / |psi| := 0 where psi = 0;
* initial object: sqrt(max(I_centre, 0)) upsampled bilinearly with low-res
  pixel r on high-res pixel s*r and a periodic boundary, zero phase;
  gamma = 1, aberrations = 0, z = 0, delta = fractional part of the nominal
  LED offsets;
* free-form pupil (the pupil-recovery reference of Section 2.2): an optional
  complex field P on the integer nodes of the crop grid (index p + m/2),
  multiplying the parametric pupil; it is evaluated at q = p - delta_i by
  bilinear interpolation between the four nodes around q, so that
  M_i(p) = A(q) exp(i chi(q)) P~(q); P = 1 (or None) is the parametric model;
* Adam (Kingma & Ba 2015, bias-corrected; or AdamW, NAdam, RMSprop, the other
  members of the Adam family) on every real component of every
  learnable tensor, every step; sub-pixel offsets clamped to +-offset_bound
  and intensity factors held at or above gamma_floor (1e-3; the amplitude loss
  takes sqrt(gamma), which long runs of Adam steps on noisy dark-field images
  can otherwise drive below zero) after each update.

Parity pins (tests/test_oracle_*.py): brute-force DFT, Parseval, closed forms
(constant object, cosine grating, global phase), central finite differences
on every gradient, zero loss/gradient at the truth, the gamma optimum,
torch.optim.Adam, AdamW, NAdam and RMSprop and their first-step closed forms, Noll's table, scipy's
periodic linear interpolation. Reconstruction quality against the paper's Fig. 4 is
"parity unpinned": the figure's values are not in the text.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Zernike polynomials, Noll ordering (Noll 1976), as 2-D Cartesian polynomials
# --------------------------------------------------------------------------


def noll_nm(j: int):
    """Noll index j >= 1 -> (n, m); m < 0 is the sine term, m > 0 the cosine."""
    n = int((math.isqrt(8 * (j - 1) + 1) - 1) // 2)
    p = j - n * (n + 1) // 2          # 1-based position within radial order n
    k = n % 2
    am = 2 * ((p + k) // 2) - k
    if am == 0:
        return n, 0
    return n, (am if j % 2 == 0 else -am)


def _pmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Product of 2-D polynomials given as coefficient grids c[i, j] x^i y^j."""
    out = np.zeros((a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1))
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            if a[i, j] != 0.0:
                out[i:i + b.shape[0], j:j + b.shape[1]] += a[i, j] * b
    return out


def _zernike_coeffs(j: int) -> np.ndarray:
    """Coefficient grid of Z_j(x, y) (x = rho cos t, y = rho sin t).

    Z = norm * R_n^|m|(rho) * {cos, sin}(|m| t), with
    R_n^|m| = sum_k (-1)^k (n-k)! / (k! ((n+|m|)/2-k)! ((n-|m|)/2-k)!) rho^(n-2k),
    norm = sqrt(n+1) for m = 0 else sqrt(2(n+1)). Each term rho^(n-2k) times
    the angular factor is (x^2+y^2)^e * Re/Im (x + i y)^|m|, e = (n-2k-|m|)/2.
    """
    n, m = noll_nm(j)
    am = abs(m)
    # angular part Re/Im (x + i y)^|m| = sum_t C(|m|, t) x^(|m|-t) (i y)^t
    ang = np.zeros((am + 1, am + 1))
    for t in range(am + 1):
        c = math.comb(am, t)
        if m >= 0 and t % 2 == 0:           # real part: i^t = (-1)^(t/2)
            ang[am - t, t] += c * (-1) ** (t // 2)
        if m < 0 and t % 2 == 1:            # imaginary part: i^t = i (-1)^((t-1)/2)
            ang[am - t, t] += c * (-1) ** ((t - 1) // 2)
    total = np.zeros((n + 1, n + 1))
    for k in range((n - am) // 2 + 1):
        coef = ((-1) ** k * math.factorial(n - k)
                / (math.factorial(k) * math.factorial((n + am) // 2 - k)
                   * math.factorial((n - am) // 2 - k)))
        e = (n - 2 * k - am) // 2
        rad = np.zeros((2 * e + 1, 2 * e + 1))        # (x^2 + y^2)^e
        for t in range(e + 1):
            rad[2 * t, 2 * (e - t)] = math.comb(e, t)
        term = _pmul(rad, ang) * coef
        total[:term.shape[0], :term.shape[1]] += term
    norm = math.sqrt(n + 1) if m == 0 else math.sqrt(2 * (n + 1))
    return norm * total


_ZC = {j: _zernike_coeffs(j) for j in range(1, 16)}


def zernike(j: int, x, y):
    return np.polynomial.polynomial.polyval2d(x, y, _ZC[j])


def zernike_grad(j: int, x, y):
    c = _ZC[j]
    dx = np.polynomial.polynomial.polyder(c, axis=0) if c.shape[0] > 1 else np.zeros((1, 1))
    dy = np.polynomial.polynomial.polyder(c, axis=1) if c.shape[1] > 1 else np.zeros((1, 1))
    return (np.polynomial.polynomial.polyval2d(x, y, dx),
            np.polynomial.polynomial.polyval2d(x, y, dy))


# --------------------------------------------------------------------------
# problem description
# --------------------------------------------------------------------------


@dataclass
class Geometry:
    """Imaging geometry (Section 2.1): grids, LED spectral offsets, pupil."""
    N: int
    m: int
    nominal: np.ndarray        # [n_leds, 2] spectral LED centres (row, col), px from DC
    R: float                   # pupil radius, spectral px
    edge: str = "aa"           # 'aa' | 'hard'
    lambda_um: float = 0.532
    dk_per_um: float = 1.0 / (64 * 0.6)

    def __post_init__(self):
        self.nominal = np.asarray(self.nominal, dtype=np.float64).reshape(-1, 2)
        self.n_int = np.rint(self.nominal).astype(np.int64)   # crop position
        assert self.N % self.m == 0 and self.m % 2 == 0

    @property
    def n_leds(self) -> int:
        return self.nominal.shape[0]

    @property
    def s(self) -> int:
        return self.N // self.m

    @property
    def centre_led(self) -> int:
        return int(np.argmin(np.hypot(self.nominal[:, 0], self.nominal[:, 1])))


@dataclass
class Params:
    """The jointly recovered quantities besides the object (Section 2.2)."""
    zernike: np.ndarray        # [14], Noll j = 2..15, rad
    defocus: float             # z, um
    gamma: np.ndarray          # [n_leds] intensity factors
    offset: np.ndarray         # [n_leds, 2] sub-pixel LED offsets delta, px
    pupil_ff: np.ndarray | None = None   # [m, m] complex free-form pupil nodes, or None (all ones)

    @staticmethod
    def initial(geom: Geometry) -> "Params":
        return Params(np.zeros(14), 0.0, np.ones(geom.n_leds),
                      geom.nominal - geom.n_int)

    def copy(self) -> "Params":
        return Params(self.zernike.copy(), float(self.defocus),
                      self.gamma.copy(), self.offset.copy(),
                      None if self.pupil_ff is None else self.pupil_ff.copy())


@dataclass
class Hparams:
    lr: dict = field(default_factory=lambda: dict(
        object=0.1, zernike=0.01, defocus=0.1, gamma=0.01, offset=0.01, pupil=0.01))
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    loss: str = "amplitude"    # 'amplitude' | 'intensity' | 'linear'
    learn: tuple = ("object",)
    offset_bound: float = 1.0
    gamma_floor: float = 1e-3  # intensity factors are held >= this (the amplitude loss takes sqrt(gamma))
    optimizer: str = "adam"    # 'adam' | 'adamw' | 'nadam' | 'rmsprop' (the Adam family of Section 2.2)
    weight_decay: float = 0.0  # AdamW's decoupled decay
    momentum_decay: float = 0.004  # NAdam's momentum schedule


# --------------------------------------------------------------------------
# model
# --------------------------------------------------------------------------


def object_spectrum(o: np.ndarray, s: int) -> np.ndarray:
    """Centred spectrum of the high-res object, DC at (N/2, N/2), scaled 1/s^2."""
    return np.fft.fftshift(np.fft.fft2(o)) / float(s * s)


def bilinear_upsample(a: np.ndarray, s: int) -> np.ndarray:
    """Upsample by integer s with bilinear weights, periodic boundary.

    Low-res pixel r sits on high-res pixel s*r (the sampling that cropping
    the centred spectrum and inverse-transforming on the m-grid implies), so
    high-res pixel Y takes source coordinate Y/s and the neighbours
    floor(Y/s) and floor(Y/s)+1 (mod m).
    """
    m0, m1 = a.shape

    def axis(n_in):
        src = np.arange(n_in * s) / s
        i0 = np.floor(src).astype(np.int64)
        return i0 % n_in, (i0 + 1) % n_in, src - i0

    y0, y1, wy = axis(m0)
    x0, x1, wx = axis(m1)
    top = a[y0][:, x0] * (1 - wx) + a[y0][:, x1] * wx
    bot = a[y1][:, x0] * (1 - wx) + a[y1][:, x1] * wx
    return top * (1 - wy)[:, None] + bot * wy[:, None]


def init_object(I_centre: np.ndarray, s: int) -> np.ndarray:
    """Initial spectrum: bilinear-upsampled centre-LED amplitude, zero phase."""
    o0 = bilinear_upsample(np.sqrt(np.maximum(np.asarray(I_centre, np.float64), 0.0)), s)
    return object_spectrum(o0.astype(np.complex128), s)


def bilinear_nodes(P: np.ndarray, qy: np.ndarray, qx: np.ndarray):
    """Bilinear interpolation of node values P[n + m/2] (n on the integer grid,
    m = P.shape[0]) at points q, with its derivatives along qy and qx.
    Returns (value, d/dqy, d/dqx, (iy, ix, fy, fx)): the lower-left node index
    (clipped to the grid) and the fractional parts."""
    m = P.shape[0]
    fy0, fx0 = np.floor(qy), np.floor(qx)
    fy, fx = qy - fy0, qx - fx0
    iy = np.clip(fy0.astype(np.int64) + m // 2, 0, m - 2)
    ix = np.clip(fx0.astype(np.int64) + m // 2, 0, m - 2)
    p00, p01 = P[iy, ix], P[iy, ix + 1]
    p10, p11 = P[iy + 1, ix], P[iy + 1, ix + 1]
    val = (1 - fy) * ((1 - fx) * p00 + fx * p01) + fy * ((1 - fx) * p10 + fx * p11)
    d_qy = (1 - fx) * (p10 - p00) + fx * (p11 - p01)
    d_qx = (1 - fy) * (p01 - p00) + fy * (p11 - p10)
    return val, d_qy, d_qx, (iy, ix, fy, fx)


def pupil(geom: Geometry, zern, z: float, delta, ff=None):
    """Pupil factor M(p) = A(q) exp(i chi(q)), q = p - delta, on the m x m grid.

    p runs over [-m/2, m/2)^2 (centred low-res spectrum index), q in px.
    chi = sum_j c_j Z_j(q/R) + z kappa(q). Returns a dict with M, A, chi,
    the Zernike values, kappa and the q-gradients of A and chi.
    """
    m, R = geom.m, float(geom.R)
    p = np.arange(m, dtype=np.float64) - m // 2
    py, px = np.meshgrid(p, p, indexing="ij")
    qy, qx = py - float(delta[0]), px - float(delta[1])
    r = np.hypot(qy, qx)
    if geom.edge == "aa":
        A = np.clip(R + 0.5 - r, 0.0, 1.0)
        ramp = (r > R - 0.5) & (r < R + 0.5)
        with np.errstate(invalid="ignore", divide="ignore"):
            dAy = np.where(ramp, -qy / r, 0.0)
            dAx = np.where(ramp, -qx / r, 0.0)
    else:
        A = (r <= R).astype(np.float64)
        dAy = np.zeros_like(r)
        dAx = np.zeros_like(r)
    xs, ys = qx / R, qy / R
    Z = np.stack([zernike(j, xs, ys) for j in range(2, 16)])
    dZ = [zernike_grad(j, xs, ys) for j in range(2, 16)]
    theta = np.tensordot(np.asarray(zern, np.float64), Z, axes=1)
    dth_x = sum(c * g[0] for c, g in zip(zern, dZ)) / R
    dth_y = sum(c * g[1] for c, g in zip(zern, dZ)) / R
    inside = A > 0
    k2 = (r * geom.dk_per_um) ** 2
    root = np.sqrt(np.where(inside, 1.0 / geom.lambda_um ** 2 - k2, 1.0))
    kappa = np.where(inside, 2 * math.pi * (root - 1.0 / geom.lambda_um), 0.0)
    dk2 = geom.dk_per_um ** 2
    dka_y = np.where(inside, -2 * math.pi * dk2 * qy / root, 0.0)
    dka_x = np.where(inside, -2 * math.pi * dk2 * qx / root, 0.0)
    chi = theta + z * kappa
    M0 = A * np.exp(1j * chi)
    out = dict(M=M0, M0=M0, A=A, chi=chi, Z=Z, kappa=kappa,
               dA=(dAy, dAx), dchi=(dth_y + z * dka_y, dth_x + z * dka_x), ff=None)
    if ff is not None:   # free-form factor P~(q) on top of the parametric pupil
        Pt, dPy, dPx, nodes = bilinear_nodes(np.asarray(ff, np.complex128), qy, qx)
        out.update(M=M0 * Pt, Pt=Pt, dP=(dPy, dPx), nodes=nodes, ff=True)
    return out


def crop(O: np.ndarray, geom: Geometry, i: int) -> np.ndarray:
    """m x m window of O centred at DC + n_i (centred low-res index)."""
    N, m = geom.N, geom.m
    r0 = N // 2 + int(geom.n_int[i, 0]) - m // 2
    c0 = N // 2 + int(geom.n_int[i, 1]) - m // 2
    assert 0 <= r0 and r0 + m <= N and 0 <= c0 and c0 + m <= N, "crop leaves the object grid"
    return O[r0:r0 + m, c0:c0 + m]


def forward_fields(O, prm: Params, geom: Geometry, i: int):
    """Eq. (3) for one LED: returns (Phi, psi, pupil dict)."""
    P = pupil(geom, prm.zernike, prm.defocus, prm.offset[i], prm.pupil_ff)
    Phi = crop(O, geom, i) * P["M"]
    psi = np.fft.ifft2(np.fft.ifftshift(Phi))
    return Phi, psi, P


def forward(O, prm: Params, geom: Geometry, idx) -> np.ndarray:
    """Predicted intensities I_i = gamma_i |psi_i|^2 for the LEDs in idx."""
    out = []
    for i in idx:
        _, psi, _ = forward_fields(O, prm, geom, int(i))
        out.append(prm.gamma[int(i)] * np.abs(psi) ** 2)
    return np.stack(out)


def loss_and_grad(O, prm: Params, geom: Geometry, idx, I_meas, loss: str = "amplitude"):
    """Batch loss (Eq. 5 summed over the batch, Eq. 13) and all gradients.

    I_meas: measured intensities for every LED, [n_leds, m, m].
    Returns (L, grads, per_led_losses) with grads keys object [N, N] complex,
    zernike [14], defocus, gamma [n_leds], offset [n_leds, 2], and pupil
    [m, m] complex (the free-form nodes; None without a free-form pupil).
    """
    m = geom.m
    gO = np.zeros_like(O, dtype=np.complex128)
    g_zern = np.zeros(14)
    g_z = 0.0
    g_gamma = np.zeros(geom.n_leds)
    g_off = np.zeros((geom.n_leds, 2))
    g_pup = None if prm.pupil_ff is None else np.zeros((m, m), np.complex128)
    per_led = []
    for i in idx:
        i = int(i)
        Phi, psi, P = forward_fields(O, prm, geom, i)
        g = prm.gamma[i]
        mag = np.abs(psi)
        meas = np.asarray(I_meas[i], np.float64)
        if loss == "amplitude":
            a = np.sqrt(np.maximum(meas, 0.0))
            res = math.sqrt(g) * mag - a
            Li = float(np.sum(res ** 2))
            with np.errstate(invalid="ignore", divide="ignore"):
                g_psi = np.where(mag > 0, 2.0 * res * math.sqrt(g) * psi / mag, 0.0)
            g_gamma[i] += float(np.sum(res * mag)) / math.sqrt(g)
        elif loss == "intensity":
            res = g * mag ** 2 - meas
            Li = float(np.sum(res ** 2))
            g_psi = 4.0 * g * res * psi
            g_gamma[i] += float(np.sum(2.0 * res * mag ** 2))
        elif loss == "linear":
            # L = sum_r w(r) I_pred(r) with weights w = I_meas: the pairing of
            # an upstream gradient dL/dI with the predicted intensities
            Li = float(np.sum(meas * g * mag ** 2))
            g_psi = 2.0 * g * meas * psi
            g_gamma[i] += float(np.sum(meas * mag ** 2))
        else:
            raise ValueError(loss)
        per_led.append(Li)
        # adjoint of psi = ifft2(ifftshift(Phi))
        g_Phi = np.fft.fftshift(np.fft.fft2(g_psi)) / float(m * m)
        M = P["M"]
        cO = crop(O, geom, i)
        crop(gO, geom, i)[...] += np.conj(M) * g_Phi
        g_M = np.conj(cO) * g_Phi
        t = np.real(np.conj(g_M) * 1j * M)              # dL/dchi per pixel
        g_zern += np.tensordot(P["Z"], t, axes=([1, 2], [0, 1]))
        g_z += float(np.sum(t * P["kappa"]))
        eP = np.exp(1j * P["chi"]) * (P["Pt"] if P["ff"] else 1.0)
        e = np.real(np.conj(g_M) * eP)                     # dL/dA per pixel
        for ax in (0, 1):
            g_off[i, ax] -= float(np.sum(t * P["dchi"][ax] + e * P["dA"][ax]))
        if P["ff"]:
            # G = dL/dP~ per pixel; P~ moves with q = p - delta, and spreads G
            # over its four nodes with the bilinear weights
            G = np.conj(P["M0"]) * g_M
            for ax in (0, 1):
                g_off[i, ax] -= float(np.sum(np.real(np.conj(G) * P["dP"][ax])))
            iy, ix, fy, fx = P["nodes"]
            for dy, dx, w in ((0, 0, (1 - fy) * (1 - fx)), (0, 1, (1 - fy) * fx),
                              (1, 0, fy * (1 - fx)), (1, 1, fy * fx)):
                np.add.at(g_pup, (iy + dy, ix + dx), w * G)
    grads = dict(object=gO, zernike=g_zern, defocus=g_z, gamma=g_gamma, offset=g_off, pupil=g_pup)
    return float(sum(per_led)), grads, per_led


def adam_update(w, g, m, v, t: int, lr: float, b1: float, b2: float, eps: float):
    """One Adam step on real arrays (Kingma & Ba 2015, Algorithm 1), in place."""
    m *= b1
    m += (1 - b1) * g
    v *= b2
    v += (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    w -= lr * mhat / (np.sqrt(vhat) + eps)


def adamw_update(w, g, m, v, t: int, lr: float, b1: float, b2: float, eps: float, wd: float):
    """AdamW (Loshchilov & Hutter 2019): the weights first decay by lr * wd, decoupled
    from the gradient, then take the Adam step."""
    w *= 1 - lr * wd
    adam_update(w, g, m, v, t, lr, b1, b2, eps)


def nadam_mu(t: int, b1: float, psi: float) -> float:
    """NAdam's momentum coefficient of step t: b1 (1 - 0.96^(t psi) / 2) (Dozat 2016, with
    the warming schedule of Sutskever et al. 2013)."""
    return b1 * (1.0 - 0.5 * 0.96 ** (t * psi))


def nadam_update(w, g, m, v, t: int, lr: float, b1: float, b2: float, eps: float,
                 prod_t: float, prod_next: float, psi: float):
    """One NAdam step (Dozat 2016): Adam's moments, but the step looks one momentum update
    ahead. prod_t = mu_1 ... mu_t and prod_next = prod_t mu_(t+1)."""
    mu, mu_next = nadam_mu(t, b1, psi), nadam_mu(t + 1, b1, psi)
    m *= b1
    m += (1 - b1) * g
    v *= b2
    v += (1 - b2) * g * g
    denom = np.sqrt(v / (1 - b2 ** t)) + eps
    w -= lr * (1 - mu) / (1 - prod_t) * g / denom
    w -= lr * mu_next / (1 - prod_next) * m / denom


def rmsprop_update(w, g, v, lr: float, alpha: float, eps: float):
    """RMSprop (Tieleman & Hinton 2012): a running mean of g^2 scales the step."""
    v *= alpha
    v += (1 - alpha) * g * g
    w -= lr * g / (np.sqrt(v) + eps)


# --------------------------------------------------------------------------
# reconstruction loop (Eq. 13-14)
# --------------------------------------------------------------------------


class Reconstruction:
    """Random-batch Adam reconstruction; the batch order is an input."""

    def __init__(self, geom: Geometry, I_meas, hp: Hparams | None = None,
                 O0=None, prm: Params | None = None):
        self.geom = geom
        self.I = np.asarray(I_meas)
        self.hp = hp or Hparams()
        self.O = (init_object(self.I[geom.centre_led], geom.s) if O0 is None
                  else np.array(O0, dtype=np.complex128))
        self.prm = prm.copy() if prm is not None else Params.initial(geom)
        self.t = 0
        self.epoch_loss = 0.0
        self._state = {}
        self._mu_prod = 1.0  # NAdam: product of the momentum coefficients so far

    def _moments(self, name, shape):
        if name not in self._state:
            self._state[name] = (np.zeros(shape), np.zeros(shape))
        return self._state[name]

    def _update(self, w, g, mm, vv, lr):
        """One step of the chosen optimiser on a real array, in place."""
        hp, t = self.hp, self.t
        if hp.optimizer == "adam":
            adam_update(w, g, mm, vv, t, lr, hp.beta1, hp.beta2, hp.eps)
        elif hp.optimizer == "adamw":
            adamw_update(w, g, mm, vv, t, lr, hp.beta1, hp.beta2, hp.eps, hp.weight_decay)
        elif hp.optimizer == "nadam":
            nadam_update(w, g, mm, vv, t, lr, hp.beta1, hp.beta2, hp.eps, self._mu_prod,
                         self._mu_prod * nadam_mu(t + 1, hp.beta1, hp.momentum_decay), hp.momentum_decay)
        elif hp.optimizer == "rmsprop":
            rmsprop_update(w, g, vv, lr, hp.beta2, hp.eps)
        else:
            raise ValueError(hp.optimizer)

    def step(self, idx) -> float:
        hp = self.hp
        if "pupil" in hp.learn and self.prm.pupil_ff is None:   # a learned free-form pupil starts at 1
            self.prm.pupil_ff = np.ones((self.geom.m, self.geom.m), np.complex128)
        L, g, _ = loss_and_grad(self.O, self.prm, self.geom, idx, self.I, hp.loss)
        self.t += 1
        t = self.t
        if hp.optimizer == "nadam":  # mu_1 ... mu_t, shared by every parameter
            self._mu_prod *= nadam_mu(t, hp.beta1, hp.momentum_decay)
        if "object" in hp.learn:
            w = np.stack([self.O.real, self.O.imag], axis=-1)
            gw = np.stack([g["object"].real, g["object"].imag], axis=-1)
            mm, vv = self._moments("object", w.shape)
            self._update(w, gw, mm, vv, hp.lr["object"])
            self.O = w[..., 0] + 1j * w[..., 1]
        for name, attr in (("zernike", "zernike"), ("gamma", "gamma"), ("offset", "offset")):
            if name in hp.learn:
                w = getattr(self.prm, attr)
                mm, vv = self._moments(name, w.shape)
                self._update(w, g[name], mm, vv, hp.lr[name])
        if "pupil" in hp.learn:
            w = np.stack([self.prm.pupil_ff.real, self.prm.pupil_ff.imag], axis=-1)
            gw = np.stack([g["pupil"].real, g["pupil"].imag], axis=-1)
            mm, vv = self._moments("pupil", w.shape)
            self._update(w, gw, mm, vv, hp.lr["pupil"])
            self.prm.pupil_ff = w[..., 0] + 1j * w[..., 1]
        if "defocus" in hp.learn:
            w = np.array([self.prm.defocus])
            mm, vv = self._moments("defocus", (1,))
            self._update(w, np.array([g["defocus"]]), mm, vv, hp.lr["defocus"])
            self.prm.defocus = float(w[0])
        if "offset" in hp.learn:
            np.clip(self.prm.offset, -hp.offset_bound, hp.offset_bound, out=self.prm.offset)
        if "gamma" in hp.learn:
            np.maximum(self.prm.gamma, hp.gamma_floor, out=self.prm.gamma)
        self.epoch_loss += L
        return L

    def run(self, batches) -> list:
        return [self.step(b) for b in batches]
