"""Seeded synthetic discs on the log-polar grid.

This module only draws input fields; it contains none of the self-gravity
arithmetic and imports nothing else from this package, so the CUDA path and
the CPU oracle can both be fed from it.

Grid convention: ``nr`` cells log-spaced between the radial edges ``r_in`` and
``r_out`` (centres r_i = r_in exp((i + 1/2) du)), ``nphi`` cells uniform in
phi (centres phi_j = (j + 1/2) 2 pi / nphi).  Arrays are row-major
``[nr][nphi]`` float64.

Recipes (all numpy PCG64, seed = 2506108120 + recipe offset):

``small_gas``        64 x 128, r in [0.2, 2.5], h = 0.05, G = 1,
                     Sigma_g = r^-1 (1 + 0.01 U(-1, 1)).
``spiral_bifluid``   256 x 512, r in [0.1, 5], h_g = 0.05, dust scale height
                     H_d = H_g sqrt(alpha / (alpha + St)), alpha = 1e-3,
                     Sigma_g = r^-1 [1 + 0.1 cos(2 (phi - cot(15 deg) ln(r / r_in)))]
                     (1 + 0.01 U), Sigma_d = 0.01 Sigma_g (1 + 0.01 U').
``lognormal_gas``    any size, r in [0.1, 5], h = 0.05,
                     Sigma = r^-1 exp(0.3 G - 0.045)
                     (1 + sum_{m=2..4} 0.05 cos(m (phi - cot(15 deg) ln(r / r_in)) + psi_m)),
                     G a unit-variance Gaussian random field with Gaussian
                     correlation length 5 cells (white noise filtered in
                     Fourier space on a [2 nr, nphi] grid, periodic in phi,
                     cropped to nr rows), psi_m uniform phases.
``batch_discs``      n independent gas + dust discs (default 64): grid drawn from
                     {128x256, 256x512, 512x1024, 1024x2048}, h_g uniform in [0.03, 0.1],
                     St from {0.01, 0.1, 1}, each a log-normal disc (recipe above,
                     its own seed) with a 1 % dust fraction.
``clumpy_gas``       Gaussian clumps Sigma (1 + A exp(-|r - r_c|^2 / 2 R^2)) on a
                     smooth r^-1 disc, the clump form of the paper's Gaussian
                     discs test (Sec. 4.4).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED0 = 2506108120
PITCH_DEG = 15.0


@dataclass
class Disc:
    nr: int
    nphi: int
    r_in: float
    r_out: float
    h_g: float
    h_d: float | None
    G: float
    sigma_g: np.ndarray
    sigma_d: np.ndarray | None
    label: str

    @property
    def cells(self) -> int:
        return self.nr * self.nphi


def _centres(nr, nphi, r_in, r_out):
    du = np.log(r_out / r_in) / nr
    r = r_in * np.exp((np.arange(nr) + 0.5) * du)
    phi = (np.arange(nphi) + 0.5) * (2.0 * np.pi / nphi)
    return r, phi


def _rng(offset):
    return np.random.Generator(np.random.PCG64(SEED0 + offset))


def dust_aspect_ratio(h_g, St, alpha=1e-3):
    """H_d = H_g sqrt(alpha / (alpha + St)) (a diffusion-settling scale height)."""
    return h_g * np.sqrt(alpha / (alpha + St))


def small_gas(nr=64, nphi=128, r_in=0.2, r_out=2.5, h=0.05, G=1.0, offset=0):
    rng = _rng(offset)
    r, _ = _centres(nr, nphi, r_in, r_out)
    sig = (1.0 / r)[:, None] * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, (nr, nphi)))
    return Disc(nr, nphi, r_in, r_out, h, None, G, sig, None, f"gas {nr}x{nphi} r^-1 + 1% noise")


def _spiral(r, phi, r_in, m):
    cot = 1.0 / np.tan(np.radians(PITCH_DEG))
    return np.cos(m * (phi[None, :] - cot * np.log(r / r_in)[:, None]))


def spiral_bifluid(St=0.1, nr=256, nphi=512, r_in=0.1, r_out=5.0, h_g=0.05, G=1.0,
                   dust_to_gas=0.01, offset=1):
    rng = _rng(offset)
    r, phi = _centres(nr, nphi, r_in, r_out)
    sg = (1.0 / r)[:, None] * (1.0 + 0.1 * _spiral(r, phi, r_in, 2))
    sg = sg * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, (nr, nphi)))
    sd = dust_to_gas * sg * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, (nr, nphi)))
    return Disc(nr, nphi, r_in, r_out, h_g, float(dust_aspect_ratio(h_g, St)), G, sg, sd,
                f"gas+dust {nr}x{nphi} St={St} m=2 spiral")


def gaussian_random_field(rng, nr, nphi, corr_cells=5.0):
    """Unit-variance Gaussian random field with correlation exp(-l^2 / (2 c^2))
    in index space: white noise filtered by exp(-pi^2 c^2 k^2) on [2 nr, nphi]."""
    w = rng.standard_normal((2 * nr, nphi))
    kx = np.fft.fftfreq(2 * nr)[:, None]
    ky = np.fft.rfftfreq(nphi)[None, :]
    filt = np.exp(-(np.pi * corr_cells) ** 2 * (kx * kx + ky * ky))
    g = np.fft.irfft2(np.fft.rfft2(w) * filt, s=(2 * nr, nphi))[:nr]
    return g / g.std()


def lognormal_gas(nr=2048, nphi=4096, r_in=0.1, r_out=5.0, h=0.05, G=1.0, offset=2,
                  sigma_ln=0.3, corr_cells=5.0):
    rng = _rng(offset)
    r, phi = _centres(nr, nphi, r_in, r_out)
    g = gaussian_random_field(rng, nr, nphi, corr_cells)
    psi = rng.uniform(0.0, 2.0 * np.pi, 3)
    sp = np.ones((nr, nphi))
    cot = 1.0 / np.tan(np.radians(PITCH_DEG))
    for m, p in zip((2, 3, 4), psi):
        sp += 0.05 * np.cos(m * (phi[None, :] - cot * np.log(r / r_in)[:, None]) + p)
    sig = (1.0 / r)[:, None] * np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2) * sp
    return Disc(nr, nphi, r_in, r_out, h, None, G, sig, None,
                f"gas {nr}x{nphi} log-normal(0.3, 5 cells) + m=2..4 spirals")


def lognormal_bifluid(nr=2048, nphi=4096, St=0.1, dust_to_gas=0.01, offset=3, **kw):
    d = lognormal_gas(nr, nphi, offset=offset, **kw)
    rng = _rng(offset + 100)
    sd = dust_to_gas * d.sigma_g * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, (nr, nphi)))
    return Disc(nr, nphi, d.r_in, d.r_out, d.h_g, float(dust_aspect_ratio(d.h_g, St)), d.G,
                d.sigma_g, sd, d.label.replace("gas", "gas+dust") + f" St={St}")


def clumpy_gas(nr=256, nphi=512, r_in=0.1, r_out=5.0, h=0.05, G=1.0, offset=4, n_clumps=3):
    rng = _rng(offset)
    r, phi = _centres(nr, nphi, r_in, r_out)
    R, P = np.meshgrid(r, phi, indexing="ij")
    x, y = R * np.cos(P), R * np.sin(P)
    sig = 1.0 / R
    for _ in range(n_clumps):
        rc = rng.uniform(0.5, 3.0)
        pc = rng.uniform(0.0, 2.0 * np.pi)
        A = rng.uniform(1.0, 10.0)
        Rc = rng.uniform(0.05, 0.2)
        d2 = (x - rc * np.cos(pc)) ** 2 + (y - rc * np.sin(pc)) ** 2
        sig = sig * (1.0 + A * np.exp(-d2 / (2.0 * Rc * Rc)))
    return Disc(nr, nphi, r_in, r_out, h, None, G, sig, None, f"gas {nr}x{nphi} {n_clumps} clumps")


def ragged_noise(nr, nphi, r_in=0.3, r_out=3.0, h=0.07, G=1.0, offset=5, bifluid=False,
                 St=0.1):
    """Uniform random surface densities (no structure) for parity edge cases."""
    rng = _rng(offset)
    sg = rng.uniform(0.5, 1.5, (nr, nphi))
    sd = 0.01 * rng.uniform(0.5, 1.5, (nr, nphi)) if bifluid else None
    return Disc(nr, nphi, r_in, r_out, h, float(dust_aspect_ratio(h, St)) if bifluid else None,
                G, sg, sd, f"noise {nr}x{nphi}")


BATCH_SHAPES = ((128, 256), (256, 512), (512, 1024), (1024, 2048))


def batch_discs(n=64, offset=10, shapes=BATCH_SHAPES, St_choices=(0.01, 0.1, 1.0)):
    """n independent gas + dust discs of uneven size (see the module docstring)."""
    rng = _rng(offset)
    discs = []
    for k in range(n):
        nr, nphi = shapes[int(rng.integers(len(shapes)))]
        h = float(rng.uniform(0.03, 0.1))
        St = float(St_choices[int(rng.integers(len(St_choices)))])
        d = lognormal_bifluid(nr, nphi, St=St, offset=offset + 1 + k, h=h)
        discs.append(d)
    return discs

