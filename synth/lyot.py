"""Synthetic Lyot-coronagraph PSF library (input preparation only).

Stands in for the off-axis PSF cubes of Sec. 2 (IPAC HLC cube) and Sec. 4.1
(PROPER cubes), which are not available.  Each PSF is the image of a point
source at an offset ``r`` along +x, made by a small scalar Fraunhofer model:

* circular pupil sampled with ``pupil_px`` points across the diameter D;
* tilt phase that moves the source to ``r`` (lambda0/D on the sky);
* seeded Noll Zernike Z4-Z11 phase error, ``wfe_rms`` waves RMS at lambda0;
* focal-plane occulter with amplitude transmission 1 - exp(-(rho/rho0)^4);
* Lyot stop of ``lyot_frac`` x D;
* final image sampled at ``s`` lambda0/D per pixel on an n x n grid whose
  optical axis sits at pixel coordinate ((n-1)/2, (n-1)/2);
* normalised so that the unocculted on-axis peak is 1 (contrast units).

All propagations are matrix Fourier transforms, so any wavelength can be
sampled on the same sky grid (lambda0/D units).  The occulter is applied with
Babinet's principle: the Lyot-plane field is the pupil field minus the inverse
transform of (1 - t) times the focal field, and 1 - t is compact.
"""
from __future__ import annotations

import numpy as np

LAMBDA0_NM = 575.0


def _noll_z4_z11(rho: np.ndarray, phi: np.ndarray) -> list[np.ndarray]:
    """Noll-normalised Zernike polynomials Z4..Z11 on the unit disk."""
    r2 = rho * rho
    return [
        np.sqrt(3.0) * (2.0 * r2 - 1.0),                       # Z4 defocus
        np.sqrt(6.0) * r2 * np.sin(2.0 * phi),                 # Z5 astig
        np.sqrt(6.0) * r2 * np.cos(2.0 * phi),                 # Z6 astig
        np.sqrt(8.0) * (3.0 * r2 * rho - 2.0 * rho) * np.sin(phi),   # Z7 coma
        np.sqrt(8.0) * (3.0 * r2 * rho - 2.0 * rho) * np.cos(phi),   # Z8 coma
        np.sqrt(8.0) * r2 * rho * np.sin(3.0 * phi),           # Z9 trefoil
        np.sqrt(8.0) * r2 * rho * np.cos(3.0 * phi),           # Z10 trefoil
        np.sqrt(5.0) * (6.0 * r2 * r2 - 6.0 * r2 + 1.0),       # Z11 spherical
    ]


def _mft_matrix(out_coords: np.ndarray, in_coords: np.ndarray, sign: float) -> np.ndarray:
    return np.exp(sign * 2j * np.pi * np.outer(out_coords, in_coords))


class LyotModel:
    """Seeded pupil + aberration description shared by every PSF of a library."""

    def __init__(self, seed: int, pupil_px: int = 64, wfe_rms: float = 0.02,
                 rho0: float = 2.5, lyot_frac: float = 0.9,
                 focal_half: float = 6.0, focal_step: float = 0.05):
        self.pupil_px = pupil_px
        k = np.arange(pupil_px, dtype=np.float64)
        self.xp = (k - (pupil_px - 1) / 2.0) / pupil_px          # units of D
        X, Y = np.meshgrid(self.xp, self.xp, indexing="xy")
        R = np.hypot(X, Y)
        self.pupil = (R <= 0.5).astype(np.float64)
        self.lyot = (R <= 0.5 * lyot_frac).astype(np.float64)
        rng = np.random.default_rng(seed)
        coeffs = rng.standard_normal(8)
        coeffs *= wfe_rms / np.sqrt(np.sum(coeffs ** 2))
        rho = np.clip(R / 0.5, 0.0, None)
        phi = np.arctan2(Y, X)
        self.opd_waves = sum(c * z for c, z in zip(coeffs, _noll_z4_z11(rho, phi))) * self.pupil
        self.X = X
        self.rho0 = rho0
        m = int(round(2 * focal_half / focal_step))
        self.uf = (np.arange(m) - (m - 1) / 2.0) * focal_step   # lambda/D
        self.df = focal_step
        self.dp = 1.0 / pupil_px

    def _pupil_field(self, offset_ld: float, lam_ratio: float) -> np.ndarray:
        """Pupil field at wavelength lambda = lambda0 * lam_ratio for a source at offset_ld (lambda0/D)."""
        phase = 2.0 * np.pi * (self.opd_waves / lam_ratio + (offset_ld / lam_ratio) * self.X)
        return self.pupil * np.exp(1j * phase)

    def _lyot_field(self, e_pupil: np.ndarray, lam_ratio: float, occulted: bool) -> np.ndarray:
        if not occulted:
            return e_pupil
        fwd = _mft_matrix(self.uf, self.xp, -1.0)
        focal = fwd @ e_pupil @ fwd.T * (self.dp * self.dp)
        U, V = np.meshgrid(self.uf, self.uf, indexing="xy")
        rho_ld = np.hypot(U, V)                                  # lambda/D at this wavelength
        blocked = np.exp(-((rho_ld * lam_ratio / self.rho0) ** 4))
        inv = _mft_matrix(self.xp, self.uf, +1.0)
        return e_pupil - inv @ (blocked * focal) @ inv.T * (self.df * self.df)

    def image(self, offset_ld: float, n: int, s: float, lam_ratio: float = 1.0,
              binning: int = 1, occulted: bool = True) -> np.ndarray:
        """n x n intensity image, pixels of s lambda0/D, axis at ((n-1)/2, (n-1)/2)."""
        e = self._lyot_field(self._pupil_field(offset_ld, lam_ratio), lam_ratio, occulted)
        e = e * self.lyot
        m = n * binning
        sub = s / binning
        u = (np.arange(m) - (m - 1) / 2.0) * sub / lam_ratio     # lambda/D at this wavelength
        w = _mft_matrix(u, self.xp, -1.0)
        field = w @ e @ w.T * (self.dp * self.dp)
        inten = np.abs(field) ** 2
        if binning > 1:
            inten = inten.reshape(n, binning, n, binning).sum(axis=(1, 3)) / (binning * binning)
        return inten

    def unocculted_peak(self, lam_ratio: float = 1.0) -> float:
        e = self._pupil_field(0.0, lam_ratio) * self.lyot
        return float(np.abs(np.sum(e) * self.dp * self.dp) ** 2)


def psf_library(radii: np.ndarray, n: int, s: float, seed: int, lam_ratio: float = 1.0,
                binning: int = 1) -> np.ndarray:
    """Radial PSF library L[k][p][q] (float64), source at radii[k] lambda0/D along +x.

    Row p grows with +y, column q with +x; the optical axis is at ((n-1)/2, (n-1)/2).
    """
    model = LyotModel(seed)
    peak = model.unocculted_peak(lam_ratio)
    lib = np.empty((len(radii), n, n), dtype=np.float64)
    for k, r in enumerate(radii):
        lib[k] = model.image(float(r), n, s, lam_ratio, binning) / peak
    return lib
