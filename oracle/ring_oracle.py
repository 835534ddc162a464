"""FP64 oracle for the ring scene model, its parameter gradient and the fit loss.

TEST INFRASTRUCTURE ONLY.  The paper's flow chart (Fig. 3) ends in retrieving
exozodi parameters from simulated images; this module gives the model and the
chain rule through S = A Z (Eq. 6) that such a retrieval needs.

Ring brightness at scene pixel j with offsets (x, y) (lambda/D), parameters
theta = (R, w, i, g, B):
  yd = y / cos i, rd = sqrt(x^2 + yd^2), mu = sin i * yd / rd (0 at rd = 0)
  G  = exp(-a (rd - R)^2 / w^2), a = 4 ln 2          (w = FWHM of the profile)
  H  = ((1 + g^2) / (1 + g^2 - 2 g mu))^(3/2)         (= HG_g(mu) / HG_g(0))
  Z_j = B G H for sqrt(x^2 + y^2) <= r_max, else 0.
Loss: L = 1/2 sum_i ((A Z - d)_i / sigma)^2, dL/dZ = A^T (A Z - d) / sigma^2,
dL/dtheta_m = sum_j dL/dZ_j dZ_j/dtheta_m.
"""
from __future__ import annotations

import numpy as np

from .psfsim_oracle import scene_offsets, forward, adjoint

ALPHA = 4.0 * np.log(2.0)


def hg(mu, g):
    """Henyey-Greenstein phase function HG_g(mu), normalised over the sphere."""
    return (1.0 - g * g) / (4.0 * np.pi * (1.0 + g * g - 2.0 * g * mu) ** 1.5)


def ring_scene(theta, N: int, S: float, r_max: float) -> np.ndarray:
    """Flattened ring scene Z (K = N^2), float64."""
    Z, _ = ring_scene_and_jacobian(theta, N, S, r_max, jacobian=False)
    return Z


def ring_scene_and_jacobian(theta, N: int, S: float, r_max: float, jacobian: bool = True):
    """Z (K,) and dZ/dtheta (K, 5) by the analytic chain rule."""
    R, w, inc, g, B = (float(v) for v in theta)
    x, y = scene_offsets(N, S)
    ci, si = np.cos(inc), np.sin(inc)
    yd = y / ci
    rd = np.sqrt(x * x + yd * yd)
    pos = rd > 0.0
    rds = np.where(pos, rd, 1.0)
    mu = np.where(pos, si * yd / rds, 0.0)
    G = np.exp(-ALPHA * (rd - R) ** 2 / (w * w))
    den = 1.0 + g * g - 2.0 * g * mu
    H = ((1.0 + g * g) / den) ** 1.5
    mask = np.sqrt(x * x + y * y) <= r_max
    Z = np.where(mask, B * G * H, 0.0)
    if not jacobian:
        return Z, None
    dyd_di = yd * si / ci                       # d(y / cos i)/di
    drd_di = np.where(pos, yd * dyd_di / rds, 0.0)
    dmu_di = np.where(pos, ci * yd / rds + si * (dyd_di * rd - yd * drd_di) / (rds * rds), 0.0)
    dG_dR = G * 2.0 * ALPHA * (rd - R) / (w * w)
    dG_dw = G * 2.0 * ALPHA * (rd - R) ** 2 / (w ** 3)
    dG_di = -G * 2.0 * ALPHA * (rd - R) / (w * w) * drd_di
    dH_dmu = 3.0 * g * H / den
    dH_dg = H * 1.5 * (2.0 * g / (1.0 + g * g) - (2.0 * g - 2.0 * mu) / den)
    J = np.stack([B * dG_dR * H, B * dG_dw * H, B * (dG_di * H + G * dH_dmu * dmu_di),
                  B * G * dH_dg, G * H], axis=1)
    J[~mask] = 0.0
    return Z, J


def fit_loss(A, theta, d, sigma, N, S, r_max) -> float:
    """L(theta) = 1/2 sum ((A Z(theta) - d) / sigma)^2."""
    res = (forward(A, ring_scene(theta, N, S, r_max)) - d) / sigma
    return 0.5 * float(res @ res)


def fit_loss_and_grad(A, theta, d, sigma, N, S, r_max):
    """(L, dL/dtheta) through Z -> A Z -> loss and back with A^T (chain rule)."""
    Z, J = ring_scene_and_jacobian(theta, N, S, r_max)
    res = forward(A, Z) - d
    loss = 0.5 * float(res @ res) / (sigma * sigma)
    gZ = adjoint(A, res / (sigma * sigma))
    return loss, J.T @ gZ
