"""FP64 oracle: interpolated PSF library A and the simulated image S = A Z.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain NumPy, float64.

Conventions (readings of the paper, each pinned by a test):
* Scene pixel (iy, ix) of an N x N scene at S lambda/D per pixel sits at
  x = (ix - (N-1)/2) S, y = (iy - (N-1)/2) S  (Eq. 2-3, scene meshgrid with the
  half-pixel shift; pinned by the 286.838 mas / 66.431 deg example of Fig. 6).
  The scene is flattened row-major: j = iy*N + ix.  Image pixel i = p*n + q.
* Polar offsets (Sec. 2, "standard 2D arctangent"): r = sqrt(x^2 + y^2),
  cos(theta) = x / r, sin(theta) = y / r; r = 0 gives theta = 0.
* Radial interpolation (Sec. 2, RegularGridInterpolator on (r, y, x) queried at
  integer pixel nodes, i.e. a lerp in r): k = max{k : r_k <= r} clamped to
  [0, n_r - 2], w = (r - r_k) / (r_{k+1} - r_k) clamped at 0 below r_0;
  r > r_last gives a zero column.  Nearest: w -> 0 or 1, ties to the lower radius.
* Rotation (Sec. 2, rotate by theta) about the array centre c = (n-1)/2, bilinear,
  no reshape, taps outside the array read 0: output pixel (p, q) samples
  column a = c + cos*(q-c) + sin*(p-c), row b = c - sin*(q-c) + cos*(p-c), so the
  core of a +x PSF at distance r lands at (x, y).
* Column j of A is the flattened rotated PSF of scene pixel j (Eq. 4-5); the
  image is S = A Z (Eq. 6).  No flux renormalisation (Sec. 3).
"""
from __future__ import annotations

import numpy as np

ARCSEC_PER_RAD = 180.0 * 3600.0 / np.pi


def lambda_over_d_mas(lam_nm: float = 575.0, diameter_m: float = 2.3631) -> float:
    """Angular size of lambda/D in milliarcseconds (parameter block, Eq. 1)."""
    return lam_nm * 1e-9 / diameter_m * ARCSEC_PER_RAD * 1e3


def scene_offsets(N: int, S: float) -> tuple[np.ndarray, np.ndarray]:
    """Field offsets (x_j, y_j) of the N*N scene pixels, j = iy*N + ix (Eq. 2-3)."""
    c = (np.arange(N, dtype=np.float64) - (N - 1) / 2.0) * S
    x = np.tile(c, N)
    y = np.repeat(c, N)
    return x, y


def polar(x, y):
    """(r, cos theta, sin theta) of field offsets (Sec. 2)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    r = np.sqrt(x * x + y * y)
    safe = np.where(r > 0.0, r, 1.0)
    cos_t = np.where(r > 0.0, x / safe, 1.0)
    sin_t = np.where(r > 0.0, y / safe, 0.0)
    return r, cos_t, sin_t


def radial_bracket(r, radii, method: str = "linear"):
    """Bracketing library index k, weight w of PSF k+1, and validity (Sec. 2)."""
    radii = np.asarray(radii, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    k = np.searchsorted(radii, r, side="right") - 1
    k = np.clip(k, 0, len(radii) - 2)
    w = (r - radii[k]) / (radii[k + 1] - radii[k])
    w = np.maximum(w, 0.0)
    if method == "nearest":
        w = np.where(w > 0.5, 1.0, 0.0)
    elif method != "linear":
        raise ValueError(method)
    valid = r <= radii[-1]
    return k, w, valid


def interpolate_radial(lib: np.ndarray, k: int, w: float) -> np.ndarray:
    """P = (1 - w) L[k] + w L[k+1] (Sec. 2, linear interpolation in offset)."""
    return (1.0 - w) * lib[k] + w * lib[k + 1]


def rotate_bilinear(P: np.ndarray, cos_t: float, sin_t: float) -> np.ndarray:
    """Rotate an n x n PSF by theta about its centre, bilinear, zero outside (Sec. 2)."""
    n = P.shape[0]
    c = (n - 1) / 2.0
    p, q = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64),
                       indexing="ij")
    du = q - c
    dv = p - c
    a = c + cos_t * du + sin_t * dv
    b = c - sin_t * du + cos_t * dv
    q0 = np.floor(a)
    p0 = np.floor(b)
    fa = a - q0
    fb = b - p0
    out = np.zeros_like(P, dtype=np.float64)
    for dp, dq, wgt in ((0, 0, (1.0 - fa) * (1.0 - fb)), (0, 1, fa * (1.0 - fb)),
                        (1, 0, (1.0 - fa) * fb), (1, 1, fa * fb)):
        rr = (p0 + dp).astype(np.int64)
        cc = (q0 + dq).astype(np.int64)
        inside = (rr >= 0) & (rr < n) & (cc >= 0) & (cc < n)
        tap = P[np.clip(rr, 0, n - 1), np.clip(cc, 0, n - 1)]
        out += np.where(inside, wgt * tap, 0.0)
    return out


def psf_column(lib: np.ndarray, radii, x: float, y: float, method: str = "linear") -> np.ndarray:
    """Flattened interpolated + rotated PSF of the field point (x, y) (Sec. 2 loop body)."""
    lib = np.asarray(lib, dtype=np.float64)
    r, cos_t, sin_t = polar(x, y)
    k, w, valid = radial_bracket(r, radii, method)
    if not bool(valid):
        return np.zeros(lib.shape[1] * lib.shape[2])
    P = interpolate_radial(lib, int(k), float(w))
    return rotate_bilinear(P, float(cos_t), float(sin_t)).ravel()


def build_points(lib, radii, xs, ys, method: str = "linear") -> np.ndarray:
    """A restricted to arbitrary field points: M x len(xs) (Eq. 4-5)."""
    cols = [psf_column(lib, radii, float(x), float(y), method) for x, y in zip(xs, ys)]
    return np.stack(cols, axis=1)


def build_A(lib, radii, N: int, S: float, method: str = "linear") -> np.ndarray:
    """Full interpolated PSF matrix A (n^2 x N^2), one scene pixel per column (Eq. 5)."""
    x, y = scene_offsets(N, S)
    return build_points(lib, radii, x, y, method)


def A_rows(lib, radii, xs, ys, rows, method: str = "linear") -> np.ndarray:
    """Rows `rows` of A for field points (xs, ys), each element from its definition.

    A[i, j] = sum over the 4 bilinear taps t of weight_t(i, j) *
              ((1 - w_j) L[k_j][t] + w_j L[k_j + 1][t]),
    the same quantity psf_column computes, evaluated one output pixel at a time
    so that large workloads can be sampled row by row.
    """
    lib = np.asarray(lib, dtype=np.float64)
    n = lib.shape[1]
    c = (n - 1) / 2.0
    r, cos_t, sin_t = polar(xs, ys)
    k, w, valid = radial_bracket(r, radii, method)
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), len(r)), dtype=np.float64)
    for t, i in enumerate(rows):
        p, q = divmod(int(i), n)
        du = q - c
        dv = p - c
        a = c + cos_t * du + sin_t * dv
        b = c - sin_t * du + cos_t * dv
        q0 = np.floor(a)
        p0 = np.floor(b)
        fa = a - q0
        fb = b - p0
        acc = np.zeros(len(r))
        for dp, dq, wgt in ((0, 0, (1.0 - fa) * (1.0 - fb)), (0, 1, fa * (1.0 - fb)),
                            (1, 0, (1.0 - fa) * fb), (1, 1, fa * fb)):
            rr = (p0 + dp).astype(np.int64)
            cc = (q0 + dq).astype(np.int64)
            inside = (rr >= 0) & (rr < n) & (cc >= 0) & (cc < n)
            rc = np.clip(rr, 0, n - 1)
            ccc = np.clip(cc, 0, n - 1)
            tap = (1.0 - w) * lib[k, rc, ccc] + w * lib[k + 1, rc, ccc]
            acc += np.where(inside, wgt * tap, 0.0)
        out[t] = np.where(valid, acc, 0.0)
    return out


def forward(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Simulated image(s) S = A Z (Eq. 6); x is (K,) or (B, K), result (M,) or (B, M)."""
    x = np.asarray(x, dtype=np.float64)
    return (A @ x.T).T


def adjoint(A: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Transpose product A^T g; g is (M,) or (B, M)."""
    g = np.asarray(g, dtype=np.float64)
    return (A.T @ g.T).T


def error_bound(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Per-pixel scale sum_j |A_ij| |x_j| used to normalise image errors."""
    return forward(np.abs(A), np.abs(x))


FLT_MIN = float(np.finfo(np.float32).tiny)


def bound_relative_error(y, y_ref, bound, floor: float = 0.0) -> np.ndarray:
    """|y - y_ref| / max(bound, floor), with 0/0 = 0 and e/0 = inf.

    A float32 result below FLT_MIN is subnormal and carries only absolute
    precision, so comparisons of float32 images pass floor=FLT_MIN: pixels
    whose bound lies below the normal range are then held to 1e-5 * FLT_MIN.
    """
    y = np.asarray(y, dtype=np.float64)
    err = np.abs(y - np.asarray(y_ref, dtype=np.float64))
    bound = np.maximum(np.asarray(bound, dtype=np.float64), floor)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.where(bound > 0.0, err / np.where(bound > 0.0, bound, 1.0),
                       np.where(err > 0.0, np.inf, 0.0))
    return rel
