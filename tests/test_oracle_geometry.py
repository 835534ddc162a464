"""Pins of the oracle's geometry, radial interpolation and rotation (CPU only).

Each test checks the FP64 oracle against something other than itself: numbers
printed in the paper (tests/golden), NumPy/SciPy routines, or exact invariants
of the method (Sec. 2-3).
"""
import json
import os

import numpy as np
import pytest

from oracle import psfsim_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _random_lib(n_r, n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(n_r, n, n))


def test_parameter_block_units():
    g = _golden("parameter_block.json")
    ld = O.lambda_over_d_mas(g["lambda_nm"], g["D_m"])
    assert round(g["s_px_lambda_over_d"] * ld, 3) == pytest.approx(g["s_px_mas"], abs=1e-9)
    half = g["N_px"] / 2 * g["S_px_mas"] / ld
    assert half == pytest.approx(g["scene_half_extent_lambda_over_d"], abs=0.01)


def test_worked_example_pins_half_pixel_meshgrid():
    """Fig. 6 / Fig. 13: 286.838 mas at 66.431 deg is a pixel centre of the 256^2 scene."""
    g = _golden("worked_example_offset.json")
    x, y = O.scene_offsets(g["N"], g["S_mas"])
    r, c, s = O.polar(x, y)
    th = np.degrees(np.arctan2(s, c))
    tol = 0.5 * 10.0 ** -g["quoted_decimals"]
    hit = (np.abs(r - g["r_mas"]) <= tol) & (np.abs(th - g["theta_deg"]) <= tol)
    assert hit.sum() == 1
    j = int(np.nonzero(hit)[0][0])
    iy, ix = divmod(j, g["N"])
    assert (ix, iy) == (160, 202)
    # The same offset is not a pixel centre of an integer-offset grid (no half-pixel shift).
    ci = (np.arange(g["N"]) - g["N"] / 2) * g["S_mas"]
    xi, yi = np.meshgrid(ci, ci)
    ri = np.hypot(xi, yi)
    ti = np.degrees(np.arctan2(yi, xi))
    assert not np.any((np.abs(ri - g["r_mas"]) <= tol) & (np.abs(ti - g["theta_deg"]) <= tol))


def test_matrix_shape_and_file_sizes():
    g = _golden("matrix_sizes.json")
    for case in g["cases"]:
        M, K = case["n"] ** 2, case["N"] ** 2
        assert M * K * 8 / 2 ** 30 == pytest.approx(case["file_GB"])
    lib = _random_lib(4, 6, 0)
    A = O.build_A(lib, np.array([0.0, 1.0, 2.0, 3.0]), 5, 0.5)
    assert A.shape == (36, 25)


def test_scene_flattening_row_major():
    x, y = O.scene_offsets(4, 1.0)
    X, Y = np.meshgrid(np.arange(4) - 1.5, np.arange(4) - 1.5, indexing="xy")
    assert np.array_equal(x, X.ravel()) and np.array_equal(y, Y.ravel())


def test_theta_zero_is_identity_and_lerp_hits_samples():
    radii = np.array([0.0, 0.75, 1.5, 3.0])   # binary fractions: the midpoint weight is exactly 1/2
    lib = _random_lib(4, 9, 1)
    for k in range(4):
        col = O.psf_column(lib, radii, radii[k], 0.0)
        assert np.array_equal(col, lib[k].ravel())
    mid = 0.5 * (radii[1] + radii[2])
    col = O.psf_column(lib, radii, mid, 0.0)
    assert np.array_equal(col, (0.5 * lib[1] + 0.5 * lib[2]).ravel())


@pytest.mark.parametrize("n", [8, 9])
def test_quarter_turns_are_exact_permutations(n):
    radii = np.array([0.0, 1.0, 2.5, 4.0])
    lib = _random_lib(4, n, 2)
    for k in (1, 2, 3):
        r = radii[k]
        base = lib[k]
        assert np.array_equal(O.psf_column(lib, radii, 0.0, r).reshape(n, n), np.rot90(base, -1))
        assert np.array_equal(O.psf_column(lib, radii, -r, 0.0).reshape(n, n), np.rot90(base, 2))
        assert np.array_equal(O.psf_column(lib, radii, 0.0, -r).reshape(n, n), np.rot90(base, 1))


def test_scene_grid_rot90_symmetry():
    """Column of the pixel at (-y, x) is the quarter-turned column of the pixel at (x, y)."""
    n, N, S = 10, 6, 0.7
    radii = np.linspace(0.0, 3.0, 7)
    lib = _random_lib(7, n, 3)
    A = O.build_A(lib, radii, N, S)
    for iy in range(N):
        for ix in range(N):
            j = iy * N + ix
            j2 = ix * N + (N - 1 - iy)           # (x, y) -> (-y, x)
            a = A[:, j].reshape(n, n)
            b = A[:, j2].reshape(n, n)
            np.testing.assert_allclose(b, np.rot90(a, -1), rtol=0, atol=1e-13)  # FP64 evaluation order only


def test_core_lands_at_field_offset():
    """One-hot scene through a library of sharp cores: image peak at (c + x/s, c + y/s)."""
    n, s, N, S = 33, 0.5, 12, 0.5
    radii = np.arange(0, 13) * 0.5                 # integer pixel offsets of the core
    c = (n - 1) / 2
    lib = np.zeros((len(radii), n, n))
    for k, r in enumerate(radii):
        lib[k, int(c), int(c + r / s)] = 1.0
    A = O.build_A(lib, radii, N, S)
    x, y = O.scene_offsets(N, S)
    rng = np.random.default_rng(4)
    for j in rng.choice(N * N, 20, replace=False):
        if np.hypot(x[j], y[j]) > radii[-1]:
            continue
        e = np.zeros(N * N)
        e[j] = 1.0
        img = O.forward(A, e)
        assert np.array_equal(img, A[:, j])       # one-hot returns the column exactly
        p, q = np.unravel_index(np.argmax(img), (n, n))
        assert abs(q - (c + x[j] / s)) <= 1.0 and abs(p - (c + y[j] / s)) <= 1.0


def test_beyond_last_radius_is_zero_and_below_first_clamps():
    radii = np.array([0.5, 1.0, 2.0])
    lib = _random_lib(3, 7, 5)
    assert not np.any(O.psf_column(lib, radii, 2.0001, 0.0))
    assert np.array_equal(O.psf_column(lib, radii, 0.2, 0.0), lib[0].ravel())
    assert np.array_equal(O.psf_column(lib, radii, 2.0, 0.0), lib[2].ravel())


def test_nearest_ties_go_low():
    radii = np.array([0.0, 1.0, 2.0])
    k, w, _ = O.radial_bracket(np.array([0.5, 0.5000001, 1.5, 0.49]), radii, "nearest")
    assert list(k) == [0, 0, 1, 0] and list(w) == [0.0, 1.0, 0.0, 0.0]


def test_linearity_and_dot_product():
    n, N, S = 12, 10, 0.6
    radii = np.linspace(0.0, 4.0, 9)
    lib = _random_lib(9, n, 6)
    A = O.build_A(lib, radii, N, S)
    rng = np.random.default_rng(7)
    x, z = rng.standard_normal((2, N * N))
    g = rng.standard_normal(n * n)
    np.testing.assert_allclose(O.forward(A, 2.0 * x - 3.0 * z),
                               2.0 * O.forward(A, x) - 3.0 * O.forward(A, z), rtol=1e-12, atol=1e-12)
    lhs = O.forward(A, x) @ g
    rhs = x @ O.adjoint(A, g)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(A) @ np.abs(x)) @ np.abs(g)


def test_rows_agree_with_columns():
    n, N, S = 11, 9, 0.45
    radii = np.array([0.0, 0.3, 1.1, 2.0, 3.5])
    lib = _random_lib(5, n, 8)
    A = O.build_A(lib, radii, N, S)
    x, y = O.scene_offsets(N, S)
    rows = np.array([0, 5, 60, 120])
    np.testing.assert_allclose(O.A_rows(lib, radii, x, y, rows), A[rows], rtol=0, atol=1e-15)


def test_against_scipy_routines_named_by_the_paper():
    """Sec. 2: RegularGridInterpolator (linear) + rotate, with order=1, no reshape, zero fill."""
    interp = pytest.importorskip("scipy.interpolate")
    ndimage = pytest.importorskip("scipy.ndimage")
    n = 15
    radii = np.array([0.0, 0.8, 1.7, 2.5, 4.0])
    lib = _random_lib(5, n, 9)
    f = interp.RegularGridInterpolator((radii, np.arange(n), np.arange(n)), lib, method="linear")
    rng = np.random.default_rng(10)
    for _ in range(12):
        x, y = rng.uniform(-2.8, 2.8, 2)
        r = np.hypot(x, y)
        if r > radii[-1]:
            continue
        pts = np.stack(np.meshgrid(np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 2)
        P = f(np.column_stack([np.full(len(pts), r), pts])).reshape(n, n)
        ref = ndimage.rotate(P, -np.degrees(np.arctan2(y, x)), reshape=False, order=1,
                             mode="grid-constant", cval=0.0)
        np.testing.assert_allclose(O.psf_column(lib, radii, x, y).reshape(n, n), ref,
                                   rtol=0, atol=1e-12)


def test_error_metric_floor_below_float32_normal_range():
    """Float32 results below FLT_MIN are subnormal: compared at 1e-5 * FLT_MIN absolute."""
    rel = O.bound_relative_error([2.0e-40, 1.0], [2.0001e-40, 1.0 + 1e-6], [2.0e-40, 1.0], floor=O.FLT_MIN)
    assert rel[0] == pytest.approx(1e-44 / O.FLT_MIN) and rel[0] < 1e-5
    assert rel[1] == pytest.approx(1e-6)
    assert O.bound_relative_error([1.0], [1.0], [0.0])[0] == 0.0
    assert np.isinf(O.bound_relative_error([1.0], [0.0], [0.0])[0])
