"""Sanity of the seeded synthetic inputs (CPU only): shapes, seeding, core positions."""
import numpy as np

from synth import lyot, scenes, workloads


def test_lyot_cores_sit_at_their_offsets_and_are_seeded():
    radii = np.array([0.0, 4.0, 8.0])
    L = lyot.psf_library(radii, 48, 0.5, seed=1)
    assert L.shape == (3, 48, 48) and np.all(L >= 0.0)
    c = (48 - 1) / 2
    for k in (1, 2):
        p, q = np.unravel_index(np.argmax(L[k]), L[k].shape)
        assert abs(q - (c + radii[k] / 0.5)) <= 1.0 and abs(p - c) <= 1.0
    assert L[0].max() < 0.05 * L[2].max()           # on-axis light is suppressed
    assert np.array_equal(L, lyot.psf_library(radii, 48, 0.5, seed=1))
    assert not np.array_equal(L, lyot.psf_library(radii, 48, 0.5, seed=2))


def test_scene_batch_is_seeded_and_masked():
    w = workloads.plain_small()
    a = workloads.scene_batch(w, 3)
    assert a.shape == (3, w.K) and np.array_equal(a, workloads.scene_batch(w, 3))
    X, Y = scenes.pixel_centres(w.N, w.S)
    assert not np.any(a[:, (np.hypot(X, Y) > w.r_max).ravel()])
