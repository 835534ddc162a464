"""The five named synthetic workloads (input preparation only).

Shapes follow the paper's use: n x n PSFs at s lambda/D per pixel applied to an
N x N scene at S lambda/D per pixel, A being n^2 x N^2 (Sec. 3).  Seeds are
2106 + workload index; scene b of a batch uses seed + 1000 * (b + 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import lyot, scenes

BASE_SEED = 2106


@dataclass
class Workload:
    name: str
    n: int
    s: float
    N: int
    S: float
    radii: np.ndarray
    binning: int = 1
    r_max: float = 0.0
    seed: int = BASE_SEED
    lam_ratios: tuple = (1.0,)
    extra: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return self.n * self.n

    @property
    def K(self) -> int:
        return self.N * self.N

    def library(self, lam_index: int = 0) -> np.ndarray:
        return lyot.psf_library(self.radii, self.n, self.s, self.seed,
                                self.lam_ratios[lam_index], self.binning)


def plain_small() -> Workload:
    """20 PSFs at 0..9.5 lambda/D, 64 x 64 at 0.5 lambda/D; one 64 x 64 scene."""
    return Workload("plain_small_64", 64, 0.5, 64, 0.5, np.arange(20) * 0.5, binning=2,
                    r_max=9.5, seed=BASE_SEED + 1)


def adjoint_128() -> Workload:
    """40 PSFs at 0..12 lambda/D, 128 x 128 at 0.25 lambda/D; ring fit workload."""
    return Workload("adjoint_fit_128", 128, 0.25, 128, 0.25, np.linspace(0.0, 12.0, 40),
                    r_max=12.0, seed=BASE_SEED + 2,
                    extra={"truth": (5.0, 1.0, np.deg2rad(60.0), 0.3, 1e-9), "sigma": 1e-11,
                           "steps": 200})


def batched_256() -> Workload:
    """60 PSFs, 256 x 256 at 0.125 lambda/D; 8 wavelengths x 64 scenes."""
    lams = tuple(1.0 + np.linspace(-0.05, 0.05, 8))
    return Workload("batched_split_bf16_256", 256, 0.125, 256, 0.125, np.linspace(0.0, 12.0, 60),
                    r_max=12.0, seed=BASE_SEED + 3, lam_ratios=lams, extra={"scenes": 64})


def fused_512() -> Workload:
    """80 PSFs, 512 x 512 at 0.0625 lambda/D; 32 two-ring scenes; A never stored."""
    return Workload("fused_512", 512, 0.0625, 512, 0.0625, np.linspace(0.0, 12.0, 80),
                    r_max=12.0, seed=BASE_SEED + 4, extra={"scenes": 32})


def ipac_shape() -> Workload:
    """The paper's IPAC geometry (Sec. 2, Eq. 1): 85 PSFs of 128^2 at 0.2 lambda/D with offsets
    sampled every 0.06 lambda/D to 4, 0.5 to 9 and 0.25 to 11 lambda/D; a 256^2 scene at
    3.529 mas = 0.0703 lambda/D per pixel (A = 16384 x 65536)."""
    radii = np.unique(np.round(np.concatenate([np.arange(0.0, 4.0, 0.06), np.arange(4.0, 9.0, 0.5),
                                               np.arange(9.0, 11.0001, 0.25)]), 6))
    mas_per_ld = 575e-9 / 2.3631 * 180.0 / np.pi * 3600e3
    return Workload("ipac_shape_128_to_256", 128, 0.2, 256, 3.529 / mas_per_ld, radii, r_max=9.0,
                    seed=BASE_SEED + 6)


def powerlaw_disk_scene(N: int, S: float, r_max: float, alpha: float = 1.34, r_in: float = 0.5) -> np.ndarray:
    """Smooth face-on dust disk with surface brightness ~ r^-alpha (the ZODIPIC default alpha of
    Sec. 2), 1e-9 at 1 lambda/D, masked beyond r_max and inside r_in."""
    X, Y = scenes.pixel_centres(N, S)
    r = np.hypot(X, Y)
    img = 1e-9 * np.power(np.maximum(r, r_in), -alpha)
    img[(r > r_max) | (r < r_in)] = 0.0
    return img


def uneven_buckets() -> list[tuple[int, float]]:
    return [(N, S) for N in (64, 96, 128, 192, 256) for S in (0.3, 0.5)]


def uneven_arrivals(count: int = 500, wave: int = 50, seed: int = BASE_SEED + 2 + 9):
    """Seeded arrival order of the uneven workload's scenes (one (N, S) bucket each), its waves
    of `wave` scenes, and the per-bucket capacity a wave needs (the most scenes any wave holds
    of one bucket)."""
    buckets = uneven_buckets()
    rng = np.random.default_rng(seed)
    order = [buckets[i] for i in rng.integers(0, len(buckets), count)]
    waves = [order[i:i + wave] for i in range(0, len(order), wave)]
    cap = max(max(wv.count(k) for k in buckets) for wv in waves)
    return order, waves, cap


def plain_small_scene(w: Workload) -> np.ndarray:
    img = scenes.ring_image(w.N, w.S, 5.0, 1.0, np.deg2rad(60.0), 0.3, 1e-9, w.r_max)
    rng = np.random.default_rng(w.seed)
    scenes.add_planets(img, w.S, rng, 2, 1e-8, 1e-8, log_uniform=False)
    return img


def random_ring_scene(N: int, S: float, r_max: float, seed: int, planets: bool = True) -> np.ndarray:
    """Seeded ring: R~U(3,9), i~U(0,80 deg), g~U(0,0.6), w=1, B=1e-9; 0-4 planets 1e-9..1e-7."""
    rng = np.random.default_rng(seed)
    R = rng.uniform(3.0, 9.0)
    inc = np.deg2rad(rng.uniform(0.0, 80.0))
    g = rng.uniform(0.0, 0.6)
    img = scenes.ring_image(N, S, R, 1.0, inc, g, 1e-9, r_max)
    if planets:
        scenes.add_planets(img, S, rng, int(rng.integers(0, 5)), 1e-9, 1e-7)
    return img


def two_ring_scene(N: int, S: float, r_max: float, seed: int) -> np.ndarray:
    """Inclined ring R~U(3,6) plus an outer ring at 2R (fused workload)."""
    rng = np.random.default_rng(seed)
    R = rng.uniform(3.0, 6.0)
    inc = np.deg2rad(rng.uniform(0.0, 80.0))
    g = rng.uniform(0.0, 0.6)
    img = scenes.ring_image(N, S, R, 1.0, inc, g, 1e-9, r_max)
    img += scenes.ring_image(N, S, 2.0 * R, 1.0, inc, g, 0.3e-9, r_max)
    return img


def scene_batch(w: Workload, count: int, kind: str = "ring") -> np.ndarray:
    out = np.empty((count, w.K), dtype=np.float64)
    for b in range(count):
        seed = w.seed + 1000 * (b + 1)
        img = two_ring_scene(w.N, w.S, w.r_max, seed) if kind == "two_ring" else \
            random_ring_scene(w.N, w.S, w.r_max, seed)
        out[b] = img.ravel()
    return out


def fit_target_noise(w: Workload, M: int) -> np.ndarray:
    """Seeded Gaussian noise (sigma) added to the fit's target image."""
    rng = np.random.default_rng(w.seed + 7)
    return rng.standard_normal(M) * w.extra["sigma"]


def fit_init(w: Workload) -> np.ndarray:
    """Seeded perturbation of the truth used as the fit's starting point."""
    rng = np.random.default_rng(w.seed + 11)
    R, wd, inc, g, B = w.extra["truth"]
    return np.array([R + rng.uniform(-0.4, 0.4), wd * rng.uniform(0.8, 1.25),
                     inc + np.deg2rad(rng.uniform(-6.0, 6.0)), g + rng.uniform(-0.1, 0.1),
                     B * rng.uniform(0.7, 1.4)])
