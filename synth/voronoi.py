"""Seeded synthetic images shaped like the paper's inputs.

The paper's photographs (MRI scan, dog portraits; Section 3.2 and Section 4.2) are not
available, so every workload here is a synthetic piecewise-constant image: a Voronoi
partition with one colour per region, an optional smooth linear colour ramp, and
Gaussian noise clipped to [0, 1].  Grey-scale (C=1), RGB (C=3) and 31-band
"hyperspectral" images (smooth random spectra per region) are supported.

This module draws random numbers and nothing else: it holds none of the method's
arithmetic (no kernel, no dynamics, no cost), so both the FP64 oracle and the CUDA
path may use it to build identical inputs.

Draw order, from ``numpy.random.default_rng(seed)`` (PCG64):
  1. ``K`` site positions, uniform in [0, H) x [0, W) (rows, cols);
  2. region colours: U[0,1]^C, or for spectra 3 Gaussians per region;
  3. ramp: angle theta ~ U[0, 2 pi), then C gains g ~ U[-1, 1] (only if amplitude > 0);
  4. noise N(0, sigma^2) of shape (H, W, C) (only if sigma > 0).
Pixel (row, col) takes the nearest site to its centre (row + 1/2, col + 1/2); on equal
distance the lower site index wins.  The result is float64, clipped to [0, 1].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class ImageSpec:
    height: int
    width: int
    channels: int = 3
    regions: int = 4
    ramp: float = 0.0          # amplitude A of the linear colour ramp
    sigma: float = 0.05        # Gaussian noise standard deviation
    spectral: bool = False     # smooth random spectra per region (for many channels)


def voronoi_labels(height: int, width: int, sites: np.ndarray) -> np.ndarray:
    """Index of the nearest site for each pixel centre; ties go to the lower index."""
    rows = np.arange(height, dtype=np.float64)[:, None] + 0.5
    cols = np.arange(width, dtype=np.float64)[None, :] + 0.5
    best = np.full((height, width), np.inf)
    lab = np.zeros((height, width), dtype=np.int64)
    for k in range(sites.shape[0]):
        d = (rows - sites[k, 0]) ** 2 + (cols - sites[k, 1]) ** 2
        closer = d < best          # strict: an equal distance keeps the lower index
        best = np.where(closer, d, best)
        lab = np.where(closer, k, lab)
    return lab


def _spectra(rng: np.random.Generator, regions: int, channels: int) -> np.ndarray:
    """Smooth random spectra: per region a sum of 3 Gaussians over the band index,
    centres U[0, C-1], widths U[2, 8], heights U[0.2, 1], rescaled to a max U[0.3, 1]."""
    band = np.arange(channels, dtype=np.float64)
    out = np.empty((regions, channels))
    for k in range(regions):
        centres = rng.uniform(0.0, channels - 1.0, size=3)
        widths = rng.uniform(2.0, 8.0, size=3)
        heights = rng.uniform(0.2, 1.0, size=3)
        s = np.zeros(channels)
        for m in range(3):
            s += heights[m] * np.exp(-0.5 * ((band - centres[m]) / widths[m]) ** 2)
        peak = rng.uniform(0.3, 1.0)
        out[k] = s * (peak / s.max())
    return out


def make_image(spec: ImageSpec, seed: int) -> np.ndarray:
    """Return an (H, W, C) float64 image in [0, 1] for ``spec`` and ``seed``."""
    H, W, C = spec.height, spec.width, spec.channels
    if H < 1 or W < 1 or C < 1 or spec.regions < 1:
        raise ValueError("image sides, channels and regions must be >= 1")
    rng = np.random.default_rng(seed)
    sites = np.stack([rng.uniform(0.0, H, size=spec.regions),
                      rng.uniform(0.0, W, size=spec.regions)], axis=1)
    if spec.spectral:
        colours = _spectra(rng, spec.regions, C)
    else:
        colours = rng.uniform(0.0, 1.0, size=(spec.regions, C))
    img = colours[voronoi_labels(H, W, sites)]
    if spec.ramp > 0.0:
        theta = rng.uniform(0.0, 2.0 * np.pi)
        gains = rng.uniform(-1.0, 1.0, size=C)
        x = (np.arange(W, dtype=np.float64)[None, :] + 0.5) / W
        y = (np.arange(H, dtype=np.float64)[:, None] + 0.5) / H
        p = x * np.cos(theta) + y * np.sin(theta)
        span = p.max() - p.min()
        u = (p - p.min()) / span - 0.5 if span > 0 else np.zeros_like(p)
        img = img + spec.ramp * u[:, :, None] * gains[None, None, :]
    if spec.sigma > 0.0:
        img = img + rng.normal(0.0, spec.sigma, size=(H, W, C))
    return np.clip(img, 0.0, 1.0)


def make_image_f32(spec: ImageSpec, seed: int) -> np.ndarray:
    """The same image cast once to float32 (the CUDA path's storage type)."""
    return make_image(spec, seed).astype(np.float32)


# Workloads used by the tests and the benchmark, named by what they are.
PARITY_64_RGB = ImageSpec(64, 64, 3, regions=4, ramp=0.0, sigma=0.05)
THROUGHPUT_1024_RGB = ImageSpec(1024, 1024, 3, regions=12, ramp=0.1, sigma=0.08)
GRADIENT_2048_RGB = ImageSpec(2048, 2048, 3, regions=24, ramp=0.1, sigma=0.1)


def batch_specs(count: int, seed: int, lo: int = 128, hi: int = 1536):
    """Uneven batch: sides H ~ U{lo..hi}, aspect a ~ U[0.5, 2], W = round(H a); the
    first two thirds RGB (K ~ U{4..32}, ramp 0.1, sigma 0.08), the rest 31-band
    spectra (sigma 0.05); a window radius R ~ U{3..7} per image.
    Returns a list of (ImageSpec, image_seed, radius)."""
    rng = np.random.default_rng(seed)
    out = []
    n_rgb = (2 * count) // 3
    for b in range(count):
        H = int(rng.integers(lo, hi + 1))
        a = rng.uniform(0.5, 2.0)
        W = max(1, int(round(H * a)))
        R = int(rng.integers(3, 8))
        K = int(rng.integers(4, 33))
        if b < n_rgb:
            spec = ImageSpec(H, W, 3, regions=K, ramp=0.1, sigma=0.08)
        else:
            spec = ImageSpec(H, W, 31, regions=K, ramp=0.0, sigma=0.05, spectral=True)
        out.append((spec, seed * 1000 + b, R))
    return out
