"""Seeded synthetic inputs for the BPFA inpainting hot path.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle's tests.  It draws frames and sampling masks and nothing else: it
holds none of the method's arithmetic (no patch geometry, no sampler, no
reconstruction).

Frames stand in for the paper's Z-contrast STEM images (Sec. "N-Dimensional
Inpainting" names STEM as the typical 2D target; the time-to-solution study of
Sec. "Time-To-Solution" uses square greyscale frames).  No real microscope data
is available, so the generator builds a hexagonal lattice of Gaussian atomic
columns, applies Poisson shot noise at a fixed mean dose and rescales to [0, 1].

Recipe (all NumPy ``default_rng(seed)``, PCG64):

* lattice: hexagonal, nearest-neighbour spacing ``spacing`` px (default 12),
  uniformly random sub-pixel origin;
* grains: ``grains=1`` gives one orientation; ``grains=2`` splits the frame at
  the vertical midline, the right grain rotated by ``boundary_deg`` (15 deg);
* columns: isotropic Gaussians with sigma ``sigma`` px (2), amplitudes
  U(0.3, 1.0) drawn per column;
* dose: clean intensity I scaled so the mean is ``dose`` e-/px (50);
  counts ~ Poisson(dose * I / mean(I)); frame = counts / max(counts); the clean
  reference is put on the same scale;
* masks: Bernoulli(frac) per pixel (``kind="random"``).

Spectrum images (``spectrum_cube``, the paper's spectral cubes in Sec.
"N-Dimensional Inpainting") are (H, W, C) cubes: at every pixel a smooth
decaying background plus Gaussian peaks at fixed channels, whose amplitudes
vary smoothly across the field of view (sums of a few random 2-D Gaussian
blobs), with Poisson noise at a mean dose and the same [0, 1] scaling.
"""
from __future__ import annotations

import numpy as np

__all__ = ["stem_frame", "random_mask", "line_hop_mask", "stem_volume", "spectrum_cube", "sparse_state"]


def _lattice_points(shape, spacing, theta, origin):
    """Hexagonal lattice points (y, x) covering ``shape`` rotated by theta."""
    h, w = shape
    a1 = np.array([1.0, 0.0]) * spacing
    a2 = np.array([0.5, np.sqrt(3.0) / 2.0]) * spacing
    rot = np.array([[np.cos(theta), -np.sin(theta)], [np.sin(theta), np.cos(theta)]])
    a1 = rot @ a1
    a2 = rot @ a2
    reach = int(np.ceil(1.5 * max(h, w) / spacing)) + 4
    ii, jj = np.meshgrid(np.arange(-reach, reach + 1), np.arange(-reach, reach + 1), indexing="ij")
    pts = ii.reshape(-1, 1) * a1 + jj.reshape(-1, 1) * a2 + origin
    # pts are (x, y); keep those within a margin of the frame
    m = 4.0 * spacing
    keep = (pts[:, 0] > -m) & (pts[:, 0] < w + m) & (pts[:, 1] > -m) & (pts[:, 1] < h + m)
    return pts[keep]


def stem_frame(shape=(128, 128), seed=0, *, spacing=12.0, sigma=2.0, grains=1,
               boundary_deg=15.0, dose=50.0, drift=(0.0, 0.0)):
    """Return ``(noisy, clean)`` float32 frames in [0, 1] (row-major, y then x).

    ``drift`` shifts the lattice origin by (dy, dx) pixels, used for frame
    sequences whose lattice moves between frames.
    """
    rng = np.random.default_rng(seed)
    h, w = shape
    origin = rng.uniform(0.0, spacing, size=2) + np.array([drift[1], drift[0]])
    yy, xx = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    intensity = np.zeros((h, w), dtype=np.float64)
    thetas = [0.0] if grains == 1 else [0.0, np.deg2rad(boundary_deg)]
    for g, theta in enumerate(thetas):
        pts = _lattice_points((h, w), spacing, theta, origin)
        amps = rng.uniform(0.3, 1.0, size=len(pts))
        if grains == 1:
            region = np.ones((h, w), dtype=bool)
        else:
            region = (xx < w / 2.0) if g == 0 else (xx >= w / 2.0)
        layer = np.zeros((h, w), dtype=np.float64)
        r = int(np.ceil(4 * sigma))
        for (px, py), amp in zip(pts, amps):
            x0, x1 = max(int(px) - r, 0), min(int(px) + r + 2, w)
            y0, y1 = max(int(py) - r, 0), min(int(py) + r + 2, h)
            if x0 >= x1 or y0 >= y1:
                continue
            dy = yy[y0:y1, x0:x1] - py
            dx = xx[y0:y1, x0:x1] - px
            layer[y0:y1, x0:x1] += amp * np.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))
        intensity += np.where(region, layer, 0.0)
    intensity += 1e-3  # keep every pixel's expected dose positive
    lam = dose * intensity / intensity.mean()
    counts = rng.poisson(lam).astype(np.float64)
    scale = max(counts.max(), 1.0)
    noisy = (counts / scale).astype(np.float32)
    clean = (lam / scale).astype(np.float32)
    return noisy, clean


def stem_volume(shape=(32, 64, 64), seed=0, *, drift_per_frame=0.3, **kw):
    """Stack of drifting lattice frames, shape (T, H, W), for 3D patches."""
    t, h, w = shape
    noisy = np.empty(shape, dtype=np.float32)
    clean = np.empty(shape, dtype=np.float32)
    for f in range(t):
        n, c = stem_frame((h, w), seed=seed, drift=(0.0, drift_per_frame * f), **kw)
        noisy[f], clean[f] = n, c
    return noisy, clean


def spectrum_cube(shape=(128, 128, 512), seed=0, *, peaks=6, width=6.0, dose=20.0):
    """Return ``(noisy, clean)`` float32 spectrum images of shape (H, W, C).

    Per pixel: background b(y, x) exp(-c / 200) plus ``peaks`` Gaussian peaks
    at channels drawn once (sigma ``width`` channels) with amplitude maps
    a_j(y, x); each map is a sum of 3 random Gaussian blobs.  Poisson noise at
    a mean of ``dose`` counts per voxel, scaled by the maximum count.
    """
    rng = np.random.default_rng(seed)
    h, w, nc = shape
    yy, xx = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")

    def blob_map():
        m = np.zeros((h, w))
        for _ in range(3):
            cy, cx = rng.uniform(0, h), rng.uniform(0, w)
            sy = rng.uniform(0.1, 0.4) * h
            m += rng.uniform(0.3, 1.0) * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * sy * sy))
        return m

    c = np.arange(nc, dtype=np.float64)
    intensity = (0.2 + 0.3 * blob_map())[:, :, None] * np.exp(-c / 200.0)[None, None, :]
    centers = rng.uniform(0.1 * nc, 0.9 * nc, size=peaks)
    for cj in centers:
        profile = np.exp(-((c - cj) ** 2) / (2.0 * width * width))
        intensity += blob_map()[:, :, None] * profile[None, None, :]
    intensity += 1e-3
    lam = dose * intensity / intensity.mean()
    counts = rng.poisson(lam).astype(np.float64)
    scale = max(counts.max(), 1.0)
    return (counts / scale).astype(np.float32), (lam / scale).astype(np.float32)


def random_mask(shape, frac, seed=0):
    """Bernoulli(frac) sampling mask as uint8 {0, 1} of the given shape."""
    rng = np.random.default_rng(seed + 0x5EED)
    return (rng.random(shape) < frac).astype(np.uint8)


def sparse_state(n_patches, P, K, seed=0, *, active=0.08, s_scale=0.5):
    """A random sampler state (D, Z, S) used as a common starting point.

    D is K x P with rows ~ N(0, I/P); Z is n_patches x K Bernoulli(active);
    S holds N(0, s_scale^2) weights where Z is set and 0 elsewhere.  All arrays
    are float32-representable so both implementations start from identical
    values.
    """
    rng = np.random.default_rng(seed + 0xD1C7)
    D = (rng.standard_normal((K, P)) / np.sqrt(P)).astype(np.float32)
    Z = (rng.random((n_patches, K)) < active).astype(np.uint8)
    S = (rng.standard_normal((n_patches, K)) * s_scale).astype(np.float32) * Z
    return D, Z, S.astype(np.float32)


def line_hop_mask(shape, frac, seed=0):
    """Line-hop sampling: in every band of h = round(1/frac) rows, each column
    keeps exactly one pixel, whose row inside the band follows a +-1 random
    walk along the columns, clamped to the band."""
    rng = np.random.default_rng(seed + 0x11E0)
    rows, cols = shape
    h = max(1, int(round(1.0 / frac)))
    mask = np.zeros(shape, dtype=np.uint8)
    for top in range(0, rows, h):
        band = min(h, rows - top)
        r = int(rng.integers(0, band))
        steps = rng.integers(-1, 2, size=cols)
        for c in range(cols):
            r = min(max(r + int(steps[c]), 0), band - 1)
            mask[top + r, c] = 1
    return mask
