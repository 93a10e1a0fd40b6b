"""Seeded synthetic grayscale images shaped like the paper's workloads.

The paper evaluates on natural 8-bit photographs that are not available here;
these generators stand in for them (piecewise-constant regions with sharp edges
plus noise, the structure an edge-preserving filter is meant for).  All images
are float32 in [0, 1].  This module holds input generation only: no step of the
filter's arithmetic lives here, so both the CUDA path and the CPU oracle can be
fed from it.

Recipes:

* ``blocks``  -- an 8 x 8 grid of constant blocks with levels ~ U[0, 1] plus
  N(0, noise^2) noise, clipped (default noise 0.05).
* ``shapes``  -- background level ~ U[0, 1]; ``n_objects`` axis-aligned rectangles
  and ``n_objects`` ellipses painted in turn (rectangle i, then ellipse i), centres
  uniform over the image, half-sizes ~ U[20, 300] * ``scale`` pixels, uniform
  intensity ~ U[0, 1]; plus N(0, noise^2), clipped (default noise 0.03).
* ``batch_sizes`` -- square sides ``round(exp(U[ln lo, ln hi]))``.
"""
from __future__ import annotations

import math

import numpy as np


def blocks(height: int, width: int, seed: int = 0, noise: float = 0.05, grid: int = 8) -> np.ndarray:
    rng = np.random.default_rng(seed)
    levels = rng.uniform(0.0, 1.0, (grid, grid))
    ys = np.minimum((np.arange(height) * grid) // max(height, 1), grid - 1)
    xs = np.minimum((np.arange(width) * grid) // max(width, 1), grid - 1)
    img = levels[ys[:, None], xs[None, :]]
    img = img + rng.normal(0.0, noise, (height, width))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def shapes(height: int, width: int, seed: int = 0, noise: float = 0.03, n_objects: int = 32,
           scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    img = np.full((height, width), rng.uniform(0.0, 1.0), dtype=np.float64)
    for _ in range(n_objects):
        for kind in (0, 1):
            cx, cy = rng.uniform(0, width), rng.uniform(0, height)
            ax, ay = rng.uniform(20.0, 300.0, 2) * scale
            val = rng.uniform(0.0, 1.0)
            x0, x1 = max(0, int(math.floor(cx - ax))), min(width, int(math.ceil(cx + ax)) + 1)
            y0, y1 = max(0, int(math.floor(cy - ay))), min(height, int(math.ceil(cy + ay)) + 1)
            if x0 >= x1 or y0 >= y1:
                continue
            yy = np.arange(y0, y1, dtype=np.float64)[:, None]
            xx = np.arange(x0, x1, dtype=np.float64)[None, :]
            if kind == 0:
                m = (np.abs(xx - cx) <= ax) & (np.abs(yy - cy) <= ay)
            else:
                m = ((xx - cx) / ax) ** 2 + ((yy - cy) / ay) ** 2 <= 1.0
            img[y0:y1, x0:x1][m] = val
    # noise in row chunks keeps peak host memory low for 8192^2 images
    out = np.empty((height, width), dtype=np.float32)
    step = max(1, (1 << 22) // max(width, 1))
    for r in range(0, height, step):
        blk = img[r:r + step] + rng.normal(0.0, noise, img[r:r + step].shape)
        out[r:r + step] = np.clip(blk, 0.0, 1.0)
    return out


def batch_sizes(n: int, lo: int, hi: int, seed: int = 1234) -> list[int]:
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(v))) for v in rng.uniform(math.log(lo), math.log(hi), n)]


def uniform(height: int, width: int, seed: int = 0) -> np.ndarray:
    """i.i.d. U[0, 1] pixels (worst case for edge structure; used in small tests)."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, (height, width)).astype(np.float32)
