"""Seeded synthetic test images shaped like the paper's test set.

The paper evaluates on USC-SIPI, DIBCO and DIV2K images, none of which ships
here; these generators stand in for them.  This module holds no encoder
arithmetic: it only draws pixels, so both the CUDA library's tests and the
FP64 oracle's tests can be fed from it.  Every image is a pure function of
its seed (numpy PCG64), returned as a 2-D uint8 array.

``gradient_scene`` -- a linear gradient, two step edges of height 60, a disk
of radius 12 (per 64 pixels of the short side) and Gaussian noise, sigma 2:
the 64x64 parity case.

``piecewise_scene`` -- piecewise-planar regions (a Voronoi partition of 8
seeds, each with its own plane), 20 straight step edges of random height
20..60, one 128x128 band-limited texture patch (16 sinusoids, frequencies at
most 0.25 cycles/pixel, RMS amplitude 20) and Gaussian noise, sigma 3: the
512x512 throughput case.

Intensities not fixed by the workload description (gradient range, plane
slopes, texture amplitude) are choices of this module and are stated above.
"""
from __future__ import annotations

import numpy as np


def _finish(img: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def gradient_scene(h: int = 64, w: int = 64, seed: int = 0, noise: float = 2.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    img = 40.0 + 120.0 * (xx / w + yy / h) / 2.0
    x0 = rng.uniform(0.25 * w, 0.75 * w)
    y0 = rng.uniform(0.25 * h, 0.75 * h)
    img += np.where(xx >= x0, 60.0, 0.0)
    img -= np.where(yy >= y0, 60.0, 0.0)
    rad = 12.0 * min(h, w) / 64.0
    cy, cx = rng.uniform(0, h), rng.uniform(0, w)
    img += np.where((yy - cy) ** 2 + (xx - cx) ** 2 <= rad * rad, 80.0, 0.0)
    img += rng.normal(0.0, noise, size=(h, w))
    return _finish(img)


def piecewise_scene(h: int = 512, w: int = 512, seed: int = 0, noise: float = 3.0,
                    n_regions: int = 8, n_edges: int = 20, patch: int = 128) -> np.ndarray:
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    # Voronoi partition, one plane per region
    sy = rng.uniform(0, h, n_regions)
    sx = rng.uniform(0, w, n_regions)
    base = rng.uniform(50.0, 200.0, n_regions)
    gy = rng.uniform(-0.15, 0.15, n_regions)
    gx = rng.uniform(-0.15, 0.15, n_regions)
    d2 = (yy[None] - sy[:, None, None]) ** 2 + (xx[None] - sx[:, None, None]) ** 2
    region = np.argmin(d2, axis=0)
    img = (base[region] + gy[region] * (yy - sy[region]) + gx[region] * (xx - sx[region]))
    # straight step edges
    for _ in range(n_edges):
        py, px = rng.uniform(0, h), rng.uniform(0, w)
        th = rng.uniform(0, np.pi)
        hgt = rng.uniform(20.0, 60.0) * rng.choice([-1.0, 1.0])
        side = (yy - py) * np.cos(th) - (xx - px) * np.sin(th) >= 0
        img += np.where(side, hgt, 0.0)
    # band-limited texture patch
    ty = int(rng.integers(0, max(1, h - patch + 1)))
    tx = int(rng.integers(0, max(1, w - patch + 1)))
    ph, pw = min(patch, h), min(patch, w)
    py_, px_ = np.mgrid[0:ph, 0:pw].astype(np.float64)
    tex = np.zeros((ph, pw))
    for _ in range(16):
        fr = rng.uniform(0.02, 0.25)
        an = rng.uniform(0, 2 * np.pi)
        phs = rng.uniform(0, 2 * np.pi)
        tex += np.cos(2 * np.pi * fr * (np.cos(an) * px_ + np.sin(an) * py_) + phs)
    tex *= 20.0 / np.sqrt(8.0)          # RMS 20 for 16 unit cosines
    img[ty:ty + ph, tx:tx + pw] += tex
    img += rng.normal(0.0, noise, size=(h, w))
    return _finish(img)


def uniform_plane(h: int, w: int, value: int) -> np.ndarray:
    return np.full((h, w), value, np.uint8)


def noise_plane(h: int, w: int, seed: int = 0, mean: float = 128.0, sigma: float = 40.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _finish(rng.normal(mean, sigma, size=(h, w)))


def uneven_sizes(n_images: int, seed: int = 0, wmin: int = 256, wmax: int = 2048,
                 hmin: int = 256, hmax: int = 1536, step: int = 64):
    """(h, w) of the `n_images` images of an uneven batch: width and height
    drawn uniformly from the multiples of `step` in [wmin, wmax] x [hmin,
    hmax], image by image from one PCG64 stream seeded with `seed`."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_images):
        w = int(rng.integers(wmin // step, wmax // step + 1)) * step
        h = int(rng.integers(hmin // step, hmax // step + 1)) * step
        out.append((h, w))
    return out


def uneven_rgb_batch(n_images: int = 64, seed: int = 0, wmin: int = 256, wmax: int = 2048,
                     hmin: int = 256, hmax: int = 1536, step: int = 64, scene=None, first: int = 0,
                     count: int | None = None):
    """RGB images of uneven sizes (``uneven_sizes``); channel c of image i is
    ``scene(h, w, seed=seed + 3 i + c)`` -- the piecewise scene (the 512x512
    workload's generator) unless another scene is given, e.g.
    ``gradient_scene``.  Only images [first, first + count) of the
    `n_images`-image batch are drawn (a shard of it; the sizes of the others
    are still consumed from the stream, so a shard is the same images as in
    the whole batch).  Returns a list of (h, w, [R, G, B]) tuples."""
    make = scene or piecewise_scene
    sizes = uneven_sizes(n_images, seed, wmin, wmax, hmin, hmax, step)
    last = n_images if count is None else min(n_images, first + count)
    return [(h, w, [make(h, w, seed=seed + 3 * i + c) for c in range(3)])
            for i, (h, w) in enumerate(sizes) if first <= i < last]
