"""Seeded synthetic inputs shaped like the paper's microscopy workloads.

The paper's own data (the Lena test image of Sec. 4.1 and the hippocampal
neuron SOFI movie of Sec. 4.4) are not available, so these generators stand in
for them.  This module holds none of the projection method's arithmetic: it
only draws images (Gaussian blobs, Poisson emitters blurred by a Gaussian PSF,
a high-pass residual normalised by sqrt of the mean).  Both the CUDA path and
the oracle consume its outputs; neither is imported here.

Every generator takes a seed and returns a float64 ``numpy`` array.  Seeds are
``numpy.random.default_rng(seed)``; defaults are 1000 + workload number.
"""
from __future__ import annotations

import numpy as np


def _gaussian_field(H, W, centers, sigma, amplitude, background=0.0):
    """background + sum_k amplitude * exp(-|r - r_k|^2 / (2 sigma^2)), evaluated
    exactly within 6 sigma of each centre (the tail beyond is < 1.6e-8 of the peak)."""
    f = np.full((H, W), float(background))
    rad = int(np.ceil(6 * sigma))
    for (cy, cx) in centers:
        r0, r1 = max(0, int(cy) - rad), min(H, int(cy) + rad + 2)
        c0, c1 = max(0, int(cx) - rad), min(W, int(cx) + rad + 2)
        if r0 >= r1 or c0 >= c1:
            continue
        rr = np.arange(r0, r1)[:, None] - cy
        cc = np.arange(c0, c1)[None, :] - cx
        f[r0:r1, c0:c1] += amplitude * np.exp(-(rr * rr + cc * cc) / (2.0 * sigma * sigma))
    return f


def blobs_residual(H=64, W=64, n_blobs=5, sigma=2.0, amplitude=6.0, seed=1001):
    """iid N(0,1) noise plus ``n_blobs`` Gaussian blobs (sigma 2 px, amplitude 6)
    centred uniformly in [m, H-m) x [m, W-m), m = min(4, H/4, W/4).  Default:
    the 64 x 64 workload (centres in [4, 60)^2)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((H, W))
    m = min(4.0, H / 4.0, W / 4.0)
    cy = rng.uniform(m, H - m, size=n_blobs)
    cx = rng.uniform(m, W - m, size=n_blobs)
    return x + _gaussian_field(H, W, list(zip(cy, cx)), sigma, amplitude)


def _smooth(y, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(y, sigma, mode="reflect")


def emitter_residual(H=512, W=512, n_emitters=400, psf_sigma=2.0, peak=100.0,
                     background=10.0, smooth_sigma=4.0, seed=1002):
    """Widefield-microscopy-like residual.

    Field = background + sum_k peak * exp(-|r - r_k|^2 / (2 psf_sigma^2)) over
    ``n_emitters`` uniformly placed point emitters (peak mean 100 photons over
    a background of 10); y ~ Poisson(field); residual = (y - G_{smooth_sigma} * y)
    / sqrt(mean y).  Default: the 512 x 512 workload with 400 emitters.
    """
    rng = np.random.default_rng(seed)
    cy = rng.uniform(0, H, size=n_emitters)
    cx = rng.uniform(0, W, size=n_emitters)
    field = _gaussian_field(H, W, list(zip(cy, cx)), psf_sigma, peak, background)
    y = rng.poisson(field).astype(np.float64)
    return (y - _smooth(y, smooth_sigma)) / np.sqrt(y.mean())


def emitter_residual_2048(seed=1003):
    """2048 x 2048 residual with 1600 emitters (same recipe as the 512 x 512 one)."""
    return emitter_residual(2048, 2048, n_emitters=1600, seed=seed)


def batch_shapes(n=256, seed=1004):
    """Image shapes of the uneven batch: side s uniform in {128,...,1024}; with
    probability 0.5 the image is s x 2s, else s x s."""
    rng = np.random.default_rng(seed)
    sides = rng.choice([128, 256, 384, 512, 768, 1024], size=n)
    rect = rng.random(n) < 0.5
    return [(int(s), int(2 * s) if r else int(s)) for s, r in zip(sides, rect)]


def batch_images(n=256, seed=1004):
    """Residuals of the uneven batch, emitter density 400 per 512^2."""
    out = []
    for idx, (H, W) in enumerate(batch_shapes(n, seed)):
        ne = max(1, int(round(400 * H * W / (512 * 512))))
        out.append(emitter_residual(H, W, n_emitters=ne, seed=seed * 7919 + idx))
    return out


def sofi_like(side=256, frames=200, density=20, on_prob=0.3, psf_sigma=1.5, peak=100.0,
              background=10.0, seed=1005):
    """Second-order-cumulant-like image: pixelwise variance over ``frames``
    frames of blinking emitters (``density`` per 64 x 64 area, each on with
    probability ``on_prob`` per frame), Gaussian PSF, Poisson noise; then the
    high-pass residual of ``emitter_residual`` normalised by its global std."""
    rng = np.random.default_rng(seed)
    ne = max(1, int(round(density * side * side / (64 * 64))))
    cy = rng.uniform(0, side, size=ne)
    cx = rng.uniform(0, side, size=ne)
    psf = [_gaussian_field(side, side, [(y, x)], psf_sigma, peak) for y, x in zip(cy, cx)]
    psf = np.stack(psf) if ne else np.zeros((0, side, side))
    s1 = np.zeros((side, side))
    s2 = np.zeros((side, side))
    for _ in range(frames):
        on = rng.random(ne) < on_prob
        f = background + np.tensordot(on.astype(np.float64), psf, axes=1)
        y = rng.poisson(f).astype(np.float64)
        s1 += y
        s2 += y * y
    var = s2 / frames - (s1 / frames) ** 2
    r = var - _smooth(var, 4.0)
    return r / r.std()


def sofi_tile(side=512, frames=200, density=20, on_prob=0.3, psf_sigma=1.5, peak=100.0,
              background=10.0, seed=1005):
    """The same second-order-cumulant-like residual as ``sofi_like`` for larger
    sides: every emitter's PSF (exact within 6 sigma) is a column of a sparse
    pixel x emitter matrix, so a frame is one sparse product."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    ne = max(1, int(round(density * side * side / (64 * 64))))
    cy = rng.uniform(0, side, size=ne)
    cx = rng.uniform(0, side, size=ne)
    rad = int(np.ceil(6 * psf_sigma))
    d = np.arange(-rad, rad + 2)
    rows, cols, vals = [], [], []
    for k in range(ne):
        yy = int(cy[k]) + d
        xx = int(cx[k]) + d
        yy = yy[(yy >= 0) & (yy < side)]
        xx = xx[(xx >= 0) & (xx < side)]
        g = peak * np.exp(-((yy[:, None] - cy[k]) ** 2 + (xx[None, :] - cx[k]) ** 2)
                          / (2.0 * psf_sigma * psf_sigma))
        idx = (yy[:, None] * side + xx[None, :]).ravel()
        rows.append(idx)
        cols.append(np.full(idx.size, k))
        vals.append(g.ravel())
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(side * side, ne))
    s1 = np.zeros(side * side)
    s2 = np.zeros(side * side)
    for _ in range(frames):
        on = (rng.random(ne) < on_prob).astype(np.float64)
        y = rng.poisson(background + M @ on).astype(np.float64)
        s1 += y
        s2 += y * y
    var = (s2 / frames - (s1 / frames) ** 2).reshape(side, side)
    r = var - _smooth(var, 4.0)
    return r / r.std()


def sofi_canvas(side=2048, tile=512, n_tiles=2, seed=1005):
    """A ``side`` x ``side`` SOFI-like residual assembled from ``n_tiles``
    independently drawn ``sofi_tile`` tiles, each placement flipped and
    transposed at random (the statistics are local, so the mosaic keeps them);
    requests of the serving workload are crops of it."""
    rng = np.random.default_rng(seed)
    tiles = [sofi_tile(tile, seed=seed + 17 * k) for k in range(n_tiles)]
    out = np.empty((side, side))
    for ty in range(0, side, tile):
        for tx in range(0, side, tile):
            t = tiles[rng.integers(n_tiles)]
            if rng.random() < 0.5:
                t = t.T
            if rng.random() < 0.5:
                t = t[::-1]
            if rng.random() < 0.5:
                t = t[:, ::-1]
            h, w = min(tile, side - ty), min(tile, side - tx)
            out[ty:ty + h, tx:tx + w] = t[:h, :w]
    return out


def request_image(canvas, side, seed):
    """A ``side`` x ``side`` request cropped from ``canvas`` at a seeded offset,
    normalised by its own standard deviation."""
    rng = np.random.default_rng(seed)
    H, W = canvas.shape
    y0 = int(rng.integers(0, H - side + 1))
    x0 = int(rng.integers(0, W - side + 1))
    c = canvas[y0:y0 + side, x0:x0 + side]
    return c / c.std()


def request_stream(n=2000, rate=500.0, seed=1006):
    """Poisson arrivals (mean ``rate`` per second) of square requests with side
    uniform in 64..2048: list of (arrival_time_s, side, seed)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    sides = rng.integers(64, 2049, size=n)
    return [(float(a), int(s), int(seed * 104729 + i)) for i, (a, s) in enumerate(zip(t, sides))]


def random_image(H, W, scale=2.0, seed=0):
    """iid N(0, scale^2) test image."""
    return np.random.default_rng(seed).standard_normal((H, W)) * scale
