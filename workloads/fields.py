"""Wave-speed fields and sources evaluated at caller-supplied coordinates.

Shapes follow the paper's workloads: Gaussian point sources, a Y-shaped
waveguide with 3x wave-speed contrast (Fig. 1), and smooth random media.
"""

from __future__ import annotations

import math

import numpy as np


def gaussian_source(X, Y, center, width):
    """Unit-mass Gaussian exp(-|x-x0|^2 / (2 w^2)) / (2 pi w^2)."""
    r2 = (X - center[0]) ** 2 + (Y - center[1]) ** 2
    return np.exp(-r2 / (2.0 * width * width)) / (2.0 * math.pi * width * width)


def _dist_to_segment(X, Y, a, b):
    ax, ay = a
    bx, by = b
    dx, dy = bx - ax, by - ay
    t = ((X - ax) * dx + (Y - ay) * dy) / (dx * dx + dy * dy)
    t = np.clip(t, 0.0, 1.0)
    return np.hypot(X - (ax + t * dx), Y - (ay + t * dy))


Y_SEGMENTS = (((0.5, 0.0), (0.5, 0.5)), ((0.5, 0.5), (0.2, 1.0)), ((0.5, 0.5), (0.8, 1.0)))


def y_channel_speed(X, Y, width=0.08, c_in=1.0 / 3.0, c_out=1.0, segments=Y_SEGMENTS):
    """Y-shaped channel: nodes within width/2 of the stem or either arm get
    c_in, all others c_out (unit-square coordinates)."""
    d = np.full(np.shape(X), np.inf)
    for a, b in segments:
        d = np.minimum(d, _dist_to_segment(X, Y, a, b))
    return np.where(d <= width / 2.0, c_in, c_out)


def random_field(gx, gy, corr_len, seed, n_modes=256):
    """Stationary Gaussian-covariance random field (mean 0, variance 1) by a
    random-phase spectral sum, g(x,y) = sqrt(2/K) sum_k cos(kx x + ky y + phi_k)
    with (kx, ky) ~ N(0, 1/corr_len^2).  Evaluated on the tensor grid
    gx (NX,) x gy (NY,) as a (NY, NX) array via a product of 1D factors."""
    rng = np.random.default_rng(seed)
    kx = rng.standard_normal(n_modes) / corr_len
    ky = rng.standard_normal(n_modes) / corr_len
    ph = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    ax = np.asarray(gx, dtype=float)[None, :] * kx[:, None] + ph[:, None]  # (K, NX)
    ay = np.asarray(gy, dtype=float)[:, None] * ky[None, :]  # (NY, K)
    # cos(a + b) = cos a cos b - sin a sin b
    left = np.concatenate([np.cos(ay), -np.sin(ay)], axis=1)  # (NY, 2K)
    right = np.concatenate([np.cos(ax), np.sin(ax)], axis=0)  # (2K, NX)
    return math.sqrt(2.0 / n_modes) * (left @ right)


def random_speed(gx, gy, corr_len=0.05, seed=3, amp=0.5, clip=1.5):
    """c = 1 + amp * clip(g, -clip, clip) for the random field g above."""
    g = np.clip(random_field(gx, gy, corr_len, seed), -clip, clip)
    return 1.0 + amp * g


def warp_nodes(X, Y, box, amp):
    """Smooth interior distortion of a node grid on the rectangle box =
    (x0, x1, y0, y1): with s, t the normalised coordinates in [0, 1],
      x += amp (x1 - x0) sin(2 pi s) sin(pi t),  y += amp (y1 - y0) sin(pi s) sin(2 pi t).
    Boundary nodes stay on their edges (both terms vanish there), so outer
    normals and edge data are those of the rectangle; the elements become
    curved quadrilaterals (orientation kept for amp < 1 / (2 pi (1 + pi/2))).
    """
    x0, x1, y0, y1 = box
    s = (np.asarray(X) - x0) / (x1 - x0)
    t = (np.asarray(Y) - y0) / (y1 - y0)
    Xw = X + amp * (x1 - x0) * np.sin(2 * math.pi * s) * np.sin(math.pi * t)
    Yw = Y + amp * (y1 - y0) * np.sin(math.pi * s) * np.sin(2 * math.pi * t)
    return Xw, Yw
