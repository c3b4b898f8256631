"""Oracle for LSH keyword generation (Sec. 4.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Points are float32
rows (n x dim); hash function i of m maps a point to keyword i * D + bucket.

  * ``pstable``  -- Eqn. (plsh): floor((a_i . p + b_i) / w) mod D, the dot
                    product accumulated by fused multiply-adds in dimension
                    order, every operation in binary32 (C++).
  * ``rbh``      -- random binning for the Laplacian kernel (Sec. 4.1.3): the
                    point's grid cell floor((p - u_i) / g_i), re-hashed into D
                    buckets (Sec. 4.1.2) by the lowbias32 finalizer (C++).
  * ``pstable_collision`` -- Datar et al.'s collision probability of one
                    p-stable function for two points at l2 distance delta.
"""
from __future__ import annotations

import math

import numpy as np

from . import _c, _lib, _p


def pstable(points, a, b, w: float, D: int) -> np.ndarray:
    pts, a, b = _c(points, np.float32), _c(a, np.float32), _c(b, np.float32)
    n, dim = pts.shape
    m = a.shape[0]
    kw = np.empty((n, m), np.uint32)
    if _lib().oracle_lsh_pstable(n, dim, _p(pts), m, _p(a), _p(b), w, D, _p(kw)) != 0:
        raise ValueError("bad LSH parameters")
    return kw


def rbh(points, g, u, key, D: int) -> np.ndarray:
    pts, g, u, key = _c(points, np.float32), _c(g, np.float32), _c(u, np.float32), \
        _c(key, np.uint32)
    n, dim = pts.shape
    m = g.shape[0]
    kw = np.empty((n, m), np.uint32)
    if _lib().oracle_lsh_rbh(n, dim, _p(pts), m, _p(g), _p(u), _p(key), D, _p(kw)) != 0:
        raise ValueError("bad LSH parameters")
    return kw


def pstable_collision(delta: float, w: float) -> float:
    """Pr[h(p) = h(q)] for ||p - q||_2 = delta (Datar et al.; the paper's
    equation after Eqn. (plsh)): with r = w / delta,
    1 - 2 Phi(-r) - 2 / (sqrt(2 pi) r) (1 - exp(-r^2 / 2))."""
    r = w / delta
    phi = 0.5 * math.erfc(r / math.sqrt(2.0))  # Phi(-r)
    return 1.0 - 2.0 * phi - 2.0 / (math.sqrt(2.0 * math.pi) * r) * (1.0 - math.exp(-r * r / 2.0))
