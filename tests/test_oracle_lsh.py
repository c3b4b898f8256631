"""Pins of the LSH keyword oracle (Sec. 4.1): the binary32 p-stable hash
agrees with the real-number definition away from bucket boundaries, and both
families collide at the rates the paper states (Datar et al.'s formula for
p-stable hashing; the Laplacian kernel for random binning) (CPU only)."""
import math

import numpy as np

import synth
from oracle import lsh


def _points(n, dim=128, config=2):
    _, v, _ = synth.lsh_keywords(n, config, 1, dim=dim, n_hash=1, want_vectors=True)
    return v


def test_pstable_matches_the_real_number_hash_away_from_boundaries():
    pts = _points(2000)
    pp = synth.lsh_params("pstable", 128, 64, 4.0, config=3)
    kw = lsh.pstable(pts, pp["a"], pp["b"], 4.0, 8192)
    s = pts.astype(np.float64) @ pp["a"].astype(np.float64).T + pp["b"].astype(np.float64)
    t = s / 4.0
    h = np.floor(t).astype(np.int64)
    want = (np.arange(64)[None, :] * 8192 + np.mod(h, 8192)).astype(np.uint32)
    diff = kw != want
    assert diff.mean() < 1e-3
    frac = t - np.round(t)
    assert np.all(np.abs(frac[diff]) < 1e-3)  # only at a bucket boundary
    for i in range(64):
        assert np.all((kw[:, i] >= i * 8192) & (kw[:, i] < (i + 1) * 8192))


def test_pstable_collision_rate_follows_datar_et_al():
    rng = np.random.default_rng(4)
    n, dim, m, w, D = 300, 64, 256, 4.0, 1 << 24
    pp = synth.lsh_params("pstable", dim, m, w, config=4)
    p = rng.standard_normal((n, dim)).astype(np.float32) * 3
    for delta in (0.5, 2.0, 4.0, 8.0):
        d = rng.standard_normal((n, dim))
        d = d / np.linalg.norm(d, axis=1, keepdims=True) * delta
        q = (p + d).astype(np.float32)
        rate = (lsh.pstable(p, pp["a"], pp["b"], w, D) == lsh.pstable(q, pp["a"], pp["b"], w, D)).mean()
        assert abs(rate - lsh.pstable_collision(delta, w)) < 0.02, delta


def test_random_binning_collides_at_the_laplacian_kernel():
    rng = np.random.default_rng(5)
    n, dim, m, sigma, D = 300, 32, 256, 10.0, 1 << 24
    rp = synth.lsh_params("rbh", dim, m, sigma, config=5)
    p = (rng.random((n, dim)) * 50).astype(np.float32)
    for l1 in (1.0, 5.0, 10.0, 20.0):
        d = rng.standard_normal((n, dim))
        d = d / np.abs(d).sum(axis=1, keepdims=True) * l1
        q = (p + d).astype(np.float32)
        rate = (lsh.rbh(p, rp["g"], rp["u"], rp["key"], D) ==
                lsh.rbh(q, rp["g"], rp["u"], rp["key"], D)).mean()
        assert abs(rate - math.exp(-l1 / sigma)) < 0.03, l1


def test_random_binning_keywords_are_deterministic_and_in_range():
    rng = np.random.default_rng(6)
    rp = synth.lsh_params("rbh", 16, 32, 5.0, config=6)
    p = (rng.random((100, 16)) * 20).astype(np.float32)
    a = lsh.rbh(p, rp["g"], rp["u"], rp["key"], 8192)
    b = lsh.rbh(p.copy(), rp["g"], rp["u"], rp["key"], 8192)
    assert np.array_equal(a, b)
    for i in range(32):
        assert np.all((a[:, i] >= i * 8192) & (a[:, i] < (i + 1) * 8192))
    # moving a point within all of its cells keeps its keywords
    cell_lo = np.floor((p[:, None, :] - rp["u"][None]) / rp["g"][None]) * rp["g"][None] + rp["u"][None]
    inside = p[:, None, :] - cell_lo  # distance to each cell's lower edge, >= 0
    eps = np.minimum(inside.min(axis=1), 1e-3) * 0.5
    c = lsh.rbh((p - eps).astype(np.float32), rp["g"], rp["u"], rp["key"], 8192)
    assert (c == a).mean() > 0.99
