"""Seeded synthetic inputs shaped like the paper's workloads (numpy PCG64 only).

The paper measures on SIFT1M, DEEP1M and GIST1M (Sec 4.1).  Those datasets are
not available here, so every workload is synthetic with the same shape and a
stated distribution.  This module holds none of the method's arithmetic: it
only draws points and queries, so that the CUDA library and the FP64 oracle can
be fed identical inputs.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_mixture(n: int, d: int, n_components: int = 20, center_range: float = 10.0,
                     sigma: float = 1.0, seed: int = 0, nq: int = 0):
    """Isotropic Gaussian mixture: centers U[-c, c]^d, per-point N(center, sigma^2 I).

    The 10k x 32 case (20 components, c = 10, sigma = 1) is the small plain
    FP32 workload.  Returns X (n, d) float32, or (X, Q) when nq > 0 (queries drawn
    from the same mixture after the points)."""
    g = _rng(seed)
    centers = g.uniform(-center_range, center_range, size=(n_components, d))
    lab = g.integers(0, n_components, size=n + nq)
    Z = g.standard_normal((n + nq, d))
    A = (centers[lab] + sigma * Z).astype(np.float32)
    return (A[:n], A[n:]) if nq else A


def sift_like(n: int, nq: int = 0, d: int = 128, n_clusters: int = 1000, seed: int = 0,
              chunk: int = 1 << 17):
    """SIFT-shaped integers in [0, 255] stored as float32.

    A 1000-cluster Gaussian mixture with a low intrinsic dimension, clipped to
    [0, 255] and rounded:
      centers      c_j = 255 * Beta(0.7, 2.2)^d         (skewed to small values)
      basis        one random orthonormal Q (d x d) shared by all clusters
      spectrum     s_k = 48 * (k + 1)^-0.6, k = 0..d-1   (decaying, ~10 effective dims)
      cluster scale a_j ~ U[0.5, 1.5]
      point        x = clip(round(c_j + a_j * Q (s * z)), 0, 255),  z ~ N(0, I)
    Queries (nq) come from the same mixture, drawn after the points."""
    g = _rng(seed)
    centers = 255.0 * g.beta(0.7, 2.2, size=(n_clusters, d))
    Qb, _ = np.linalg.qr(g.standard_normal((d, d)))
    spec = 48.0 * (np.arange(d) + 1.0) ** -0.6
    scale = g.uniform(0.5, 1.5, size=n_clusters)
    tot = n + nq
    lab = g.integers(0, n_clusters, size=tot)
    out = np.empty((tot, d), np.float32)
    M = (spec[:, None] * Qb.T)  # (d, d): z @ M = Q (s * z) as row vectors
    for s in range(0, tot, chunk):
        e = min(tot, s + chunk)
        z = g.standard_normal((e - s, d))
        x = centers[lab[s:e]] + scale[lab[s:e], None] * (z @ M)
        out[s:e] = np.clip(np.rint(x), 0.0, 255.0)
    return (out[:n], out[n:]) if nq else out


def gist_like(n: int, nq: int = 0, d: int = 960, n_clusters: int = 500, seed: int = 0,
              chunk: int = 1 << 15):
    """GIST-shaped float32: a 500-cluster Gaussian mixture with per-dimension
    scales s_k log-uniform in [0.1, 10]; centers N(0, (2 s_k)^2), points
    N(center, s_k^2).  Queries from the same mixture, drawn after the points."""
    g = _rng(seed)
    s = np.exp(g.uniform(np.log(0.1), np.log(10.0), size=d))
    centers = 2.0 * s * g.standard_normal((n_clusters, d))
    tot = n + nq
    lab = g.integers(0, n_clusters, size=tot)
    out = np.empty((tot, d), np.float32)
    for a in range(0, tot, chunk):
        b = min(tot, a + chunk)
        out[a:b] = centers[lab[a:b]] + s * g.standard_normal((b - a, d))
    return (out[:n], out[n:]) if nq else out


def deep_like(n: int, nq: int = 0, d: int = 96, n_clusters: int = 50, kappa: float = 8.0,
              seed: int = 0):
    """DEEP-shaped unit vectors: a von Mises-Fisher-like mixture made by
    normalising mu_j * kappa + N(0, I) with unit mean directions mu_j."""
    g = _rng(seed)
    mu = g.standard_normal((n_clusters, d))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    tot = n + nq
    lab = g.integers(0, n_clusters, size=tot)
    x = kappa * mu[lab] + g.standard_normal((tot, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x = x.astype(np.float32)
    return (x[:n], x[n:]) if nq else x


def small_integers(n: int, d: int, lo: int = -8, hi: int = 8, seed: int = 0, nq: int = 0):
    """Integer coordinates in [lo, hi] stored as float32.  Every squared distance
    and inner product is then an exact integer in FP32 and FP64, so the FP32
    device path and the FP64 oracle must agree bit for bit, ties included."""
    g = _rng(seed)
    A = g.integers(lo, hi + 1, size=(n + nq, d)).astype(np.float32)
    return (A[:n], A[n:]) if nq else A
