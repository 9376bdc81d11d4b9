"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the only code shared by the CUDA path (tests, bench) and the
oracle's tests.  It holds random draws and nothing of the method itself: no
ranks, no pseudo-distances, no stress.  Every generator takes an explicit seed
and returns float32 arrays, rounded once, so that both sides consume identical
bits.

Shapes and contamination models follow the paper's experiments:

* Gaussian data with outlier rows multiplied by 10 sd(X) (Section V-A, UCI
  contamination experiment).
* 28x28 image-like rows: values on a sparse blob mask plus Gaussian pixel noise,
  clipped to [0, 1] (Section V-B, MNIST with noise).  The real MNIST digits are
  not available; these blobs stand in for them.
* Gaussian mixtures with heavy-tailed Student-t contamination and the heavy
  tailed families of Section V-C.
* Batches of UCI-sized problems (n and p drawn over the ranges of Table I).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20260101


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def gaussian_outliers(n: int, p: int, seed: int, frac: float = 0.05,
                      factor: float = 10.0) -> np.ndarray:
    """X ~ N(0, 1) with round(frac*n) random rows multiplied by factor*sd(X)."""
    rng = _rng(seed)
    X = rng.standard_normal((n, p))
    n_out = int(round(frac * n))
    if n_out:
        rows = rng.choice(n, n_out, replace=False)
        X[rows] *= factor * X.std()
    return np.ascontiguousarray(X, dtype=np.float32)


def _blob_prototypes(rng: np.random.Generator, side: int, n_protos: int) -> np.ndarray:
    yy, xx = np.mgrid[0:side, 0:side].astype(np.float64)
    protos = np.zeros((n_protos, side, side), dtype=bool)
    for q in range(n_protos):
        field = np.zeros((side, side))
        for _ in range(int(rng.integers(1, 4))):
            cy, cx = rng.uniform(side * 0.25, side * 0.75, size=2)
            s = rng.uniform(side / 14.0, side / 6.0)
            field += np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * s * s))
        coverage = rng.uniform(0.15, 0.20)
        thr = np.quantile(field, 1.0 - coverage)
        protos[q] = field > thr
    return protos


def _shift(mask: np.ndarray, dy: int, dx: int) -> np.ndarray:
    out = np.zeros_like(mask)
    side = mask.shape[0]
    ys = slice(max(dy, 0), side + min(dy, 0))
    yd = slice(max(-dy, 0), side + min(-dy, 0))
    xs = slice(max(dx, 0), side + min(dx, 0))
    xd = slice(max(-dx, 0), side + min(-dx, 0))
    out[ys, xs] = mask[yd, xd]
    return out


def image_like(n: int, seed: int, side: int = 28, n_protos: int = 10,
               jitter: int = 2, noise_sd: float = 0.1) -> np.ndarray:
    """Noisy image-like rows of length side*side.

    Each row picks one of n_protos blob masks (1-3 Gaussian blobs thresholded
    to 15-20% of the pixels), shifted by up to +-jitter pixels.  Masked pixels
    are U[0, 1], the rest 0; N(0, noise_sd^2) is added to every pixel and the
    result is clipped to [0, 1], which leaves exact 0 and 1 values (ties).
    """
    rng = _rng(seed)
    protos = _blob_prototypes(rng, side, n_protos)
    shifts = [(dy, dx) for dy in range(-jitter, jitter + 1)
              for dx in range(-jitter, jitter + 1)]
    bank = np.stack([_shift(protos[q], dy, dx) for q in range(n_protos)
                     for (dy, dx) in shifts]).reshape(len(protos) * len(shifts), -1)
    pick = rng.integers(0, bank.shape[0], size=n)
    X = rng.random((n, side * side), dtype=np.float32)
    X *= bank[pick]
    X += rng.standard_normal((n, side * side), dtype=np.float32) * np.float32(noise_sd)
    np.clip(X, 0.0, 1.0, out=X)
    return np.ascontiguousarray(X, dtype=np.float32)


def gaussian_mixture(n: int, p: int, seed: int, n_clusters: int = 10,
                     centre_sd: float = 5.0, heavy_frac: float = 0.03,
                     t_df: float = 1.5) -> np.ndarray:
    """Mixture of n_clusters unit Gaussians with centres ~ N(0, centre_sd^2 I).

    round(heavy_frac*n) rows get Student-t(t_df) noise added to every feature.
    """
    rng = _rng(seed)
    centres = rng.normal(0.0, centre_sd, size=(n_clusters, p))
    lab = rng.integers(0, n_clusters, size=n)
    X = centres[lab] + rng.standard_normal((n, p))
    n_h = int(round(heavy_frac * n))
    if n_h:
        rows = rng.choice(n, n_h, replace=False)
        X[rows] += rng.standard_t(t_df, size=(n_h, p))
    return np.ascontiguousarray(X, dtype=np.float32)


def heavy_tailed(n: int, d: int, kind: str, seed: int) -> np.ndarray:
    """The six heavy-tailed families of Section V-C."""
    rng = _rng(seed)
    if kind == "gauss_contaminated":
        X = rng.standard_normal((n, d))
        m = rng.random(n) < 0.05
        X[m] = rng.normal(0.0, 10.0, size=(int(m.sum()), d))
    elif kind == "cauchy":
        X = rng.standard_cauchy((n, d))
    elif kind == "weibull":
        X = rng.weibull(0.5, size=(n, d))
    elif kind == "pareto":
        X = rng.pareto(2.0, size=(n, d)) + 1.0
    elif kind == "student":
        X = rng.standard_t(2.0, size=(n, d))
    elif kind == "lognormal":
        X = rng.lognormal(0.0, 1.5, size=(n, d))
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(X, dtype=np.float32)


def integer_valued(n: int, p: int, seed: int, levels: int = 5) -> np.ndarray:
    """Small integer features (many exact ties), like the Integer columns of Table I."""
    rng = _rng(seed)
    return rng.integers(0, levels, size=(n, p)).astype(np.float32)


def uci_like_batch(n_problems: int, seed: int, n_range=(100, 4000),
                   p_range=(4, 60)) -> list:
    """UCI-sized problems: n ~ U{n_range}, p ~ U{p_range}, 2-6 Gaussian clusters,
    5% outlier rows times 10 sd(X); every fourth problem rounded to integers."""
    rng = _rng(seed)
    out = []
    for q in range(n_problems):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        c = int(rng.integers(2, 7))
        centres = rng.normal(0.0, 3.0, size=(c, p))
        X = centres[rng.integers(0, c, size=n)] + rng.standard_normal((n, p))
        n_out = int(round(0.05 * n))
        rows = rng.choice(n, n_out, replace=False)
        X[rows] *= 10.0 * X.std()
        if q % 4 == 3:
            X = np.round(X)
        out.append(np.ascontiguousarray(X, dtype=np.float32))
    return out


def y_init(n: int, k: int, seed: int, sd: float = 0.1) -> np.ndarray:
    """Initial embedding Y0 ~ N(0, sd^2), sd = 0.1 (variance 1e-2)."""
    rng = _rng(seed)
    return np.ascontiguousarray(rng.normal(0.0, sd, size=(n, k)), dtype=np.float32)


def distinct_vectors(nseg: int, m: int, seed: int) -> np.ndarray:
    """Segments of m distinct values each (a random permutation of a grid)."""
    rng = _rng(seed)
    base = np.arange(m, dtype=np.float32) - m / 2
    return np.stack([rng.permutation(base) for _ in range(nseg)]).astype(np.float32)


def tied_vectors(nseg: int, m: int, seed: int, levels: int = 4) -> np.ndarray:
    """Segments drawn from a few levels, so most values are tied."""
    rng = _rng(seed)
    return (rng.integers(-levels // 2, levels - levels // 2, size=(nseg, m))
            .astype(np.float32) * np.float32(0.5))


# Named workloads (sizes as the paper's experiments suggest; the seed is
# SEED_BASE + an id).
WORKLOADS = {
    "gauss-outliers-n200-p10": dict(kind="gaussian_outliers", n=200, p=10, k=2,
                                    nu=[2.0], iters=100, seed=SEED_BASE + 1),
    "image-n2000-p784": dict(kind="image_like", n=2000, p=784, k=2,
                             nu=[1.5, 2.0, 3.0], iters=100, seed=SEED_BASE + 2),
    "mixture-n5000-p50": dict(kind="gaussian_mixture", n=5000, p=50, k=2,
                              nu=[2.0], iters=500, seed=SEED_BASE + 3),
    "uci-batch-64": dict(kind="uci_like_batch", n_problems=64, k=2,
                         nu=list(np.linspace(1.1, 4.0, 8)), restarts=8,
                         iters=200, seed=SEED_BASE + 4),
    "image-n20000-p784": dict(kind="image_like", n=20000, p=784, k=2,
                              nu=[2.0], iters=200, seed=SEED_BASE + 5),
    # smaller case of the same kind for profiler captures (BF16 Delta > L2)
    "image-n12000-p784": dict(kind="image_like", n=12000, p=784, k=2,
                              nu=[2.0], iters=200, seed=SEED_BASE + 6),
}


def make_X(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    if w["kind"] == "gaussian_outliers":
        return gaussian_outliers(w["n"], w["p"], w["seed"])
    if w["kind"] == "image_like":
        return image_like(w["n"], w["seed"])
    if w["kind"] == "gaussian_mixture":
        return gaussian_mixture(w["n"], w["p"], w["seed"])
    raise ValueError(name)
