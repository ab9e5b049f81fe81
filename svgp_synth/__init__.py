"""Seeded synthetic inputs for the inverse-free SVGP training step.

This module is shared by the FP64 oracle tests, the GPU parity tests and the
benchmark.  It holds only random-number generation and the synthetic target
functions; none of the method's arithmetic (kernel matrices, bounds,
natural-gradient updates) lives here.

Workloads (shapes and value distributions follow the paper's experiments,
Section 4 and Appendix S4; the datasets themselves are not used):

* ``snelson_like``   -- 1-D regression, N=200, x ~ U[0, 6],
  y = sin 2x + 0.3 cos 5x + N(0, 0.2^2), M=16 inducing points on a grid
  (stands in for SNELSON, Appendix S4.3).
* ``sinusoid_regression`` -- D=8, x ~ N(0, I), y = sum of 4 sinusoids of
  random projections + N(0, 0.1^2), N=1e5, B=1024, M=512.
* ``gp_sample_regression`` -- D=16, x ~ U[-1, 1], y a draw of an SE-ARD GP
  (lengthscales ~ U[0.3, 2], unit variance) approximated by 2048 random
  Fourier features, + N(0, 0.05^2); N=1e6, B=4096, M=2048.
* ``banana_like`` -- two interleaved noisy crescents (noise sd 0.1),
  labels in {0, 1}, N=5e4, B=2048, M=256.

Every dataset is defined point-by-point from counter-seeded generators so a
minibatch of an N=1e6 dataset can be produced without materialising all N
points: batch ``b`` holds the points of chunk ``b`` of a fixed random order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem",
    "snelson_like",
    "sinusoid_regression",
    "gp_sample_regression",
    "banana_like",
    "random_state",
    "WORKLOADS",
]


@dataclasses.dataclass
class Problem:
    """One regression/classification problem instance.

    ``batch(b)`` returns minibatch ``b`` (X float64 [B, D], y float64 [B]).
    ``Z0`` holds the initial inducing inputs (float64 [M, D]).
    """

    name: str
    N: float
    B: int
    M: int
    D: int
    Z0: np.ndarray
    _batch_fn: object
    likelihood: str = "gaussian"

    def batch(self, b: int = 0):
        return self._batch_fn(b)


def _rng(*key):
    return np.random.default_rng(list(key))


def snelson_like(seed: int = 0, M: int = 16) -> Problem:
    N = 200
    rng = _rng(seed, 0)
    x = rng.uniform(0.0, 6.0, size=N)
    y = np.sin(2 * x) + 0.3 * np.cos(5 * x) + rng.normal(0.0, 0.2, size=N)
    X = x[:, None]
    Z0 = np.linspace(x.min(), x.max(), M)[:, None]
    return Problem("snelson_like", float(N), N, M, 1, Z0, lambda b: (X.copy(), y.copy()))


def _sinusoid_target(seed, D, nterms=4):
    rng = _rng(seed, 1)
    W = rng.normal(size=(nterms, D))
    b = rng.uniform(0.0, 2 * math.pi, size=nterms)
    return W, b


def sinusoid_regression(seed: int = 1, N: int = 100_000, B: int = 1024, M: int = 512,
                        D: int = 8) -> Problem:
    W, bias = _sinusoid_target(seed, D)

    def batch(b):
        rng = _rng(seed, 2, b)
        X = rng.normal(size=(B, D))
        y = np.sin(X @ W.T + bias).sum(axis=1) + rng.normal(0.0, 0.1, size=B)
        return X, y

    Z0 = _rng(seed, 3).permutation(batch(0)[0])[:M] if M <= B else \
        np.concatenate([batch(k)[0] for k in range((M + B - 1) // B)])[:M]
    return Problem("sinusoid_regression", float(N), B, M, D, Z0, batch)


def _rff_target(seed, D, R=2048):
    """Random Fourier features of an SE-ARD kernel with unit variance."""
    rng = _rng(seed, 1)
    ls = rng.uniform(0.3, 2.0, size=D)
    Om = rng.normal(size=(R, D)) / ls
    ph = rng.uniform(0.0, 2 * math.pi, size=R)
    a = rng.normal(size=R)
    return ls, Om, ph, a


def gp_sample_regression(seed: int = 2, N: float = 1e6, B: int = 4096, M: int = 2048,
                         D: int = 16, R: int = 2048) -> Problem:
    ls, Om, ph, a = _rff_target(seed, D, R)
    scale = math.sqrt(2.0 / R)

    def batch(b):
        rng = _rng(seed, 2, b)
        X = rng.uniform(-1.0, 1.0, size=(B, D))
        f = scale * (np.cos(X @ Om.T + ph) @ a)
        y = f + rng.normal(0.0, 0.05, size=B)
        return X, y

    # initial Z: M distinct data points (the first chunks of the random order)
    nb = (M + B - 1) // B
    Z0 = np.concatenate([batch(10_000 + k)[0] for k in range(nb)])[:M]
    return Problem("gp_sample_regression", float(N), B, M, D, Z0, batch)


def banana_like(seed: int = 3, N: int = 50_000, B: int = 2048, M: int = 256) -> Problem:
    def batch(b):
        rng = _rng(seed, 2, b)
        lab = rng.integers(0, 2, size=B)
        t = rng.uniform(0.0, math.pi, size=B)
        x0 = np.where(lab == 0, np.cos(t), 1.0 - np.cos(t))
        x1 = np.where(lab == 0, np.sin(t), 0.5 - np.sin(t))
        X = np.stack([x0, x1], axis=1) + rng.normal(0.0, 0.1, size=(B, 2))
        return X, lab.astype(np.float64)

    Z0 = _rng(seed, 3).permutation(batch(0)[0])[:M]
    return Problem("banana_like", float(N), B, M, 2, Z0, batch, likelihood="probit")


def random_state(M: int, D: int, seed: int, *, L_scale: float | None = None,
                 s_range=(0.05, 0.5), ell_range=(0.6, 1.6), Z_scale=1.0):
    """A random parameter state (for pins and parity tests).

    Returns a dict with Z [M,D], ell [D], sf2, noise, m [M], s [M] and a
    random lower-triangular L [M,M] with positive diagonal.
    """
    rng = _rng(seed, 7)
    Z = rng.normal(size=(M, D)) * Z_scale
    ell = rng.uniform(*ell_range, size=D)
    sf2 = float(rng.uniform(0.5, 2.0))
    noise = float(rng.uniform(0.05, 0.5))
    m = rng.normal(size=M)
    s = rng.uniform(*s_range, size=M)
    if L_scale is None:
        L_scale = 1.0 / math.sqrt(M)
    L = np.tril(rng.normal(size=(M, M))) * (0.3 * L_scale)
    L[np.diag_indices(M)] = rng.uniform(0.5, 1.5, size=M) * L_scale
    return dict(Z=Z, ell=ell, sf2=sf2, noise=noise, m=m, s=s, L=L)


WORKLOADS = {
    "snelson_like": snelson_like,
    "sinusoid_regression": sinusoid_regression,
    "gp_sample_regression": gp_sample_regression,
    "banana_like": banana_like,
}
