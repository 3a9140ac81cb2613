"""Seeded synthetic inputs shared by the oracle checks, the GPU tests and bench.

This module draws point clouds, weights and request streams.  It holds none
of the solver's arithmetic (no centering of features, no lift, no cost, no
Sinkhorn); both the oracle and the CUDA path start from its outputs.

Every generator takes an integer seed and uses numpy's PCG64.  The shapes
and value distributions follow the paper's workloads (radius-1 normalised 3D
shapes of 4k-250k points, D = 16..64 features, eps from 1e-1 down to 1e-3,
uniform weights; Section 6 "Setup" and Appendix E), which are not available
here: these clouds stand in for them.
"""

from __future__ import annotations

import math

import numpy as np

F64 = np.float64


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_weights(n: int) -> np.ndarray:
    """a_i = 1/N (every experiment in the paper uses uniform weights)."""
    return np.full(n, 1.0 / n, dtype=F64)


def random_weights(n: int, seed: int, spread: float = 1.0) -> np.ndarray:
    """Positive weights summing to one, log-normal with the given spread."""
    w = np.exp(spread * rng(seed).standard_normal(n))
    return w / w.sum()


def random_orthogonal(d: int, g: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian matrix with the
    signs of R's diagonal folded into Q)."""
    A = g.standard_normal((d, d))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))[None, :]


def normalize_radius(x: np.ndarray) -> np.ndarray:
    """Shift to the unweighted mean and scale so the largest norm is 1 (the
    paper normalises every input shape to radius 1)."""
    x = x - x.mean(axis=0)
    return x / np.sqrt((x * x).sum(axis=1)).max()


def square_rotated(n: int = 1000, seed: int = 0, noise: float = 0.01):
    """2D squared-Euclidean workload: x ~ U[0,1]^2, y = R_theta x + N(0, noise^2),
    then shuffled; theta ~ U[0, 2 pi).  eps = 1e-2 * diam^2 with diam the
    bounding-box diagonal of x.  Returns dict(x, y, a, b, eps, perm, theta)."""
    g = rng(seed)
    x = g.random((n, 2))
    theta = g.uniform(0.0, 2.0 * math.pi)
    R = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    y = x @ R.T + noise * g.standard_normal((n, 2))
    perm = g.permutation(n)
    y = y[perm]
    lo, hi = x.min(axis=0), x.max(axis=0)
    diam = float(np.sqrt(((hi - lo) ** 2).sum()))
    return {"x": x, "y": y, "a": uniform_weights(n), "b": uniform_weights(n),
            "eps": 1e-2 * diam * diam, "perm": perm, "theta": theta}


def gmm_blobs(n: int, g: np.random.Generator, n_blobs: int = 8) -> np.ndarray:
    """3D mixture of anisotropic Gaussian blobs: means U[-1,1]^3, covariance
    Q diag(sigma^2) Q^T with sigma log-uniform in [0.03, 0.3], Q random."""
    means = g.uniform(-1.0, 1.0, (n_blobs, 3))
    covs = []
    for _ in range(n_blobs):
        sig = np.exp(g.uniform(math.log(0.03), math.log(0.3), 3))
        Q = random_orthogonal(3, g)
        covs.append((Q * sig[None, :]))          # x = mean + Q diag(sig) z
    counts = g.multinomial(n, np.full(n_blobs, 1.0 / n_blobs))
    parts = []
    for k in range(n_blobs):
        z = g.standard_normal((counts[k], 3))
        parts.append(means[k] + z @ covs[k].T)
    x = np.concatenate(parts, axis=0)
    return x[g.permutation(n)]


def gmm_rigid(n: int = 100_000, seed: int = 0, m: int | None = None, jitter: float = 0.01):
    """3D workload: x = 8-blob Gaussian mixture; y = (random rotation/reflection
    of x) + translation + N(0, (jitter * diam)^2), shuffled; both clouds
    normalised to radius 1.  If m != n, y is built from its own draw of m
    points of the same mixture.  Returns dict(x, y, a, b)."""
    m = n if m is None else m
    g = rng(seed)
    x = gmm_blobs(n, g)
    src = x if m == n else gmm_blobs(m, rng(seed + 7919))
    Q = random_orthogonal(3, g)
    shift = g.uniform(-1.0, 1.0, 3)
    diam = float(np.sqrt(((src.max(0) - src.min(0)) ** 2).sum()))
    y = src @ Q.T + shift + jitter * diam * g.standard_normal((m, 3))
    y = y[g.permutation(m)]
    return {"x": normalize_radius(x), "y": normalize_radius(y),
            "a": uniform_weights(n), "b": uniform_weights(m)}


def sphere_warp(n: int = 250_000, seed: int = 0, amp: float = 0.15):
    """Points on the unit sphere (normalised Gaussians) and the same points
    under y = Q (x + amp tanh(A x + c)) mapped back to the sphere, shuffled;
    A ~ N(0, 1)/sqrt(3), c ~ U[-1, 1]^3."""
    g = rng(seed)
    z = g.standard_normal((n, 3))
    x = z / np.sqrt((z * z).sum(1))[:, None]
    A = g.standard_normal((3, 3)) / math.sqrt(3.0)
    c = g.uniform(-1.0, 1.0, 3)
    Q = random_orthogonal(3, g)
    w = x + amp * np.tanh(x @ A.T + c)
    w = w @ Q.T
    y = w / np.sqrt((w * w).sum(1))[:, None]
    y = y[g.permutation(n)]
    return {"x": x, "y": y, "a": uniform_weights(n), "b": uniform_weights(n)}


def serving_requests(n_req: int = 512, seed: int = 0, rate: float = 1.0,
                     n_min: int = 500, n_max: int = 50_000):
    """Request stream: Poisson arrivals (exponential gaps of mean 1/rate s),
    N and M independently log-uniform in [n_min, n_max], penalty squared
    (D = 3) or lifted with D = 16 or 32 (probability 1/3 each), eps
    log-uniform in [1e-3, 1e-1].  Point clouds are drawn lazily from
    gmm_rigid with the request's own seed.  Returns a list of dicts."""
    g = rng(seed)
    t = 0.0
    out = []
    for r in range(n_req):
        t += g.exponential(1.0 / rate)
        n = int(round(math.exp(g.uniform(math.log(n_min), math.log(n_max)))))
        m = int(round(math.exp(g.uniform(math.log(n_min), math.log(n_max)))))
        kind = int(g.integers(0, 3))
        D = (3, 16, 32)[kind]
        eps = float(math.exp(g.uniform(math.log(1e-3), math.log(1e-1))))
        out.append({"id": r, "arrival": t, "n": n, "m": m, "D": D,
                    "penalty": "sqeuclid" if kind == 0 else "power",
                    "eps": eps, "seed": int(seed) * 100_003 + r})
    return out


def random_features(n: int, d: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Gaussian rows, for kernel-level tests that need arbitrary inputs."""
    return scale * rng(seed).standard_normal((n, d))
