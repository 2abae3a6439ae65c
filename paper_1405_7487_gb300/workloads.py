"""Seeded synthetic particle sets for the FMM (inputs only, no FMM arithmetic).

These generators feed both the CUDA path and the double-precision oracle, so
they hold nothing of the method itself: only the particle distributions the
paper evaluates (Sec. III, "Cube", "Sphere" and "Plummer", Table 1) and the
loss weights of the differentiable workload.  Every array is float32, drawn
with ``numpy.random.default_rng(seed)`` in a fixed order so that a seed names
one input exactly.

Distributions (readings of the paper, which only names them):
  * cube:    positions i.i.d. uniform in [0, 1)^3, charges uniform [-1, 1).
  * plummer: radius r = a / sqrt(X^(-2/3) - 1) with X ~ U(0, 1), a = 1,
             redrawn while r > r_max (20); isotropic direction; equal charges
             1/N.
  * sphere:  points uniform on the unit sphere surface, charges uniform
             [-1, 1).
"""

from __future__ import annotations

import numpy as np


def cube(n: int, seed: int) -> np.ndarray:
    """(n, 4) float32 x, y, z, q: uniform cube [0,1)^3, charges U[-1, 1)."""
    rng = np.random.default_rng(seed)
    xyz = rng.random((n, 3))
    q = rng.uniform(-1.0, 1.0, n)
    return np.concatenate([xyz, q[:, None]], axis=1).astype(np.float32)


def _directions(rng, n):
    cz = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([s * np.cos(ph), s * np.sin(ph), cz], axis=1)


def plummer(n: int, seed: int, a: float = 1.0, r_max: float = 20.0) -> np.ndarray:
    """(n, 4) float32: Plummer sphere (scale a, truncated at r_max), q = 1/n."""
    rng = np.random.default_rng(seed)
    r = np.empty(n)
    filled = 0
    while filled < n:
        X = rng.random(n - filled)
        X = X[X > 0.0]
        rr = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        rr = rr[rr <= r_max]
        r[filled:filled + rr.shape[0]] = rr
        filled += rr.shape[0]
    xyz = r[:, None] * _directions(rng, n)
    q = np.full(n, 1.0 / n)
    return np.concatenate([xyz, q[:, None]], axis=1).astype(np.float32)


def sphere(n: int, seed: int) -> np.ndarray:
    """(n, 4) float32: uniform on the unit sphere surface, charges U[-1, 1)."""
    rng = np.random.default_rng(seed)
    xyz = _directions(rng, n)
    q = rng.uniform(-1.0, 1.0, n)
    return np.concatenate([xyz, q[:, None]], axis=1).astype(np.float32)


def weights(n: int, seed: int) -> np.ndarray:
    """(n,) float32 loss weights w ~ N(0, 1)."""
    return np.random.default_rng(seed).standard_normal(n).astype(np.float32)


def sample_targets(n: int, count: int, seed: int = 7) -> np.ndarray:
    """First `count` entries of a seeded permutation of range(n) (int64)."""
    return np.random.default_rng(seed).permutation(n)[: min(count, n)].astype(np.int64)


# The workloads the library is measured on (sizes and parameters of the
# paper's Table 1 cases, scaled to one GPU).
WORKLOADS = {
    "cube4k_p4": dict(dist="cube", n=4096, seed=1, p=4, theta=0.4, ncrit=64),
    "cube1m_p10": dict(dist="cube", n=1 << 20, seed=2, p=10, theta=0.4, ncrit=64),
    "plummer1m_p8": dict(dist="plummer", n=1 << 20, seed=3, p=8, theta=0.5, ncrit=32),
    "cube256k_p8_grad": dict(dist="cube", n=1 << 18, seed=4, p=8, theta=0.4, ncrit=64, wseed=40),
    "cube16m": dict(dist="cube", n=1 << 24, seed=5, p=(4, 8, 12, 16), theta=0.4, ncrit=64),
    # Table 1 case 2: bodies on a sphere surface, P = 10, theta = 0.4, N_crit = 512
    "sphere1m_p10": dict(dist="sphere", n=1 << 20, seed=6, p=10, theta=0.4, ncrit=512),
}


def make(name_or_spec, n: int | None = None) -> np.ndarray:
    """Particles of a named workload (optionally with a different n)."""
    spec = WORKLOADS[name_or_spec] if isinstance(name_or_spec, str) else name_or_spec
    nn = spec["n"] if n is None else n
    gen = {"cube": cube, "plummer": plummer, "sphere": sphere}[spec["dist"]]
    return gen(nn, spec["seed"])
