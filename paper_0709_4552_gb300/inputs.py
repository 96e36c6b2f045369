"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only -- none of the method's arithmetic
(no forces, potentials, prediction or correction).  It draws, with numpy's
PCG64 generator and a stated seed:

* ``plummer``: a Plummer sphere (the initial model of Sec. 2) sampled with the
  Aarseth, Henon & Wielen (1974) recipe, centred on its centre of mass and
  scaled analytically to virial N-body units (G = M = 1, E = -1/4): positions
  times 3 pi / 16, velocities times sqrt(16 / (3 pi)).
* ``salpeter_masses``: a Salpeter (1955) mass function dN/dm ~ m^-2.35 on
  [0.1, 100], inverse-CDF sampled, normalised to total mass 1 (Sec. 6 names
  the Salpeter spectrum for production runs).
* ``sample_indices``: a sorted seeded subset of particle indices (active
  blocks and sampled parity checks).
* ``ensemble_sizes``: cluster sizes log-uniform in [lo, hi].
* ``block_size``: the average block size law n = 0.20 N^0.81 of Sec. 3.2.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["plummer", "salpeter_masses", "sample_indices", "ensemble_sizes", "block_size",
           "SALPETER_ALPHA", "SALPETER_MLO", "SALPETER_MHI"]

SALPETER_ALPHA = 2.35
SALPETER_MLO = 0.1
SALPETER_MHI = 100.0


def salpeter_masses(N: int, rng: np.random.Generator, alpha: float = SALPETER_ALPHA,
                    mlo: float = SALPETER_MLO, mhi: float = SALPETER_MHI) -> np.ndarray:
    """N masses from dN/dm ~ m^-alpha on [mlo, mhi], normalised to sum 1."""
    u = rng.random(N)
    e = 1.0 - alpha
    lo, hi = mlo ** e, mhi ** e
    m = (lo + u * (hi - lo)) ** (1.0 / e)
    return m / m.sum()


def _isotropic(rng: np.random.Generator, mag: np.ndarray) -> np.ndarray:
    n = mag.shape[0]
    z = (1.0 - 2.0 * rng.random(n)) * mag
    phi = 2.0 * math.pi * rng.random(n)
    rho = np.sqrt(np.maximum(mag * mag - z * z, 0.0))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def plummer(N: int, seed: int, masses: str = "equal", rmax: float = 10.0):
    """Plummer sphere of N particles in virial N-body units.

    Returns (m[N], x[N,3], v[N,3]) as float64.  ``masses`` is ``"equal"``
    (m = 1/N) or ``"salpeter"``.  Masses are drawn first, from the same
    stream, then radii, position angles, speeds and velocity angles.
    """
    if N <= 0:
        raise ValueError("N must be positive")
    rng = np.random.default_rng(seed)
    if masses == "equal":
        m = np.full(N, 1.0 / N)
    elif masses == "salpeter":
        m = salpeter_masses(N, rng)
    else:
        raise ValueError(f"unknown mass spectrum {masses!r}")
    # radii: cumulative mass fraction X -> r = (X^(-2/3) - 1)^(-1/2), r <= rmax
    r = np.empty(0)
    while r.shape[0] < N:
        X = rng.random(2 * (N - r.shape[0]) + 16)
        X = X[X > 0.0]
        rr = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        r = np.concatenate([r, rr[rr <= rmax]])
    r = r[:N]
    x = _isotropic(rng, r)
    # speeds: q from g(q) = q^2 (1 - q^2)^(7/2) by rejection (max of g < 0.1),
    # v = q * v_escape,  v_escape = sqrt(2) (1 + r^2)^(-1/4)
    q = np.empty(0)
    while q.shape[0] < N:
        k = 12 * (N - q.shape[0]) + 16
        X4 = rng.random(k)
        X5 = rng.random(k)
        ok = 0.1 * X5 < X4 * X4 * (1.0 - X4 * X4) ** 3.5
        q = np.concatenate([q, X4[ok]])
    q = q[:N]
    vmag = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v = _isotropic(rng, vmag)
    # centre of mass at rest in the origin
    x -= (m[:, None] * x).sum(axis=0) / m.sum()
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    # analytic scaling to virial units (Plummer scale length 3 pi / 16)
    x *= 3.0 * math.pi / 16.0
    v *= math.sqrt(16.0 / (3.0 * math.pi))
    return m, np.ascontiguousarray(x), np.ascontiguousarray(v)


def sample_indices(N: int, k: int, seed: int) -> np.ndarray:
    """Sorted k distinct indices in [0, N): the first k of a seeded shuffle."""
    k = min(int(k), int(N))
    rng = np.random.default_rng(seed)
    return np.sort(rng.permutation(N)[:k]).astype(np.int64)


def ensemble_sizes(n_clusters: int = 512, lo: int = 256, hi: int = 16384, seed: int = 7) -> np.ndarray:
    """Cluster sizes round(exp(U(ln lo, ln hi)))."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), n_clusters)
    return np.clip(np.rint(np.exp(u)), lo, hi).astype(np.int64)


def block_size(N: int) -> int:
    """Average block size n = 0.20 N^0.81 (Sec. 3.2), at least 1."""
    return max(1, int(round(0.20 * N ** 0.81)))
