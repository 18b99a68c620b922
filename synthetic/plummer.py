"""Seeded synthetic workloads: Plummer spheres, active sets, Kepler pairs, ensembles.

Plummer sampling follows the recipe of Aarseth, Henon & Wielen (1974), which
the paper cites for its initial conditions (Sect. 4, "Results"): radii from
the inverse cumulative mass profile, isotropic directions, speeds by von
Neumann rejection on the isotropic distribution function, centre-of-mass
removal, and equal masses.  Lengths and speeds are then converted from
Plummer units (G = M = a = 1, E = -3 pi / 64) to Henon N-body units
(G = M = 1, E = -1/4) by the analytic factors 3 pi / 16 and (16 / 3 pi)^(1/2).
The sample is not rescaled to exact virial equilibrium: that would need a
pairwise potential sum, which belongs to the method under test, so the
sampled energy equals -1/4 only up to O(N^-1/2) fluctuations.

The paper does not state where the radial distribution is truncated; draws
of the cumulative mass fraction above 0.999 are rejected and redrawn.

Random numbers come from the counter-based SplitMix64 in ``synthetic.rng``.
"""
from __future__ import annotations

import math

import numpy as np

from . import rng

# Sub-stream identifiers (one per kind of draw) for the Plummer sampler.
_S_RADIUS, _S_POSDIR, _S_SPEED, _S_VELDIR = 1, 2, 3, 4
_S_ACTIVE, _S_CLUSTER_N = 5, 6
_MAX_ATTEMPTS = 1 << 20  # attempts per particle reserved in the counter space
MASS_FRACTION_CUT = 0.999
HENON_LENGTH = 3.0 * math.pi / 16.0


def _isotropic(seed: int, stream: int, idx: np.ndarray):
    u = rng.uniform(seed, stream, 2 * idx)
    w = rng.uniform(seed, stream, 2 * idx + 1)
    cz = 2.0 * u - 1.0
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    ph = 2.0 * math.pi * w
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)


def _radii(seed: int, n: int) -> np.ndarray:
    idx = np.arange(n, dtype=np.uint64)
    r = np.empty(n)
    pending = np.arange(n)
    attempt = 0
    while pending.size:
        ctr = idx[pending] * np.uint64(_MAX_ATTEMPTS) + np.uint64(attempt)
        X = rng.uniform_open(seed, _S_RADIUS, ctr)
        ok = X <= MASS_FRACTION_CUT
        sel = pending[ok]
        r[sel] = 1.0 / np.sqrt(X[ok] ** (-2.0 / 3.0) - 1.0)
        pending = pending[~ok]
        attempt += 1
    return r


def _speed_fractions(seed: int, n: int) -> np.ndarray:
    """q = v / v_esc by rejection on g(q) = q^2 (1 - q^2)^(7/2) under the box 0.1."""
    idx = np.arange(n, dtype=np.uint64)
    q = np.empty(n)
    pending = np.arange(n)
    attempt = 0
    while pending.size:
        ctr = (idx[pending] * np.uint64(_MAX_ATTEMPTS) + np.uint64(attempt)) * np.uint64(2)
        qq = rng.uniform(seed, _S_SPEED, ctr)
        yy = 0.1 * rng.uniform(seed, _S_SPEED, ctr + np.uint64(1))
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[pending[ok]] = qq[ok]
        pending = pending[~ok]
        attempt += 1
    return q


def plummer_sphere(n: int, seed: int, *, henon: bool = True):
    """Equal-mass Plummer sphere of ``n`` particles.

    Returns ``(m, x, v)``: masses (n,), positions (n, 3), velocities (n, 3),
    all float64.  Total mass 1; centre of mass at rest at the origin.
    With ``henon=False`` the result stays in Plummer units (a = 1).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    idx = np.arange(n, dtype=np.uint64)
    r = _radii(seed, n)
    x = r[:, None] * _isotropic(seed, _S_POSDIR, idx)
    v_esc = math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vel = (_speed_fractions(seed, n) * v_esc)[:, None] * _isotropic(seed, _S_VELDIR, idx)
    m = np.full(n, 1.0 / n)
    x -= (m[:, None] * x).sum(axis=0) / m.sum()
    vel -= (m[:, None] * vel).sum(axis=0) / m.sum()
    if henon:
        x *= HENON_LENGTH
        vel /= math.sqrt(HENON_LENGTH)
    return m, np.ascontiguousarray(x), np.ascontiguousarray(vel)


def active_subset(n: int, n_act: int, seed: int) -> np.ndarray:
    """Seeded uniform sample of ``n_act`` distinct indices of ``range(n)``, ascending, int32."""
    if not 0 <= n_act <= n:
        raise ValueError("need 0 <= n_act <= n")
    if n_act == n:
        return np.arange(n, dtype=np.int32)
    keys = rng.bits(seed, _S_ACTIVE, np.arange(n, dtype=np.uint64))
    pick = np.argpartition(keys, n_act - 1)[:n_act] if n_act else np.array([], dtype=np.int64)
    return np.sort(pick).astype(np.int32)


def ensemble_sizes(n_clusters: int, seed: int, lo: int = 256, hi: int = 8192) -> np.ndarray:
    """Cluster sizes floor(exp(U(ln lo, ln hi))), one per cluster (int64)."""
    u = rng.uniform(seed, _S_CLUSTER_N, np.arange(n_clusters, dtype=np.uint64))
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def kepler_pair(e: float, *, a: float = 1.0, m1: float = 0.5, m2: float = 0.5):
    """Two bodies on a Kepler ellipse (G = 1) at pericentre, centre of mass at rest.

    Semi-major axis ``a``, eccentricity ``e``; the relative orbit lies in the
    x-y plane with pericentre on +x.  Period 2 pi (a^3 / (m1 + m2))^(1/2),
    energy -m1 m2 / (2 a).
    """
    mt = m1 + m2
    rp = a * (1.0 - e)
    vp = math.sqrt(mt * (1.0 + e) / (a * (1.0 - e)))
    rel_x = np.array([rp, 0.0, 0.0])
    rel_v = np.array([0.0, vp, 0.0])
    x = np.stack([-m2 / mt * rel_x, m1 / mt * rel_x])
    v = np.stack([-m2 / mt * rel_v, m1 / mt * rel_v])
    return np.array([m1, m2]), x, v
