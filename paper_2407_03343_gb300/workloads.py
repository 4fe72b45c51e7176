"""Seeded synthetic sphere configurations shaped like the paper's workloads.

This module only places spheres and draws boundary data; it holds none of the
method's arithmetic, so both the CUDA library's tests and the CPU oracle can take
their inputs from it.  All generators are deterministic for a given seed.

two_spheres        two unit spheres on the x axis with gap delta (Sec. 3, Sec. 5.1).
gap_sweep          18 gaps log-spaced in [1e-3, 1] and the three relative motions
                   (squeezing, shearing, counter-rotation) of Sec. 5.1.
suspension         P spheres in a cube of volume fraction phi, grown from uniformly
                   placed seeds by attaching new spheres to one or two existing spheres at
                   gaps drawn log-uniformly in [gap_lo, gap_hi] (near contacts), every pair
                   kept at least min_gap apart.  Random rigid velocities ~ N(0, 1).
batch              64 independent suspensions with P_i log-uniform in [2, 256],
                   phi_i ~ U(0.05, 0.3).
cluster            fixed clusters grown so that every sphere has a neighbour exactly gap away
                   (Sec. 4, Ex. 2; Sec. 5.2), with shear_flow / uniform_flow as background flows.
"""
from __future__ import annotations

import math

import numpy as np


def two_spheres(delta: float, radius: float = 1.0):
    a = radius
    return np.array([[0.0, 0.0, 0.0], [(2.0 + delta) * a, 0.0, 0.0]])


def motion(kind: str):
    """Rigid velocities (v, omega) for two spheres on the x axis."""
    v = np.zeros((2, 3))
    om = np.zeros((2, 3))
    if kind == "squeeze":
        v[0, 0], v[1, 0] = 1.0, -1.0
    elif kind == "shear":
        v[0, 1], v[1, 1] = 1.0, -1.0
    elif kind == "rotate":
        om[0, 2], om[1, 2] = 1.0, -1.0
    elif kind == "cotranslate":
        v[0, 0], v[1, 0] = 1.0, 1.0
    else:
        raise ValueError(kind)
    return v, om


def gap_sweep_gaps(n: int = 18):
    return [10.0 ** (-3.0 + 3.0 * i / (n - 1)) for i in range(n)]


def _ok(c, centres, count, min_dist):
    if count == 0:
        return True
    d = np.linalg.norm(centres[:count] - c[None, :], axis=1)
    return bool(np.all(d >= min_dist))


def _random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def suspension(P: int, phi: float, seed: int, radius: float = 1.0, gap_lo: float = 1e-3,
               gap_hi: float = 1e-1, min_gap: float = 1e-3, seed_frac: float = 0.1,
               double_frac: float = 0.5, max_tries: int = 200000):
    """Centres (P, 3) in a cube [0, L]^3 with L = (P (4/3) pi a^3 / phi)^(1/3)."""
    rng = np.random.default_rng(seed)
    a = radius
    L = (P * 4.0 / 3.0 * math.pi * a ** 3 / phi) ** (1.0 / 3.0)
    centres = np.zeros((P, 3))
    n = 0
    n_seed = max(1, int(round(seed_frac * P)))
    tries = 0
    while n < min(n_seed, P):
        c = rng.uniform(a, L - a, size=3) if L > 2 * a else rng.uniform(0, L, size=3)
        if _ok(c, centres, n, (2.0 + min_gap) * a):
            centres[n] = c
            n += 1
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place seed spheres")
    while n < P:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not grow the suspension")
        i = int(rng.integers(0, n))
        g1 = a * 10.0 ** rng.uniform(math.log10(gap_lo), math.log10(gap_hi))
        c = None
        if n >= 2 and rng.uniform() < double_frac:
            # touch sphere i and its nearest other sphere j at the same time
            d = np.linalg.norm(centres[:n] - centres[i][None, :], axis=1)
            d[i] = np.inf
            j = int(np.argmin(d))
            g2 = a * 10.0 ** rng.uniform(math.log10(gap_lo), math.log10(gap_hi))
            r1, r2 = 2 * a + g1, 2 * a + g2
            dij = d[j]
            if dij < r1 + r2:
                e = (centres[j] - centres[i]) / dij
                x = (dij * dij + r1 * r1 - r2 * r2) / (2 * dij)
                h2 = r1 * r1 - x * x
                if h2 > 0:
                    u = _random_unit(rng)
                    u = u - np.dot(u, e) * e
                    nu = np.linalg.norm(u)
                    if nu > 1e-8:
                        c = centres[i] + x * e + math.sqrt(h2) * u / nu
        if c is None:
            c = centres[i] + (2 * a + g1) * _random_unit(rng)
        if np.any(c < 0.0) or np.any(c > L):
            continue
        if _ok(c, centres, n, (2.0 + min_gap) * a):
            centres[n] = c
            n += 1
    return centres


def tetrahedron(delta: float, radius: float = 1.0):
    """Four spheres on the vertices of a regular tetrahedron, every pair delta (radius units) apart."""
    a = radius
    edge = (2.0 + delta) * a
    v = np.array([[1.0, 1.0, 1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
    return v * (edge / (2.0 * math.sqrt(2.0)))


def cluster(P: int, gap: float, seed: int, radius: float = 1.0, max_tries: int = 100000):
    """P spheres grown one at a time, each placed `gap` from a randomly chosen earlier sphere in
    a random direction and at least `gap` from all others, so that every sphere has a neighbour
    exactly `gap` away."""
    rng = np.random.default_rng(seed)
    a = radius
    centres = np.zeros((P, 3))
    n, tries = 1, 0
    while n < P:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not grow the cluster")
        i = int(rng.integers(0, n))
        c = centres[i] + (2.0 + gap) * a * _random_unit(rng)
        d = np.linalg.norm(centres[:n] - c[None, :], axis=1)
        d[i] = np.inf
        if np.all(d >= (2.0 + gap) * a * (1.0 - 1e-12)):
            centres[n] = c
            n += 1
    return centres


def shear_flow(rate: float = 5.0):
    """Background shear flow of the fixed-cluster example (Sec. 4, Ex. 2) as (U, E, Omega) of
    u_inf(x) = U + E x + Omega x x: E = (rate / 2) [[0, 1, 0], [1, 0, 0], [0, 0, 0]],
    Omega = (0, 0, -rate / 2), i.e. u_inf = (rate y, 0, 0)."""
    E = 0.5 * rate * np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    return np.zeros(3), E, np.array([0.0, 0.0, -0.5 * rate])


def uniform_flow(speed: float = 5.0):
    """Uniform background flow of the same example: u_inf = (speed, 0, 0)."""
    return np.array([speed, 0.0, 0.0]), np.zeros((3, 3)), np.zeros(3)


def rigid_velocities(P: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(P, 3)), rng.normal(size=(P, 3))


def batch(n_problems: int = 64, seed: int = 5, p_lo: int = 2, p_hi: int = 256):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        P = int(round(10.0 ** rng.uniform(math.log10(p_lo), math.log10(p_hi))))
        phi = float(rng.uniform(0.05, 0.3))
        out.append(suspension(P, phi, seed=int(rng.integers(0, 2 ** 31))))
    return out


def count_near_contacts(centres, radius=1.0, cut=0.15):
    c = np.asarray(centres)
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2) / radius - 2.0
    iu = np.triu_indices(c.shape[0], 1)
    g = d[iu]
    return int(np.sum(g < cut)), float(g.min()) if g.size else float("inf")
