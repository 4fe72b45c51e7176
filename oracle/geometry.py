"""Discretisation of P equal spheres (oracle side, FP64, numpy).

Follows the paper's recipe:
  * basic proxy and collocation grids (Sec. 2.1): N proxy Stokeslets on a concentric
    sphere of radius R_p, M0 collocation nodes on the surface.  The paper uses
    spherical designs, which are not available here; quasi-uniform Fibonacci grids
    (the paper's own alternative, Sec. 2.1, and the cap construction eq. thetacap
    with a full opening) replace them.
  * contacts and image lines (Sec. 2.3): accumulation radius eq. Racc, critical gap
    eq. deltastar, image nodes eq. line_points / eq. tj.
  * adaptive image count eq. image_est and collocation caps eq. colloc_nbr /
    eq. thetacap (Sec. 5.1), area weights of the left preconditioner
    (Sec. 5.1, remark left-precond).

Readings of ambiguous passages (all listed in the design notes):
  * eq. thetacap is read as cos(theta_j) = 1 - j (1 - cos beta) / M, j = 1..M, i.e. a
    cap of half-angle beta about the contact axis (the printed cos(beta)/M makes
    every cap nearly a hemisphere, contradicting Fig. sweep_cone).
  * the full-sphere Fibonacci grid uses the midpoint rule
    cos(theta_j) = 1 - (2j - 1)/n, phi_j = 2 pi j / Phi mod 2 pi, j = 1..n.
  * eq. image_est is capped at nim_max = 20 (the text states 20 suffice for
    delta >= 1e-3, while the formula gives 21 there).
  * eq. tj is applied as printed whenever n_im > 0, also when
    R_acc < R_p (1 + Delta) (then the nodes lie just outside R_acc, still inside
    the sphere).
  * area weights: basic node 4 pi a^2 / M0; cap node 2 pi a^2 (1 - cos beta) / M_cap.
  * the contact frame (e1, e2, e) about the unit axis e: h = e_z if |e_z| <= 0.9
    else e_x, e1 = normalise(h - (h.e) e), e2 = e x e1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

GOLDEN_RATIO = (1.0 + math.sqrt(5.0)) / 2.0


@dataclass
class Params:
    """Discretisation parameters; defaults are the paper's coarse choice (Sec. 3, Sec. 5.1)."""
    n_proxy: int = 686            # N, proxy Stokeslets per sphere
    r_proxy: float = 0.63         # R_p (radius units)
    m_basic: int = 823            # M0 ~ 1.2 N basic collocation nodes
    delta_offset: float = 0.05    # Delta in eq. tj
    alpha1: int = 6               # cap upsampling, eq. colloc_nbr
    alpha2: int = 6
    beta1: float = math.pi / 5    # cap half-angles (Sec. 5.1)
    beta2: float = math.pi / 60
    eps_trunc: float = 5e-12      # relative SVD truncation (Sec. 5, App. A.1)
    nim_a: float = 8.72           # eq. image_est constants
    nim_b: float = 6.15
    nim_cut: float = 0.15
    nim_max: int = 20
    nim_fixed: int = -1           # >= 0 forces n_im for every contact with gap < nim_cut
    nim_min: int = 0              # lower bound on n_im below nim_cut (0: eq. image_est as printed)
    left_precond: int = 1         # row scaling W (Sec. 5.1 remark left-precond)
    visc: float = 1.0             # viscosity mu
    n_check: int = 500            # check points per sphere for eps_res (Sec. 4)


def fibonacci_sphere(n: int) -> np.ndarray:
    """n quasi-uniform unit vectors (Fibonacci grid, midpoint rule in cos(theta))."""
    j = np.arange(1, n + 1, dtype=np.float64)
    cos_t = 1.0 - (2.0 * j - 1.0) / n
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = np.mod(2.0 * math.pi * j / GOLDEN_RATIO, 2.0 * math.pi)
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def cap_directions(m: int, beta: float) -> np.ndarray:
    """eq. thetacap (reading: half-angle beta): m unit vectors in the frame whose third
    axis is the contact axis, columns (e1, e2, e) coefficients."""
    j = np.arange(1, m + 1, dtype=np.float64)
    cos_t = 1.0 - j * (1.0 - math.cos(beta)) / m
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = np.mod(2.0 * math.pi * j / GOLDEN_RATIO, 2.0 * math.pi)
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def contact_frame(e: np.ndarray):
    """Orthonormal (e1, e2) perpendicular to the unit axis e (reading in module doc)."""
    h = np.array([0.0, 0.0, 1.0]) if abs(e[2]) <= 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = h - np.dot(h, e) * e
    e1 = e1 / np.linalg.norm(e1)
    e2 = np.cross(e, e1)
    return e1, e2


def r_acc(delta: float) -> float:
    """eq. Racc: distance from a unit sphere's centre to its accumulation point."""
    return 1.0 + delta / 2.0 - math.sqrt(delta + delta * delta / 4.0)


def delta_star(rp: float) -> float:
    """eq. deltastar: the gap at which R_acc equals R_p."""
    return (1.0 - rp) ** 2 / rp


def n_images(delta: float, p: Params) -> int:
    """eq. image_est, capped at nim_max (or forced to nim_fixed)."""
    if delta >= p.nim_cut:
        return 0
    if p.nim_fixed >= 0:
        return int(p.nim_fixed)
    n = max(math.ceil(-p.nim_a * math.log10(delta) - p.nim_b), p.nim_min)
    return int(min(max(n, 0), p.nim_max))


def image_radii(delta: float, n_im: int, p: Params) -> np.ndarray:
    """eq. tj: n_im distances t_j (unit sphere) from the centre along the contact axis."""
    t0 = p.r_proxy * (1.0 + p.delta_offset)
    j = np.arange(1, n_im + 1, dtype=np.float64)
    return t0 + (r_acc(delta) - t0) * np.cos((j - 1.0) / (2.0 * n_im) * math.pi)


@dataclass
class Contact:
    k: int          # lower sphere index
    kp: int         # higher sphere index
    delta: float    # gap in radius units
    n_im: int


@dataclass
class Sphere:
    centre: np.ndarray
    colloc: np.ndarray          # (M_k, 3) collocation nodes
    weight: np.ndarray          # (M_k,) area weights w_i
    proxy: np.ndarray           # (N, 3) proxy Stokeslet positions
    image: np.ndarray           # (n_img_k, 3) image nodes (each carries S, R and D)
    partners: list = field(default_factory=list)


@dataclass
class Discretisation:
    params: Params
    radius: float
    centres: np.ndarray
    contacts: list
    spheres: list
    check: list                 # per sphere (n_check, 3) check points


def find_contacts(centres: np.ndarray, a: float, p: Params):
    """All pairs with gap < nim_cut that receive images; raises on overlap."""
    P = centres.shape[0]
    out = []
    for k in range(P):
        for kp in range(k + 1, P):
            d = float(np.linalg.norm(centres[kp] - centres[k]))
            delta = d / a - 2.0
            if delta <= 0.0:
                raise ValueError(f"spheres {k} and {kp} overlap or touch (gap {delta})")
            n = n_images(delta, p)
            if n > 0:
                out.append(Contact(k, kp, delta, n))
    return out


def build(centres, radius: float = 1.0, p: Params | None = None) -> Discretisation:
    """Build the full discretisation for spheres of equal radius at ``centres``."""
    p = p or Params()
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    a = float(radius)
    P = centres.shape[0]
    contacts = find_contacts(centres, a, p)
    basic_c = fibonacci_sphere(p.m_basic)
    basic_p = fibonacci_sphere(p.n_proxy)
    chk = fibonacci_sphere(p.n_check)[:, [1, 2, 0]]   # axis-permuted so it differs from the collocation grid
    w_basic = 4.0 * math.pi * a * a / p.m_basic
    spheres, check = [], []
    per = [[] for _ in range(P)]
    for c in contacts:
        per[c.k].append((c.kp, c))
        per[c.kp].append((c.k, c))
    for k in range(P):
        ck = centres[k]
        X = [ck + a * basic_c]
        W = [np.full(p.m_basic, w_basic)]
        imgs = []
        partners = sorted(per[k], key=lambda t: t[0])
        for kp, c in partners:
            e = centres[kp] - ck
            e = e / np.linalg.norm(e)
            e1, e2 = contact_frame(e)
            t = image_radii(c.delta, c.n_im, p)
            imgs.append(ck + a * t[:, None] * e[None, :])
            for alpha, beta in ((p.alpha1, p.beta1), (p.alpha2, p.beta2)):
                m = int(alpha) * 3 * c.n_im
                d = cap_directions(m, beta)
                X.append(ck + a * (d[:, :1] * e1 + d[:, 1:2] * e2 + d[:, 2:3] * e))
                W.append(np.full(m, 2.0 * math.pi * a * a * (1.0 - math.cos(beta)) / m))
        spheres.append(Sphere(
            centre=ck.copy(),
            colloc=np.concatenate(X, axis=0),
            weight=np.concatenate(W),
            proxy=ck + a * p.r_proxy * basic_p,
            image=np.concatenate(imgs, axis=0) if imgs else np.zeros((0, 3)),
            partners=[kp for kp, _ in partners],
        ))
        check.append(ck + a * chk)
    return Discretisation(params=p, radius=a, centres=centres, contacts=contacts,
                          spheres=spheres, check=check)
