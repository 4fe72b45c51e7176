"""Pins for the oracle's discretisation (Sec. 2.1, Sec. 2.3, Sec. 5.1)."""
import math

import numpy as np
import pytest

from oracle import geometry as g


def kelvin(x, c):
    """eq. reflect written as the classical inversion in a unit sphere about c."""
    d = x - c
    return c + d / np.dot(d, d)


@pytest.mark.parametrize("rp", [0.5, 0.6, 0.63, 0.7, 0.8])
def test_racc_at_critical_gap_is_proxy_radius(rp):
    assert math.isclose(g.r_acc(g.delta_star(rp)), rp, rel_tol=1e-13)


def test_delta_star_printed_value():
    # Sec. 3 prints delta* ~ 0.129 for R_p = 0.7.
    assert abs(g.delta_star(0.7) - 0.129) < 5e-4


@pytest.mark.parametrize("delta", [1e-3, 1e-2, 0.1, 0.5])
def test_accumulation_point_is_fixed_point_of_reflections(delta):
    c1 = np.zeros(3)
    c2 = np.array([2.0 + delta, 0.0, 0.0])
    x = c2.copy()
    for _ in range(4000):
        x = kelvin(x, c1)      # image in sphere 1
        x = kelvin(x, c2)      # image of that in sphere 2
    x1 = kelvin(x, c1)
    assert math.isclose(np.linalg.norm(x1 - c1), g.r_acc(delta), rel_tol=1e-9)
    # eq. acc_points: midpoint minus sqrt(delta + delta^2/4) along the axis
    xacc = 0.5 * (c1 + c2) - math.sqrt(delta + delta * delta / 4) * (c2 - c1) / np.linalg.norm(c2 - c1)
    assert np.allclose(x1, xacc, atol=1e-9)


def test_image_count_rule():
    p = g.Params()
    # eq. image_est by hand: ceil(-8.72 log10(delta) - 6.15)
    assert g.n_images(1e-2, p) == 12          # 17.44 - 6.15 = 11.29
    assert g.n_images(0.05, p) == 6           # 11.345 - 6.15 = 5.195
    assert g.n_images(0.1, p) == 3            # 8.72 - 6.15 = 2.57
    assert g.n_images(0.149, p) == 2
    assert g.n_images(0.15, p) == 0
    assert g.n_images(0.3, p) == 0
    assert g.n_images(1e-3, p) == 20          # 20.01 -> 21, capped at 20 (Sec. 5.1 text)
    q = g.Params(nim_fixed=10)
    assert g.n_images(0.1, q) == 10 and g.n_images(0.2, q) == 0
    # opt-in lower bound (not in the paper): applies below nim_cut only, the rule still wins above it
    m = g.Params(nim_cut=0.3, nim_min=2)
    assert g.n_images(0.2, m) == 2 and g.n_images(0.29, m) == 2 and g.n_images(0.3, m) == 0
    assert g.n_images(0.1, m) == 3 and g.n_images(1e-2, m) == 12


def test_image_radii_half_chebyshev():
    p = g.Params(r_proxy=0.63)
    for delta in (1e-3, 1e-2, 0.1):
        n = g.n_images(delta, p)
        t = g.image_radii(delta, n, p)
        assert math.isclose(t[0], g.r_acc(delta), rel_tol=1e-14)
        assert np.all(np.diff(t) < 0)
        assert t[-1] > p.r_proxy * (1 + p.delta_offset)
        assert t[0] < 1.0
        # equal steps in the Chebyshev angle
        th = np.arccos((t - p.r_proxy * 1.05) / (t[0] - p.r_proxy * 1.05))
        assert np.allclose(np.diff(th), math.pi / (2 * n), atol=1e-7)


def test_fibonacci_sphere():
    x = g.fibonacci_sphere(800)
    assert x.shape == (800, 3)
    assert np.allclose(np.linalg.norm(x, axis=1), 1.0)
    assert np.linalg.norm(x.mean(axis=0)) < 2.0 / 800
    # second moments of a uniform distribution on the sphere: E[x x^T] = I/3
    assert np.allclose(x.T @ x / 800, np.eye(3) / 3, atol=5e-3)


def test_cap_nodes_and_weights():
    p = g.Params(n_proxy=100, m_basic=150)
    delta = 1e-2
    centres = np.array([[0.0, 0.0, 0.0], [0.3, 2.0 + delta, 0.1]])
    centres[1] = centres[1] / np.linalg.norm(centres[1]) * (2 + delta)
    a = 1.5
    d = g.build(centres * a, a, p)
    n = g.n_images(delta, p)
    assert len(d.contacts) == 1 and d.contacts[0].n_im == n
    sp = d.spheres[0]
    m = 18 * n
    # eq. colloc_nbr / eq. Mest
    assert sp.colloc.shape[0] == p.m_basic + 2 * m
    assert sp.image.shape[0] == n
    assert np.allclose(np.linalg.norm(sp.colloc - sp.centre, axis=1), a)
    e = (d.spheres[1].centre - sp.centre) / np.linalg.norm(d.spheres[1].centre - sp.centre)
    for cap, beta in ((0, p.beta1), (1, p.beta2)):
        pts = sp.colloc[p.m_basic + cap * m: p.m_basic + (cap + 1) * m]
        cos_t = (pts - sp.centre) @ e / a
        assert np.all(cos_t >= math.cos(beta) - 1e-12)
        assert math.isclose(cos_t.min(), math.cos(beta), rel_tol=1e-12)
    # weights: the basic grid covers the sphere area, each cap its own area
    w = sp.weight
    assert math.isclose(w[:p.m_basic].sum(), 4 * math.pi * a * a, rel_tol=1e-12)
    assert math.isclose(w[p.m_basic:p.m_basic + m].sum(), 2 * math.pi * a * a * (1 - math.cos(p.beta1)), rel_tol=1e-12)
    # image nodes on the centre-centre line at radii t_j a
    t = g.image_radii(delta, n, p)
    assert np.allclose(sp.image, sp.centre + a * t[:, None] * e[None, :])
    # the partner's images point the other way
    assert np.allclose(d.spheres[1].image, d.spheres[1].centre - a * t[:, None] * e[None, :])


def test_tetrahedron_counts():
    # each sphere of a regular tetrahedron with gap 1e-3 has 3 contacts of n_im = 20:
    # M^(k) = M0 + 2 * 6 * 3 * 3 * 20 (eq. Mest) and N^(k) = N + 3 * 3 * 20 (eq. Nk)
    s = 2.001
    pts = np.array([[0, 0, 0], [s, 0, 0], [s / 2, s * math.sqrt(3) / 2, 0],
                    [s / 2, s / (2 * math.sqrt(3)), s * math.sqrt(2.0 / 3.0)]])
    p = g.Params(n_proxy=50, m_basic=60)
    d = g.build(pts, 1.0, p)
    assert len(d.contacts) == 6
    for sp in d.spheres:
        assert sp.colloc.shape[0] == 60 + 2160
        assert sp.image.shape[0] == 60


def test_overlap_rejected():
    with pytest.raises(ValueError):
        g.build([[0, 0, 0], [1.9, 0, 0]], 1.0, g.Params(n_proxy=20, m_basic=30))
