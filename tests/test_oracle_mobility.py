"""Pins for the oracle's mobility solve (bordered reading; the paper defers the mobility
formulation to another paper): closed forms for one sphere, consistency with the paper's
resistance formulation, Brenner's squeeze force inverted, reciprocity."""
import math

import numpy as np

from oracle import brenner, geometry, solve
from paper_2407_03343_gb300 import workloads


def test_single_sphere_mobility_closed_form():
    # U = F / (6 pi mu a), Omega = T / (8 pi mu a^3)
    p = geometry.Params(n_proxy=300, r_proxy=0.7, m_basic=400, visc=0.8)
    a = 1.3
    d = geometry.build([[0.5, -1.0, 2.0]], a, p)
    F = np.array([[1.0, -2.0, 0.5]])
    T = np.array([[0.3, 0.2, -1.0]])
    V, W, _ = solve.MobilitySystem(d).solve(F, T)
    assert np.allclose(V, F / (6 * math.pi * 0.8 * a), rtol=1e-5)
    assert np.allclose(W, T / (8 * math.pi * 0.8 * a ** 3), rtol=1e-5)


def test_mobility_is_consistent_with_resistance():
    p = geometry.Params(n_proxy=200, r_proxy=0.7, m_basic=300, nim_fixed=6)
    c = np.array([[0.0, 0.0, 0.0], [1.2, 1.6, 0.5]])
    c[1] *= 2.05 / np.linalg.norm(c[1])
    d = geometry.build(c, 1.0, p)
    ms = solve.MobilitySystem(d)
    rng = np.random.default_rng(3)
    F, T = rng.normal(size=(2, 3)), rng.normal(size=(2, 3))
    V, W, sol = ms.solve(F, T)
    Fc, Tc = solve.forces_torques(d, sol.lam)
    assert np.allclose(Fc, F, atol=1e-9) and np.allclose(Tc, T, atol=1e-9)
    # the paper's resistance formulation driven by these velocities gives back F and T
    r = solve.DenseSystem(d, ms.op).solve(V, W)
    Fr, Tr = solve.forces_torques(d, r.lam)
    assert np.allclose(Fr, F, atol=1e-8) and np.allclose(Tr, T, atol=1e-8)
    # and the mobility matrix is the inverse of the resistance matrix
    Rm = solve.resistance_matrix(d, solve.DenseSystem(d, ms.op))
    u = np.linalg.solve(Rm, np.concatenate([np.r_[F[k], T[k]] for k in range(2)]))
    assert np.allclose(u, np.concatenate([np.r_[V[k], W[k]] for k in range(2)]), atol=1e-8)


def test_squeeze_mobility_inverts_brenner():
    p = geometry.Params(n_proxy=300, r_proxy=0.7, m_basic=600, nim_fixed=10)
    d = geometry.build(workloads.two_spheres(0.1), 1.0, p)
    fb = brenner.squeeze_force(0.1)
    F = np.array([[fb, 0.0, 0.0], [-fb, 0.0, 0.0]])
    V, W, _ = solve.MobilitySystem(d).solve(F, np.zeros((2, 3)))
    assert np.allclose(V, [[1, 0, 0], [-1, 0, 0]], atol=1e-3)
    assert np.abs(W).max() < 1e-3


def test_free_sphere_follows_linear_flow():
    # Faxen's laws for a force- and torque-free sphere in u_inf = U + E x + w x x:
    # V = u_inf(c), Omega = w + curl(E x) / 2, with curl(E x)_i = eps_ijk E_kj
    p = geometry.Params(n_proxy=300, r_proxy=0.7, m_basic=400)
    c = np.array([0.4, -0.7, 1.1])
    d = geometry.build([c], 1.0, p)
    U = np.array([0.2, -0.1, 0.3])
    E = np.array([[0.1, 1.0, -0.3], [0.2, -0.4, 0.5], [0.0, 0.7, 0.3]])
    w = np.array([0.3, -0.2, 0.6])
    bg = solve.Background(U=U, E=E, omega=w)
    zero = np.zeros((1, 3))
    V, W, _ = solve.MobilitySystem(d).solve(zero, zero, bg)
    curl = np.array([E[2, 1] - E[1, 2], E[0, 2] - E[2, 0], E[1, 0] - E[0, 1]])
    assert np.allclose(V[0], U + E @ c + np.cross(w, c), atol=1e-6)
    assert np.allclose(W[0], w + 0.5 * curl, atol=1e-6)
