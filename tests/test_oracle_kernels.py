"""Pins for the oracle's fundamental solutions against facts outside their formulas.

* The Stokeslet solves the Stokes equations with the textbook pressure
  p = f.r / (4 pi |r|^3), so its 1/(8 pi mu) normalisation and both terms are fixed
  by mu Lap u = grad p and div u = 0 (finite differences).
* The rotlet equals half the curl of the Stokeslet field (the antisymmetric part of
  the force dipole, Sec. 2.3), which fixes its sign and normalisation.
* The potential dipole is minus 1/(4 pi) times the gradient of the scalar d.r/|r|^3
  (a source-sink doublet, eq. doublet), divergence free and harmonic.
"""
import math

import numpy as np

from oracle import kernels

H = 1e-3
X0 = np.array([0.7, -0.4, 1.1])
Y0 = np.array([0.05, 0.1, -0.2])
F0 = np.array([0.3, -1.2, 0.8])


def field(kind, x, strength, visc=1.0):
    r = x - Y0
    if kind == "S":
        return kernels.stokeslet(r, visc) @ strength
    if kind == "R":
        return kernels.rotlet(r, visc) @ strength
    return kernels.dipole(r) @ strength


def grad_vec(fun, x, h=H):
    """J[i, j] = d fun_i / d x_j by 4th-order central differences."""
    J = np.zeros((3, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        J[:, j] = (-fun(x + 2 * e) + 8 * fun(x + e) - 8 * fun(x - e) + fun(x - 2 * e)) / (12 * h)
    return J


def laplacian(fun, x, h=H):
    out = -6.0 * fun(x) * (1 + 0j).real
    acc = 0.0
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        acc = acc + (-fun(x + 2 * e) + 16 * fun(x + e) - 30 * fun(x) + 16 * fun(x - e) - fun(x - 2 * e)) / (12 * h * h)
    return acc


def test_stokeslet_hand_value():
    # r = (1, 2, 2), |r| = 3: S = (I/3 + r r^T / 27) / (8 pi)
    S = kernels.stokeslet(np.array([1.0, 2.0, 2.0]))
    c = 1.0 / (8 * math.pi)
    assert np.isclose(S[0, 0], c * 10 / 27, rtol=1e-14)
    assert np.isclose(S[0, 1], c * 2 / 27, rtol=1e-14)
    assert np.isclose(S[1, 1], c * 13 / 27, rtol=1e-14)
    assert np.isclose(S[1, 2], c * 4 / 27, rtol=1e-14)
    assert np.allclose(S, S.T)


def test_stokeslet_solves_stokes_equations():
    visc = 1.7
    u = lambda x: field("S", x, F0, visc)
    p = lambda x: np.array([np.dot(F0, x - Y0) / (4 * math.pi * np.linalg.norm(x - Y0) ** 3)])
    lap = laplacian(u, X0)
    gp = grad_vec(lambda x: np.repeat(p(x), 3), X0)[0]
    assert np.allclose(visc * lap, gp, rtol=1e-6, atol=1e-8 * np.abs(gp).max())
    assert abs(np.trace(grad_vec(u, X0))) < 1e-9


def test_rotlet_is_half_curl_of_stokeslet():
    J = grad_vec(lambda x: field("S", x, F0), X0)
    curl = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
    assert np.allclose(field("R", X0, F0), 0.5 * curl, rtol=1e-8, atol=1e-12)
    assert abs(np.trace(grad_vec(lambda x: field("R", x, F0), X0))) < 1e-9
    assert np.allclose(laplacian(lambda x: field("R", x, F0), X0), 0.0, atol=1e-7)


def test_rotlet_viscosity_scaling():
    r = np.array([0.3, 0.2, -0.9])
    assert np.allclose(kernels.rotlet(r, 2.0) * 2.0, kernels.rotlet(r, 1.0))


def test_dipole_is_gradient_of_doublet_potential():
    phi = lambda x: np.dot(F0, x - Y0) / np.linalg.norm(x - Y0) ** 3
    g = grad_vec(lambda x: np.repeat(phi(x), 3), X0)[0]
    assert np.allclose(field("D", X0, F0), -g / (4 * math.pi), rtol=1e-8, atol=1e-12)
    assert abs(np.trace(grad_vec(lambda x: field("D", x, F0), X0))) < 1e-9
    assert np.allclose(laplacian(lambda x: field("D", x, F0), X0), 0.0, atol=1e-6)


def test_block_matrix_layout_brute_force():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(4, 3)) * 3
    Y = rng.normal(size=(3, 3)) * 0.2
    lam = rng.normal(size=9)
    for kind in ("S", "R", "D"):
        A = kernels.block_matrix(X, Y, kind, 1.3)
        for i in range(4):
            u = np.zeros(3)
            for j in range(3):
                r = X[i] - Y[j]
                if kind == "S":
                    blk = kernels.stokeslet(r, 1.3)
                elif kind == "R":
                    blk = kernels.rotlet(r, 1.3)
                else:
                    blk = kernels.dipole(r)
                u += blk @ lam[3 * j:3 * j + 3]
            assert np.allclose(A[3 * i:3 * i + 3] @ lam, u, rtol=1e-13)
