"""Pins for the oracle's MFS solves against closed forms, Brenner's series,
reciprocal-theorem invariants and brute force."""
import math

import numpy as np
import pytest

from oracle import brenner, geometry, kernels, solve
from paper_2407_03343_gb300 import workloads


def small(**kw):
    base = dict(n_proxy=300, r_proxy=0.7, m_basic=400)
    base.update(kw)
    return geometry.Params(**base)


@pytest.mark.parametrize("a", [1.0, 2.0])
def test_single_sphere_drag_and_torque(a):
    # Stokes drag 6 pi mu a U and torque 8 pi mu a^3 Omega (force on the fluid, Sec. 2.3 remark)
    p = small(visc=1.3)
    d = geometry.build([[0.5, -1.0, 2.0]], a, p)
    U = np.array([[0.3, -0.7, 1.1]])
    W = np.array([[-0.4, 0.2, 0.9]])
    sol = solve.solve_o2(d, U, W)
    F, T = solve.forces_torques(d, sol.lam)
    assert np.allclose(F, 6 * math.pi * 1.3 * a * U, rtol=1e-5, atol=1e-5 * np.abs(6 * math.pi * 1.3 * a * U).max())
    assert np.allclose(T, 8 * math.pi * 1.3 * a ** 3 * W, rtol=1e-5, atol=1e-5 * np.abs(8 * math.pi * 1.3 * a ** 3 * W).max())
    assert solve.residual_max(d, sol.lam, U, W) < 1e-3


def test_single_sphere_exterior_flow_is_exact_solution():
    # translating sphere: u = (3a/4)(U/r + (U.r) r/r^3) + (a^3/4)(U/r^3 - 3 (U.r) r/r^5)
    p = small()
    d = geometry.build([[0.0, 0.0, 0.0]], 1.0, p)
    U = np.array([[1.0, 0.5, -0.2]])
    sol = solve.solve_o2(d, U, np.zeros((1, 3)))
    x = np.array([[1.5, 0.2, 0.1], [0.0, 3.0, 0.0], [-2.0, -2.0, 1.0]])
    u = solve.velocity(d, sol.lam, x)
    r = np.linalg.norm(x, axis=1)[:, None]
    ur = (x @ U[0])[:, None]
    exact = 0.75 * (U / r + ur * x / r ** 3) + 0.25 * (U / r ** 3 - 3 * ur * x / r ** 5)
    assert np.allclose(u, exact, atol=2e-5)


def test_squeeze_force_matches_brenner_with_images():
    # config of the plain-method case: gap 0.1, R_p = 0.7, 10 image points per line
    p = geometry.Params(n_proxy=300, r_proxy=0.7, m_basic=600, nim_fixed=10)
    d = geometry.build(workloads.two_spheres(0.1), 1.0, p)
    v, om = workloads.motion("squeeze")
    sol = solve.solve_o2(d, v, om)
    F, _ = solve.forces_torques(d, sol.lam)
    fb = brenner.squeeze_force(0.1)
    assert abs(F[0, 0] - fb) / fb < 1e-3
    assert abs(F[1, 0] + fb) / fb < 1e-3
    assert abs(F[0, 1]) + abs(F[0, 2]) < 1e-3 * fb


def test_images_are_needed_at_small_gap():
    # without images the proxy sphere cannot resolve squeezing at delta = 0.02 (Sec. 3)
    v, om = workloads.motion("squeeze")
    fb = brenner.squeeze_force(0.02)
    errs = []
    for nim in (0, 10):
        p = geometry.Params(n_proxy=300, r_proxy=0.7, m_basic=500, nim_fixed=nim)
        d = geometry.build(workloads.two_spheres(0.02), 1.0, p)
        sol = solve.solve_o2(d, v, om)
        F, _ = solve.forces_torques(d, sol.lam)
        errs.append(abs(F[0, 0] - fb) / fb)
    assert errs[1] < 1e-3 < errs[0]


def test_resistance_matrix_symmetric_positive_definite():
    p = geometry.Params(n_proxy=200, r_proxy=0.7, m_basic=300, nim_fixed=6)
    c = np.array([[0.0, 0.0, 0.0], [1.2, 1.6, 0.5]])
    c[1] *= 2.05 / np.linalg.norm(c[1])
    d = geometry.build(c, 1.0, p)
    Rm = solve.resistance_matrix(d)
    assert np.abs(Rm - Rm.T).max() < 2e-3 * np.abs(Rm).max()
    assert np.linalg.eigvalsh(0.5 * (Rm + Rm.T)).min() > 0
    # swapping the spheres permutes the matrix (pair symmetry)
    d2 = geometry.build(c[::-1].copy(), 1.0, p)
    Rm2 = solve.resistance_matrix(d2)
    perm = np.r_[6:12, 0:6]
    assert np.abs(Rm2 - Rm[np.ix_(perm, perm)]).max() < 2e-3 * np.abs(Rm).max()


def test_o1_o2_o3_agree():
    p = geometry.Params(n_proxy=200, r_proxy=0.7, m_basic=300, nim_fixed=6)
    d = geometry.build(workloads.two_spheres(0.1), 1.0, p)
    v = np.array([[0.3, 1.0, -0.2], [-0.5, 0.1, 0.4]])
    om = np.array([[0.2, -0.3, 1.0], [0.0, 0.6, -0.1]])
    s2 = solve.solve_o2(d, v, om)
    s3 = solve.solve_o3(d, v, om, tol=1e-9)
    s1 = solve.solve_o1(d, v, om)
    F2, T2 = solve.forces_torques(d, s2.lam)
    F3, T3 = solve.forces_torques(d, s3.lam)
    F1, T1 = solve.forces_torques(d, s1.lam)
    ft = np.abs(np.r_[F2.ravel(), T2.ravel()]).max()
    # same formulation: agree to the GMRES tolerance
    assert np.abs(np.r_[F3.ravel(), T3.ravel()] - np.r_[F2.ravel(), T2.ravel()]).max() < 1e-6 * ft
    # different approximations (Sec. 2.2): agree to the discretisation error
    assert np.abs(np.r_[F1.ravel(), T1.ravel()] - np.r_[F2.ravel(), T2.ravel()]).max() < 1e-3 * ft
    x = d.check[0]
    u1 = solve.velocity(d, s1.lam, x)
    u2 = solve.velocity(d, s2.lam, x)
    assert np.abs(u1 - u2).max() < 1e-2 * np.abs(u2).max()


def test_three_step_apply_brute_force():
    # tiny problem: G_hat mu built from explicit loops over node/source pairs
    p = geometry.Params(n_proxy=8, r_proxy=0.6, m_basic=12, nim_fixed=1, alpha1=1, alpha2=1)
    d = geometry.build(workloads.two_spheres(0.05), 1.0, p)
    op = solve.Operator(d)
    rng = np.random.default_rng(1)
    mu = rng.normal(size=op.n)
    out = op.apply(mu)
    mus = op.split(mu)
    lam_hat = [solve.pinv_apply(op.f[k], mus[k]) for k in range(2)]
    ref = []
    for k in range(2):
        sp = d.spheres[k]
        w = np.sqrt(sp.weight)
        uk = np.zeros((sp.colloc.shape[0], 3))
        kp = 1 - k
        q = d.spheres[kp]
        f, t, dd = solve.split_strengths(d, kp, lam_hat[kp])
        yS = np.concatenate([q.proxy, q.image])
        for i, x in enumerate(sp.colloc):
            for j, y in enumerate(yS):
                uk[i] += kernels.stokeslet(x - y) @ f[j]
            for j, y in enumerate(q.image):
                uk[i] += kernels.rotlet(x - y) @ t[j] + kernels.dipole(x - y) @ dd[j]
        ref.append(mus[k] + (w[:, None] * uk).ravel())
    assert np.allclose(out, np.concatenate(ref), rtol=1e-10, atol=1e-12 * np.abs(out).max())


def test_truncation_drops_small_singular_values():
    p = geometry.Params(n_proxy=200, r_proxy=0.7, m_basic=300, nim_fixed=10)
    d = geometry.build(workloads.two_spheres(0.05), 1.0, p)
    B = solve.scaled_block(d, 0, 0)
    s = np.linalg.svd(B, compute_uv=False)
    f = solve.one_body_factor(B, 5e-12)
    assert f.s.shape[0] == int(np.sum(s >= 5e-12 * s[0])) < s.shape[0]
    # the pseudo-inverse is a left inverse on the retained range
    lam = f.V @ np.random.default_rng(2).normal(size=f.s.shape[0])
    assert np.allclose(solve.pinv_apply(f, B @ lam), lam, atol=1e-6 * np.abs(lam).max())


def test_translation_invariance_and_linearity():
    p = geometry.Params(n_proxy=150, r_proxy=0.7, m_basic=220, nim_fixed=4)
    c = workloads.two_spheres(0.08)
    d1 = geometry.build(c, 1.0, p)
    d2 = geometry.build(c + np.array([3.0, -7.0, 11.0]), 1.0, p)
    sys1 = solve.DenseSystem(d1)
    sys2 = solve.DenseSystem(d2)
    v1, o1 = workloads.motion("shear")
    v2, o2 = workloads.motion("rotate")
    a = solve.forces_torques(d1, sys1.solve(v1, o1).lam)
    b = solve.forces_torques(d2, sys2.solve(v1, o1).lam)
    assert np.allclose(np.r_[a[0], a[1]], np.r_[b[0], b[1]], atol=1e-8 * np.abs(np.r_[a[0], a[1]]).max())
    c12 = solve.forces_torques(d1, sys1.solve(v1 + 2 * v2, o1 + 2 * o2).lam)
    c2 = solve.forces_torques(d1, sys1.solve(v2, o2).lam)
    assert np.allclose(c12[0], a[0] + 2 * c2[0], atol=1e-8 * np.abs(c12[0]).max())


def test_fixed_sphere_in_background_flow():
    # a sphere held fixed in u_inf = U + w x (x - c) feels the flow as if it moved with -U and
    # rotated with -w: F = -6 pi mu a U, T = -8 pi mu a^3 w (on the fluid); in a pure strain
    # about its centre it exerts neither force nor torque
    p = small(visc=0.7)
    c = np.array([0.3, -0.2, 0.5])
    d = geometry.build([c], 1.0, p)
    U = np.array([0.4, -0.3, 0.8])
    w = np.array([0.2, 0.5, -0.6])
    zero = np.zeros((1, 3))
    # rotation about the sphere's centre: w x (x - c) = w x x - w x c
    bg = solve.Background(U=U - np.cross(w, c), omega=w)
    sol = solve.solve_o2(d, zero, zero, bg)
    F, T = solve.forces_torques(d, sol.lam)
    assert np.allclose(F[0], -6 * math.pi * 0.7 * U, atol=1e-5 * 6 * math.pi * 0.7)
    assert np.allclose(T[0], -8 * math.pi * 0.7 * w, atol=1e-5 * 8 * math.pi * 0.7)
    E = np.array([[0.3, 0.2, 0.0], [0.2, -0.1, 0.4], [0.0, 0.4, -0.2]])   # symmetric, traceless
    sol = solve.solve_o2(d, zero, zero, solve.Background(U=-E @ c, E=E))
    F, T = solve.forces_torques(d, sol.lam)
    scale = 6 * math.pi * 0.7 * np.abs(E).max()   # drag scale of the strain velocities
    assert np.abs(F).max() < 1e-5 * scale and np.abs(T).max() < 1e-5 * scale


def test_rotating_sphere_exterior_flow_is_exact_solution():
    # rotating sphere: u = (a / r)^3 Omega x r
    p = small()
    a = 1.2
    d = geometry.build([[0.0, 0.0, 0.0]], a, p)
    W = np.array([[0.3, -0.8, 0.5]])
    sol = solve.solve_o2(d, np.zeros((1, 3)), W)
    x = np.array([[1.8, 0.3, -0.2], [0.0, 0.0, 3.0], [-2.5, 1.5, 1.0]])
    u = solve.velocity(d, sol.lam, x)
    r = np.linalg.norm(x, axis=1)[:, None]
    exact = (a / r) ** 3 * np.cross(W, x)
    assert np.allclose(u, exact, atol=2e-5 * np.abs(W).max())


def test_minimum_images_close_the_image_free_window():
    # at gap 0.2 the printed rule places no images and the coarse proxy sphere alone misses the
    # 1e-3 residual target; two images per sphere bring it below (plain least squares, O1)
    kw = dict(n_proxy=686, r_proxy=0.63, m_basic=823)
    rng = np.random.default_rng(2)
    v, w = rng.normal(size=(2, 3)), rng.normal(size=(2, 3))
    c = workloads.two_spheres(0.2)
    d0 = geometry.build(c, 1.0, geometry.Params(**kw))
    d2 = geometry.build(c, 1.0, geometry.Params(nim_cut=0.3, nim_min=2, **kw))
    assert sum(s.image.shape[0] for s in d0.spheres) == 0 and all(s.image.shape[0] == 2 for s in d2.spheres)
    e0 = solve.residual_max(d0, solve.solve_o1(d0, v, w).lam, v, w)
    e2 = solve.residual_max(d2, solve.solve_o1(d2, v, w).lam, v, w)
    assert e0 > 3e-3 and e2 < 5e-4
