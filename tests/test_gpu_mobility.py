"""Mobility solve on the GPU (prescribed forces and torques, velocities found) against the
oracle's dense bordered solve, through the C ABI.

Tolerances: velocities within 1e-5 of the largest velocity (the force/torque target of the
resistance tests carried through the O(1) mobility matrix), with the GPU solve converged to
1e-9 (FP64) / 1e-8 (MIXED) so that the solver tolerance does not dominate.
"""
import math

import numpy as np
import pytest

from oracle import geometry, solve
from paper_2407_03343_gb300 import mfs, workloads

pytestmark = pytest.mark.gpu

C1 = dict(n_proxy=300, r_proxy=0.7, m_basic=600, nim_fixed=10)
TOL = {"fp64": 1e-9, "mixed": 1e-8}


def pair_centres():
    c = np.array([[0.0, 0.0, 0.0], [1.2, 1.6, 0.5]])
    c[1] *= 2.1 / np.linalg.norm(c[1])
    return c


@pytest.fixture(scope="module")
def pair():
    c = pair_centres()
    ctx = mfs.Context(0)
    ctx.set_spheres(c)
    ctx.build(**C1)
    d = geometry.build(c, 1.0, geometry.Params(**C1))
    ms = solve.MobilitySystem(d)
    yield ctx, d, ms
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_sphere_mobility_closed_form(prec):
    visc, a = 0.8, 1.3
    ctx = mfs.Context(0)
    ctx.set_spheres([[0.5, -1.0, 2.0]], radius=a)
    ctx.build(n_proxy=300, r_proxy=0.7, m_basic=400, visc=visc)
    F = np.array([[1.0, -2.0, 0.5]])
    T = np.array([[0.3, 0.2, -1.0]])
    ctx.set_forces_torques(F, T)
    ctx.solve(precision=prec, tol=TOL[prec])
    V, W = ctx.rigid_velocities()
    ctx.close()
    assert np.allclose(V, F / (6 * math.pi * visc * a), rtol=1e-5)
    assert np.allclose(W, T / (8 * math.pi * visc * a ** 3), rtol=1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pair_mobility_matches_oracle(pair, prec):
    ctx, d, ms = pair
    rng = np.random.default_rng(5)
    F, T = rng.normal(size=(2, 3)), rng.normal(size=(2, 3))
    Vr, Wr, _ = ms.solve(F, T)
    ctx.set_forces_torques(F, T)
    info = ctx.solve(precision=prec, tol=TOL[prec])
    assert info.converged
    V, W = ctx.rigid_velocities()
    scale = max(np.abs(Vr).max(), np.abs(Wr).max())
    assert np.abs(V - Vr).max() <= 1e-5 * scale
    assert np.abs(W - Wr).max() <= 1e-5 * scale
    # the forces and torques of the solution are the prescribed ones
    Fc, Tc = ctx.forces_torques()
    assert np.abs(Fc - F).max() <= 1e-6 * np.abs(F).max()
    assert np.abs(Tc - T).max() <= 1e-6 * np.abs(T).max()


def test_pair_mobility_in_background_flow(pair):
    # force- and torque-free pair in a shear flow
    ctx, d, ms = pair
    E = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    zero = np.zeros((2, 3))
    Vr, Wr, _ = ms.solve(zero, zero, solve.Background(E=E))
    ctx.set_background_flow(E=E)
    try:
        ctx.set_forces_torques(zero, zero)
        ctx.solve(precision="mixed", tol=1e-8)
        V, W = ctx.rigid_velocities()
    finally:
        ctx.set_background_flow()
    scale = max(np.abs(Vr).max(), np.abs(Wr).max())
    assert np.abs(V - Vr).max() <= 1e-5 * scale
    assert np.abs(W - Wr).max() <= 1e-5 * scale


def test_resistance_then_mobility_round_trip():
    # five spheres with near contacts (smallest gap 1.1e-3): the forces and torques of a
    # resistance solve, prescribed in the mobility solve, give back the velocities (both on the
    # GPU; the dense oracle is not accurate enough on clusters).  This direction is the
    # well-conditioned one: the mobility matrix is bounded, while the resistance matrix grows
    # like 1/gap and would amplify the solver tolerance by ~4e3 in the other direction.
    c = workloads.suspension(5, 0.15, seed=11)
    ctx = mfs.Context(0)
    ctx.set_spheres(c)
    ctx.build(n_proxy=260, r_proxy=0.63, m_basic=420)
    rng = np.random.default_rng(7)
    V, W = rng.normal(size=(5, 3)), rng.normal(size=(5, 3))
    ctx.set_rigid_velocities(V, W)
    assert ctx.solve(precision="mixed", tol=1e-9, max_iter=2000).converged
    F, T = ctx.forces_torques()
    ctx.set_forces_torques(F, T)
    assert ctx.solve(precision="mixed", tol=1e-9, max_iter=2000).converged
    Vm, Wm = ctx.rigid_velocities()
    ctx.close()
    scale = max(np.abs(V).max(), np.abs(W).max())
    assert np.abs(Vm - V).max() <= 1e-5 * scale
    assert np.abs(Wm - W).max() <= 1e-5 * scale


def test_mobility_errors(pair):
    ctx, _, _ = pair
    ctx.set_rigid_velocities(np.zeros((2, 3)), np.zeros((2, 3)))
    with pytest.raises(mfs.MfsError, match="STATE"):
        ctx.rigid_velocities()
    with pytest.raises(mfs.MfsError, match="ARG"):
        ctx.set_forces_torques(np.full((2, 3), np.nan), np.zeros((2, 3)))
    ctx.set_forces_torques(np.ones((2, 3)), np.zeros((2, 3)))
    with pytest.raises(mfs.MfsError, match="UNSUPPORTED"):
        ctx.solve(precision="fp32")
    with pytest.raises(mfs.MfsError, match="UNSUPPORTED"):
        mfs.batch_solve([ctx], precision="fp32")
    # zero data: the solve returns zero velocities without iterating
    ctx.set_forces_torques(np.zeros((2, 3)), np.zeros((2, 3)))
    info = ctx.solve(precision="mixed")
    assert info.converged and info.iters == 0
    V, W = ctx.rigid_velocities()
    assert not V.any() and not W.any()


def test_free_sphere_follows_linear_flow():
    # Faxen's laws: V = u_inf(c), Omega = w + curl(E x) / 2 for a force- and torque-free sphere
    c = np.array([0.4, -0.7, 1.1])
    U = np.array([0.2, -0.1, 0.3])
    E = np.array([[0.1, 1.0, -0.3], [0.2, -0.4, 0.5], [0.0, 0.7, 0.3]])
    w = np.array([0.3, -0.2, 0.6])
    ctx = mfs.Context(0)
    ctx.set_spheres([c])
    ctx.build(n_proxy=300, r_proxy=0.7, m_basic=400)
    ctx.set_background_flow(U, E, w)
    ctx.set_forces_torques(np.zeros((1, 3)), np.zeros((1, 3)))
    assert ctx.solve(precision="mixed", tol=1e-9).converged
    V, W = ctx.rigid_velocities()
    ctx.close()
    curl = np.array([E[2, 1] - E[1, 2], E[0, 2] - E[2, 0], E[1, 0] - E[0, 1]])
    assert np.allclose(V[0], U + E @ c + np.cross(w, c), atol=1e-6)
    assert np.allclose(W[0], w + 0.5 * curl, atol=1e-6)


def test_batched_mobility_matches_single_solves():
    # mobility problems (forces and torques prescribed, velocities found) and a resistance problem
    # in one lockstep batch: each must reproduce its own single solve, which the tests above tie
    # to the oracle's dense bordered system
    rng = np.random.default_rng(21)
    kw = dict(n_proxy=120, r_proxy=0.63, m_basic=240)
    geoms = [workloads.two_spheres(0.05), workloads.suspension(4, 0.15, seed=11), np.array([[0.0, 0.0, 0.0]]),
             workloads.two_spheres(0.2)]
    ctxs, loads = [], []
    for i, c in enumerate(geoms):
        ctx = mfs.Context(0)
        ctx.set_spheres(c)
        ctx.build(**kw)
        P = c.shape[0]
        if i < 3:
            F, T = rng.normal(size=(P, 3)), rng.normal(size=(P, 3))
            ctx.set_forces_torques(F, T)
            loads.append(("mobility", F, T))
        else:
            v, w = rng.normal(size=(P, 3)), rng.normal(size=(P, 3))
            ctx.set_rigid_velocities(v, w)
            loads.append(("resistance", v, w))
        ctxs.append(ctx)
    infos = mfs.batch_solve(ctxs, precision="mixed", tol=1e-8)
    assert all(i.converged == 1 for i in infos)
    batch_out = []
    for ctx, (kind, a, b) in zip(ctxs, loads):
        batch_out.append(ctx.rigid_velocities() if kind == "mobility" else ctx.forces_torques())
    for ctx, (kind, a, b), got in zip(ctxs, loads, batch_out):
        if kind == "mobility":
            ctx.set_forces_torques(a, b)
        else:
            ctx.set_rigid_velocities(a, b)
        info = ctx.solve(precision="mixed", tol=1e-8)
        assert info.converged == 1
        ref = ctx.rigid_velocities() if kind == "mobility" else ctx.forces_torques()
        scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
        assert max(np.abs(got[0] - ref[0]).max(), np.abs(got[1] - ref[1]).max()) <= 1e-6 * scale, kind
        if kind == "mobility":
            # the forces and torques of the batched solution are the prescribed ones
            F, T = ctx.forces_torques()
            assert np.abs(F - a).max() <= 1e-6 * np.abs(a).max() and np.abs(T - b).max() <= 1e-6 * np.abs(b).max()
    for ctx in ctxs:
        ctx.close()
