"""Fixed clusters in a background flow (Sec. 4, Ex. 2, Table cluster_table).

A cluster is grown so that every sphere has a neighbour exactly delta away; it is held fixed
in a shear flow u_inf = (5 y, 0, 0) or a uniform flow u_inf = (5, 0, 0), so the disturbance
velocity must cancel u_inf on every surface (eq. bc).  The spheres do not move relative to one
another, and the paper runs this example with the basic method (no images, Sec. 4), so every
sphere shares the basic factor: one SVD, and step 1 of the passes as one tensor-core product.

Checked:
  * a 10-sphere cluster in each flow against the oracle's O3 solve: forces/torques to 1e-5,
    velocity at the check points to 1e-3;
  * the paper's P = 100 settings of Table cluster_table (N = 686 proxies, GMRES tolerance 1e-6):
    the solve converges in a number of iterations close to the table's 92, 122, 116 (within 30 %;
    the Fibonacci grids that stand in for the spherical designs change the count slightly;
    measured 93 / 111 / 108); the surface residual (eq. residual) relative to each sphere's
    largest boundary speed stays at the table's ~1e-4 level (below 1e-3; measured 1e-4..2.2e-4),
    and pointwise, where the shear flow's boundary data is not near its zero plane, below 1e-2
    (measured 2e-3..5e-3: the Fibonacci grids are coarser than the designs); the strengths stay
    moderate (the table prints max |lambda| of 9.8 and 9.5 for R_p = 0.75 and 316 for 0.65;
    measured 7.9 / 8.1 / 167).
"""
import numpy as np
import pytest

from oracle import geometry, solve
from paper_2407_03343_gb300 import mfs, workloads
from tests.layout import lib_to_oracle

pytestmark = pytest.mark.gpu

BASIC = dict(nim_fixed=0)   # no images: the basic method


def _flow(kind):
    return workloads.shear_flow(5.0) if kind == "shear" else workloads.uniform_flow(5.0)


@pytest.mark.parametrize("kind", ["shear", "uniform"])
def test_small_cluster_in_flow_matches_oracle(kind):
    centres = workloads.cluster(10, 1e-2, seed=4)
    kw = dict(n_proxy=200, r_proxy=0.75, m_basic=240, **BASIC)
    U, E, Om = _flow(kind)
    d = geometry.build(centres, 1.0, geometry.Params(**kw))
    zero = np.zeros((10, 3))
    bg = solve.Background(U=U, E=E, omega=Om)
    sol = solve.solve_o3(d, zero, zero, background=bg, tol=1e-9)
    with mfs.Context(0) as ctx:
        ctx.set_spheres(centres)
        ctx.build(**kw, tensor_step1=2)
        ctx.set_background_flow(U=U, E=E, Omega=Om)
        ctx.set_rigid_velocities(zero, zero)
        info = ctx.solve(precision="mixed", tol=1e-8)
        assert info.converged == 1
        F, T = ctx.forces_torques()
        Fo, To = solve.forces_torques(d, sol.lam)
        ref = np.abs(np.r_[Fo.ravel(), To.ravel()]).max()
        assert np.abs(np.r_[F.ravel() - Fo.ravel(), T.ravel() - To.ravel()]).max() <= 1e-5 * ref
        x = np.concatenate(d.check)
        uo = solve.velocity(d, sol.lam, x)
        assert np.abs(ctx.eval_velocity(x) - uo).max() <= 1e-3 * np.abs(uo).max()


def _surface_residuals(ctx, d, U, E, Om):
    """eq. residual at the check points, u_bc = -u_inf: (a) the pointwise ratio |u - u_bc| / |u_bc|
    where |u_bc| is at least 1e-2 of its largest value on that sphere (the shear flow vanishes on
    the plane y = 0, which runs through the cluster; there the pointwise ratio has no meaning),
    (b) |u - u_bc| relative to the largest |u_bc| on that sphere; the largest of each."""
    pw = rel = 0.0
    for x in d.check:
        u = ctx.eval_velocity(x)
        ubc = -(U[None, :] + x @ E.T + np.cross(Om[None, :], x))
        nb = np.linalg.norm(ubc, axis=1)
        err = np.linalg.norm(u - ubc, axis=1)
        keep = nb >= 1e-2 * nb.max()
        pw = max(pw, float((err[keep] / nb[keep]).max()))
        rel = max(rel, float(err.max() / nb.max()))
    return pw, rel


@pytest.mark.parametrize("delta,r_p,printed_iters", [(1e-2, 0.75, 92), (1e-3, 0.75, 122), (1e-3, 0.65, 116)])
def test_cluster_table_settings(delta, r_p, printed_iters):
    centres = workloads.cluster(100, delta, seed=1)
    kw = dict(n_proxy=686, r_proxy=r_p, m_basic=823, **BASIC)
    U, E, Om = workloads.shear_flow(5.0)
    with mfs.Context(0) as ctx:
        ctx.set_spheres(centres)
        ctx.build(**kw)
        assert ctx.sizes().n_factors == 1
        ctx.set_background_flow(U=U, E=E, Omega=Om)
        ctx.set_rigid_velocities(np.zeros((100, 3)), np.zeros((100, 3)))
        info = ctx.solve(precision="mixed", tol=1e-6)
        assert info.converged == 1
        # measured: 93 / 111 / 108 against the printed 92 / 122 / 116
        assert 0.7 * printed_iters <= info.iters <= 1.3 * printed_iters, info.iters
        d = geometry.build(centres, 1.0, geometry.Params(**kw))
        pw, rel = _surface_residuals(ctx, d, U, E, Om)
        # measured: pointwise 2e-3..5e-3, relative to the sphere's largest boundary speed 1e-4..2.2e-4
        # (the table prints 6.9e-5..1.1e-4)
        assert pw <= 1e-2 and rel <= 1e-3, (pw, rel)
        lam = lib_to_oracle(d, ctx.strengths())
        lam_max = max(np.abs(x).max() for x in lam)
        # measured: 7.9 / 8.1 / 167 against the printed 9.8 / 9.5 / 316
        assert lam_max <= (20.0 if r_p > 0.7 else 1000.0), lam_max
