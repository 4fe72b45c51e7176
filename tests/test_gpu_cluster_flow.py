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
    the solve converges in a number of iterations of the size the table prints (92, 122, 116;
    the Fibonacci grids that stand in for the spherical designs change the count, so only the
    size is compared: within a factor of three), the largest relative surface residual at the
    check points (eq. residual) meets the paper's 1e-3 target, and the strengths stay
    moderate (the table prints max |lambda| of 9.8 and 9.5 for R_p = 0.75 and 316 for 0.65).
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


def _surface_residual(ctx, d, U, E, Om):
    """eq. residual: max over the check points of |u - u_bc| / |u_bc|, u_bc = -u_inf."""
    x = np.concatenate(d.check)
    u = ctx.eval_velocity(x)
    ubc = -(U[None, :] + x @ E.T + np.cross(Om[None, :], x))
    return float((np.linalg.norm(u - ubc, axis=1) / np.linalg.norm(ubc, axis=1)).max())


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
        assert printed_iters / 3 <= info.iters <= 3 * printed_iters, info.iters
        d = geometry.build(centres, 1.0, geometry.Params(**kw))
        assert _surface_residual(ctx, d, U, E, Om) <= 1e-3
        lam = lib_to_oracle(d, ctx.strengths())
        lam_max = max(np.abs(x).max() for x in lam)
        assert lam_max <= (100.0 if r_p > 0.7 else 3000.0)
