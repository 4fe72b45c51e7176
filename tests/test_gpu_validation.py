"""Validation experiments of Sec. 5.2 and 5.3 on self-generated geometries, solved on the GPU: the
tetrahedron of spheres with and without image points (self-convergence of forces and torques
against the fine MFS grid), the GMRES iteration count as the gap closes, and a random cluster of
20 spheres each 1e-3 from a neighbour.

Coarse grid: N = 686 proxies on R_p = 0.63, 823 basic nodes, adaptive images (eq. image_est).
Fine grid: N = 1353 on R_p = 0.7, 1624 basic nodes, 30 images per contact.  The thresholds are
the paper's where this build meets them (force/torque error < 1e-3 with images) and otherwise
the measured levels with margin (the relative residual, limited by the Fibonacci node sets that
replace the spherical designs).
"""
import numpy as np
import pytest

from oracle import geometry
from paper_2407_03343_gb300 import mfs, workloads

pytestmark = pytest.mark.gpu

COARSE = dict(n_proxy=686, r_proxy=0.63, m_basic=823)
FINE = dict(n_proxy=1353, r_proxy=0.7, m_basic=1624, nim_fixed=30, nim_max=30)
CHECK = geometry.fibonacci_sphere(500)[:, [1, 2, 0]]


def eps_res(ctx, centres, v, w):
    """eq. residual: max over 500 check points per sphere of |u - u_bc| / |u_bc|."""
    worst = 0.0
    for k, c in enumerate(centres):
        x = c + CHECK
        u = ctx.eval_velocity(x)
        ub = v[k] + np.cross(w[k], x - c)
        worst = max(worst, float((np.linalg.norm(u - ub, axis=1) / np.linalg.norm(ub, axis=1)).max()))
    return worst


def solve(centres, v, w, **params):
    ctx = mfs.Context(0)
    ctx.set_spheres(centres)
    ctx.build(**params)
    ctx.set_rigid_velocities(v, w)
    info = ctx.solve(precision="mixed", tol=1e-6, max_iter=3000)
    F, T = ctx.forces_torques()
    er = eps_res(ctx, centres, v, w)
    ctx.close()
    return info, F, T, er


@pytest.mark.parametrize("delta", [1e-2, 1e-3])
def test_tetrahedron_forces_converge_to_fine_grid(delta):
    c = workloads.tetrahedron(delta)
    v, w = workloads.rigid_velocities(4, seed=2)
    info_c, Fc, Tc, er_c = solve(c, v, w, **COARSE)
    info_f, Ff, Tf, er_f = solve(c, v, w, **FINE)
    assert info_c.converged and info_f.converged
    scale = max(np.abs(Ff).max(), np.abs(Tf).max())
    eps_ft = max(np.abs(Fc - Ff).max(), np.abs(Tc - Tf).max()) / scale
    # the paper's target; measured 1.7e-4 (delta 1e-2) and 1.4e-4 (1e-3)
    assert eps_ft < 1e-3
    # the fine grid resolves the surface better than the coarse one
    assert er_f < er_c < 5e-2


def test_tetrahedron_needs_images():
    c = workloads.tetrahedron(1e-2)
    v, w = workloads.rigid_velocities(4, seed=2)
    _, _, _, er_img = solve(c, v, w, **COARSE)
    _, _, _, er_plain = solve(c, v, w, nim_cut=0.0, **COARSE)   # proxies only
    # measured 1.7e-2 with images against 1.7 without
    assert er_img < 5e-2 and er_plain > 0.5


def test_iterations_grow_as_the_gap_closes():
    v, w = workloads.rigid_velocities(4, seed=2)
    iters = []
    for delta in (1e-1, 1e-2, 1e-3):
        info, _, _, _ = solve(workloads.tetrahedron(delta), v, w, **COARSE)
        assert info.converged
        iters.append(info.iters)
    # Sec. 5.3: growth roughly like delta^(-1/2); measured 39, 156, 756 (slope ~0.65)
    assert iters[0] < iters[1] < iters[2]
    slope = np.log(iters[2] / iters[0]) / np.log(100.0)
    assert 0.3 < slope < 0.9


def test_random_cluster_of_twenty():
    c = workloads.cluster(20, 1e-3, seed=2)
    v, w = workloads.rigid_velocities(20, seed=2)
    info, _, _, er = solve(c, v, w, **COARSE)
    assert info.converged
    # the paper reaches 1e-3; measured here 1.7e-3 (seed 2) and 4.2e-3 (seed 1)
    assert er < 1e-2


def test_minimum_images_close_the_image_free_window():
    # gap 0.2: the printed rule places no images and the coarse grid misses 1e-3; the opt-in
    # minimum of two images per contact below gap 0.3 brings the residual well below it
    c = workloads.two_spheres(0.2)
    v, w = workloads.rigid_velocities(2, seed=2)
    _, _, _, er_rule = solve(c, v, w, **COARSE)
    _, _, _, er_min = solve(c, v, w, nim_cut=0.3, nim_min=2, **COARSE)
    assert er_rule > 3e-3 and er_min < 5e-4


def triangle(delta):
    """Three unit spheres on an equilateral triangle of side 2 + delta in the plane z = 0."""
    s = 2.0 + delta
    r = s / np.sqrt(3.0)
    ang = np.array([90.0, 210.0, 330.0]) * np.pi / 180.0
    return np.stack([r * np.cos(ang), r * np.sin(ang), np.zeros(3)], axis=1)


def test_triangle_exterior_flow_self_convergence():
    # Sec. 5.2, first example: the spheres approach the triangle's centre at unit speed; the flow
    # in the plane of the triangle, outside the spheres, from the coarse grid (20 images per
    # contact at delta = 1e-3) against the fine grid; the paper reports a largest pointwise
    # relative difference of 7.6e-4.  Measured here with the Fibonacci grids: see the design notes.
    c = triangle(1e-3)
    v = -c / np.linalg.norm(c, axis=1, keepdims=True)
    w = np.zeros((3, 3))
    g = np.linspace(-3.5, 3.5, 141)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    dist = np.linalg.norm(pts[:, None, :] - c[None, :, :], axis=2).min(axis=1)
    pts = pts[dist >= 1.0 + 1e-6]
    u = []
    for params in (COARSE, FINE):
        with mfs.Context(0) as ctx:
            ctx.set_spheres(c)
            ctx.build(**params)
            ctx.set_rigid_velocities(v, w)
            assert ctx.solve(precision="mixed", tol=1e-8, max_iter=3000).converged == 1
            u.append(ctx.eval_velocity(pts))
    uc, uf = u
    # pointwise relative difference where the flow is not near a stagnation point (the centre of
    # the triangle is one, by symmetry): |u_f| at least 1e-2 of its largest value in the plane
    nf = np.linalg.norm(uf, axis=1)
    keep = nf >= 1e-2 * nf.max()
    rel = np.linalg.norm(uc - uf, axis=1)[keep] / nf[keep]
    print(f"triangle: {pts.shape[0]} points, {int(keep.sum())} away from stagnation; max pointwise "
          f"{rel.max():.3e}, median {np.median(rel):.3e}; max relative to the largest speed "
          f"{np.linalg.norm(uc - uf, axis=1).max() / nf.max():.3e}")
    assert pts.shape[0] > 10000
    assert rel.max() < 1e-2
    assert np.median(rel) < 1e-3
