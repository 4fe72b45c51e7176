"""CUDA path against the FP64 CPU oracle, element by element, through the C ABI.

Sizes span several 512-node target tiles, several 256-source proxy tiles and 128-node
image tiles, each with a ragged tail.

Tolerances, from the arithmetic:
  * pair sums with O(1) strengths: FP64 and double-float 1e-11 of the field; FP32 2e-5
    (rounding over ~1e3 terms, compensated cross-tile sums).
  * pair sums whose strengths come from the truncated pseudo-inverse of a random vector
    (amplified ~1e9) cancel massively; the error bound is then relative to the absolute
    sum  sum_j |S_ij| |lambda_j|  (the condition number of the sum): 1e-13 of it for FP64
    and double-float, while FP32 misses the field itself by more than 1%.
  * one-body pseudo-inverse: lambda_hat for a random vector depends on eps-level details of
    two different SVD codes (1e-4 relative); its effect B lambda_hat much less (1e-5 |mu|).
  * end-to-end: force/torque error <= 1e-5 and surface-velocity error <= 1e-3 (the stated
    targets) against an oracle solved well below the GMRES tolerance, because at the
    paper's tolerance 1e-6 the forces are themselves only converged to ~1e-5.
    Two-sphere cases use the dense LU solve O2; clusters use matrix-free GMRES O3 (the
    dense G_hat of O2 loses ~1e-5 there, as Sec. 2.2 warns).
"""
import math

import numpy as np
import pytest

from oracle import brenner, geometry, solve
from paper_2407_03343_gb300 import mfs, workloads
from tests.layout import lib_to_oracle, oracle_to_lib

pytestmark = pytest.mark.gpu

C1 = dict(n_proxy=300, r_proxy=0.7, m_basic=600, nim_fixed=10)


def make(centres, **kw):
    ctx = mfs.Context(0)
    ctx.set_spheres(centres)
    ctx.build(**kw)
    d = geometry.build(centres, 1.0, geometry.Params(**kw))
    return ctx, d


def cluster5():
    c = workloads.suspension(5, 0.15, seed=11)
    return c


@pytest.fixture(scope="module")
def c1():
    ctx, d = make(workloads.two_spheres(0.1), **C1)
    op = solve.Operator(d)
    yield ctx, d, op
    ctx.close()


@pytest.fixture(scope="module")
def c5():
    kw = dict(n_proxy=260, r_proxy=0.63, m_basic=420)
    ctx, d = make(cluster5(), **kw)
    op = solve.Operator(d)
    yield ctx, d, op
    ctx.close()


def test_discretisation_matches_oracle(c1, c5):
    for ctx, d, _ in (c1, c5):
        x, w, owner = ctx.collocation()
        X = np.concatenate([s.colloc for s in d.spheres])
        W = np.concatenate([s.weight for s in d.spheres])
        O = np.concatenate([np.full(s.colloc.shape[0], k) for k, s in enumerate(d.spheres)])
        assert x.shape == X.shape
        assert np.allclose(x, X, atol=1e-12) and np.allclose(w, W, rtol=1e-13) and np.array_equal(owner, O)
        pos, typ = ctx.source_layout()
        s = ctx.sizes()
        assert s.n_contacts == len(d.contacts)
        assert s.n_image_nodes == sum(sp.image.shape[0] for sp in d.spheres)
        ref_pos, ref_typ = [], []
        for sp in d.spheres:
            ref_pos.append(sp.proxy)
            ref_typ.append(np.zeros(sp.proxy.shape[0], int))
            ref_pos.append(np.repeat(sp.image, 3, axis=0))
            ref_typ.append(np.tile([0, 1, 2], sp.image.shape[0]))
        assert np.allclose(pos, np.concatenate(ref_pos), atol=1e-12)
        assert np.array_equal(typ, np.concatenate(ref_typ))


def test_rhs_matches_oracle(c5):
    ctx, d, _ = c5
    v, om = workloads.rigid_velocities(d.centres.shape[0], seed=3)
    ctx.set_rigid_velocities(v, om)
    U, E, Om = np.array([0.5, -1.0, 0.2]), np.array([[0, 2.5, 0], [2.5, 0, 0], [0, 0, 0.0]]), np.array([0, 0, -2.5])
    ctx.set_background_flow(U, E, Om)
    b = ctx.rhs()
    ref = np.concatenate(solve.rhs(d, v, om, solve.Background(U, E, Om)))
    ctx.set_background_flow()
    assert np.allclose(b, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def pair_reference(d, op, lam_hat_list, mu):
    mus = op.split(mu)
    out = []
    for k in range(len(d.spheres)):
        acc = mus[k].copy()
        for kp in range(len(d.spheres)):
            if kp != k:
                acc = acc + op.block(k, kp) @ lam_hat_list[kp]
        out.append(acc)
    return np.concatenate(out)


@pytest.mark.parametrize("which", ["c1", "c5"])
def test_pair_apply_matches_oracle(which, c1, c5, request):
    ctx, d, op = c1 if which == "c1" else c5
    rng = np.random.default_rng(7)
    lam_o = [rng.normal(size=solve.n_unknowns(d, k)) for k in range(len(d.spheres))]
    mu = rng.normal(size=op.n)
    ref = pair_reference(d, op, lam_o, mu)
    lam_l = oracle_to_lib(d, lam_o)
    field = np.abs(ref - mu).max()
    out64 = ctx.apply_pairs(lam_l, mu, mfs.FP64)
    assert np.abs(out64 - ref).max() <= 1e-11 * field
    outdw = ctx.apply_pairs(lam_l, mu, mfs.MIXED)
    assert np.abs(outdw - ref).max() <= 1e-11 * field
    out32 = ctx.apply_pairs(lam_l, mu, mfs.FP32)
    assert np.abs(out32 - ref).max() <= 2e-5 * field


def test_pair_apply_with_cancellation(c1):
    # strengths from the truncated pseudo-inverse of a random vector: |lambda_hat| ~ 1e9 |field|
    ctx, d, op = c1
    rng = np.random.default_rng(17)
    mu = rng.normal(size=op.n)
    lam_o = [solve.pinv_apply(op.f[k], m) for k, m in enumerate(op.split(mu))]
    ref = pair_reference(d, op, lam_o, mu)
    # absolute sum of the terms per row
    abs_sum = np.concatenate([np.abs(op.block(k, 1 - k)) @ np.abs(lam_o[1 - k]) for k in range(2)])
    field = np.abs(ref - mu).max()
    assert max(np.abs(l).max() for l in lam_o) / field > 1e6
    lam_l = oracle_to_lib(d, lam_o)
    for prec in (mfs.FP64, mfs.MIXED):
        out = ctx.apply_pairs(lam_l, mu, prec)
        assert np.all(np.abs(out - ref) <= 1e-13 * abs_sum + 1e-12 * field)
    out32 = ctx.apply_pairs(lam_l, mu, mfs.FP32)
    assert np.abs(out32 - ref).max() > 1e-2 * field   # why plain FP32 cannot serve the solve


def test_precond_matches_oracle(c1):
    ctx, d, op = c1
    rng = np.random.default_rng(8)
    mu = rng.normal(size=op.n)
    lam_gpu = lib_to_oracle(d, ctx.apply_precond(mu, mfs.FP64))
    mus = op.split(mu)
    for k in range(len(d.spheres)):
        f = op.f[k]
        ref = solve.pinv_apply(f, mus[k])
        B = op.block(k, k)
        # the projection B B^+ mu is insensitive to how the SVD was computed
        assert np.abs(B @ lam_gpu[k] - B @ ref).max() <= 1e-5 * np.abs(mus[k]).max()
        assert np.abs(lam_gpu[k] - ref).max() <= 1e-4 * np.abs(ref).max()
    # smooth data (scaled rigid-motion boundary data): strengths still ~1e5, same sensitivity
    v = np.array([[0.3, 1.0, -0.2], [-0.5, 0.1, 0.4]])
    om = np.array([[0.2, -0.3, 1.0], [0.0, 0.6, -0.1]])
    wb = np.concatenate(solve.rhs(d, v, om))
    lam_s = lib_to_oracle(d, ctx.apply_precond(wb, mfs.FP64))
    for k, m in enumerate(op.split(wb)):
        ref = solve.pinv_apply(op.f[k], m)
        B = op.block(k, k)
        # what the method uses of lambda_hat, its image B lambda_hat = U U^T m (the projection of
        # the data on the retained singular space), agrees far more closely than lambda_hat
        assert np.abs(B @ lam_s[k] - B @ ref).max() <= 1e-6 * np.abs(m).max()
        # lambda_hat itself is not unique under the truncated SVD (near-threshold directions):
        # only 1e-4 relative between two backward-stable SVD codes
        assert np.abs(lam_s[k] - ref).max() <= 1e-4 * np.abs(ref).max()
    # FP32 factors: relative accuracy of lambda_hat itself
    lam32 = lib_to_oracle(d, ctx.apply_precond(mu, mfs.FP32))
    for k in range(len(d.spheres)):
        ref = solve.pinv_apply(op.f[k], mus[k])
        assert np.abs(lam32[k] - ref).max() <= 1e-4 * np.abs(ref).max()


def test_operator_matches_oracle(c5):
    ctx, d, op = c5
    # smooth vector (scaled rigid-motion data) and its image under G_hat
    v, om = workloads.rigid_velocities(d.centres.shape[0], seed=12)
    mu = np.concatenate(solve.rhs(d, v, om))
    for vec in (mu, op.apply(mu)):
        ref = op.apply(vec)
        for prec in (mfs.FP64, mfs.MIXED):
            out = ctx.apply_operator(vec, prec)
            assert np.abs(out - ref).max() <= 1e-7 * np.abs(ref).max()
    # random vector: strengths amplified ~1e9, SVD-detail sensitive
    rng = np.random.default_rng(9)
    mu = rng.normal(size=op.n)
    ref = op.apply(mu)
    for prec in (mfs.FP64, mfs.MIXED):
        out = ctx.apply_operator(mu, prec)
        assert np.abs(out - ref).max() <= 1e-4 * np.abs(ref).max()


def ft_error(F, T, Fo, To):
    ref = np.abs(np.r_[Fo.ravel(), To.ravel()]).max()
    return np.abs(np.r_[F.ravel() - Fo.ravel(), T.ravel() - To.ravel()]).max() / ref


TOL = {"fp64": 1e-9, "mixed": 1e-8}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_matches_oracle_c1(precision, c1):
    ctx, d, op = c1
    v = np.array([[0.3, 1.0, -0.2], [-0.5, 0.1, 0.4]])
    om = np.array([[0.2, -0.3, 1.0], [0.0, 0.6, -0.1]])
    ctx.set_rigid_velocities(v, om)
    info = ctx.solve(precision=precision, tol=TOL[precision])
    assert info.converged == 1 and info.rel_residual <= TOL[precision]
    F, T = ctx.forces_torques()
    sol = solve.DenseSystem(d, op).solve(v, om)
    Fo, To = solve.forces_torques(d, sol.lam)
    assert ft_error(F, T, Fo, To) <= 1e-5
    x = np.concatenate(d.check)
    u = ctx.eval_velocity(x)
    uo = solve.velocity(d, sol.lam, x)
    assert np.abs(u - uo).max() <= 1e-5 * np.abs(uo).max()


@pytest.fixture(scope="module")
def c5_oracle(c5):
    _, d, op = c5
    v, om = workloads.rigid_velocities(d.centres.shape[0], seed=4)
    sol = solve.solve_o3(d, v, om, op=op, tol=1e-9)
    return v, om, sol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_matches_oracle_cluster(precision, c5, c5_oracle):
    ctx, d, op = c5
    v, om, sol = c5_oracle
    ctx.set_rigid_velocities(v, om)
    info = ctx.solve(precision=precision, tol=TOL[precision])
    assert info.converged == 1
    F, T = ctx.forces_torques()
    Fo, To = solve.forces_torques(d, sol.lam)
    assert ft_error(F, T, Fo, To) <= 1e-5
    x = np.concatenate(d.check)
    u = ctx.eval_velocity(x)
    uo = solve.velocity(d, sol.lam, x)
    assert np.abs(u - uo).max() <= 1e-3 * np.abs(uo).max()


def test_paper_tolerance_solve_is_accurate_to_discretisation(c5, c5_oracle):
    # at the paper's GMRES tolerance 1e-6 the surface velocity still matches to 1e-3
    ctx, d, op = c5
    v, om, sol = c5_oracle
    ctx.set_rigid_velocities(v, om)
    info = ctx.solve(precision="mixed")
    assert info.converged == 1 and info.rel_residual <= 1e-6
    x = np.concatenate(d.check)
    u = ctx.eval_velocity(x)
    uo = solve.velocity(d, sol.lam, x)
    assert np.abs(u - uo).max() <= 1e-3 * np.abs(uo).max()
    F, T = ctx.forces_torques()
    Fo, To = solve.forces_torques(d, sol.lam)
    assert ft_error(F, T, Fo, To) <= 1e-3


def test_squeeze_matches_brenner(c1):
    ctx, d, _ = c1
    v, om = workloads.motion("squeeze")
    ctx.set_rigid_velocities(v, om)
    ctx.solve(precision="mixed")
    F, _ = ctx.forces_torques()
    fb = brenner.squeeze_force(0.1)
    assert abs(F[0, 0] - fb) / fb < 1e-3 and abs(F[1, 0] + fb) / fb < 1e-3


def test_single_sphere_drag():
    with mfs.Context(0) as ctx:
        ctx.set_spheres([[1.0, 2.0, 3.0]], radius=1.5)
        ctx.build(n_proxy=300, r_proxy=0.7, m_basic=400)
        U, W = np.array([[0.3, -0.7, 1.1]]), np.array([[-0.4, 0.2, 0.9]])
        ctx.set_rigid_velocities(U, W)
        ctx.solve(precision="mixed", tol=1e-8)
        F, T = ctx.forces_torques()
        assert np.allclose(F, 6 * math.pi * 1.5 * U, rtol=1e-5, atol=1e-5 * 6 * math.pi * 1.5)
        assert np.allclose(T, 8 * math.pi * 1.5 ** 3 * W, rtol=1e-5, atol=1e-5 * 8 * math.pi * 1.5 ** 3)
        s = ctx.sizes()
        assert s.n_contacts == 0 and s.n_factors == 1 and s.pairs_fp == 0


def test_zero_boundary_data_gives_zero():
    with mfs.Context(0) as ctx:
        ctx.set_spheres(workloads.two_spheres(0.3))
        ctx.build(n_proxy=100, r_proxy=0.63, m_basic=150)
        ctx.set_rigid_velocities(np.zeros((2, 3)), np.zeros((2, 3)))
        info = ctx.solve()
        F, T = ctx.forces_torques()
        assert info.iters == 0 and np.all(F == 0) and np.all(T == 0)
        assert ctx.eval_velocity(np.zeros((0, 3))).shape == (0, 3)


def test_errors_are_reported():
    with mfs.Context(0) as ctx:
        with pytest.raises(mfs.MfsError) as e:
            ctx.build()
        assert e.value.status == -4
        ctx.set_spheres(workloads.two_spheres(0.1))
        with pytest.raises(mfs.MfsError) as e:
            ctx.solve()
        assert e.value.status == -4
        with pytest.raises(mfs.MfsError) as e:
            ctx.set_spheres(np.array([[0, 0, 0], [3, 0, 0.0]]), radius=[1.0, 1.2])
        assert e.value.status == -3
        ctx.set_spheres(np.array([[0, 0, 0], [1.99, 0, 0.0]]))
        with pytest.raises(mfs.MfsError) as e:
            ctx.build(n_proxy=50, m_basic=80)
        assert e.value.status == -2
        ctx.set_spheres(workloads.two_spheres(0.5))
        ctx.build(n_proxy=50, m_basic=80)
        ctx.set_rigid_velocities(np.ones((2, 3)), np.zeros((2, 3)))
        with pytest.raises(mfs.MfsError) as e:
            ctx.solve(restart=1000)
        assert e.value.status == -1
        info = ctx.solve(max_iter=1, max_refine=1, allow_not_converged=True)
        assert info.converged == 0
