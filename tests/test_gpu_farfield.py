"""Far field of the GMRES passes (equivalent Stokeslets for distant spheres) against the oracle.

The oracle has no far field: it sums every pair exactly (eq. uAll).  The far field is an
approximation of that sum, so it is judged against the exact operator with a stated tolerance:
  * the pass operator (Sigma^+ U^T from FP32, near spheres in double-float, far spheres through
    their FP32 equivalent sources) matches the oracle's exact operator to 1e-5 of its largest
    value on smooth data and on a Krylov-like vector; the same operator without the far field
    (every sphere near) matches to 1e-7, and the all-pairs pass operator to 1e-10 (the same
    double-float sums, in another order when the all-pairs kernel splits sources over CTAs, whose
    rounding relative to the result grows with the cancellation of the Krylov-like vector);
  * a MIXED solve with the far field, whose refinement residual uses every pair exactly, meets
    the stated targets against the oracle's O3 solve (forces/torques 1e-5, velocity 1e-3).
"""
import numpy as np
import pytest

from oracle import geometry, solve
from paper_2407_03343_gb300 import mfs, workloads

pytestmark = pytest.mark.gpu

KW = dict(n_proxy=150, r_proxy=0.63, m_basic=300)
FAR = dict(far_dist=4.0, far_n_eq=300, far_r_eq=1.0, far_r_chk=2.0, far_eps=1e-6)


# two near-contact pairs (gaps 0.1 and 0.05, images on) and six spheres 4-9 radii apart
CENTRES = np.array([[0.0, 0.0, 0.0], [2.1, 0.0, 0.0], [0.0, 6.0, 0.0], [0.0, 8.05, 0.0], [6.5, 0.5, 0.3],
                    [6.0, 6.5, -0.4], [3.2, 3.1, 5.0], [-4.5, 3.0, 2.0], [9.5, 3.0, -3.0], [3.0, -5.0, 1.0]])


@pytest.fixture(scope="module")
def dilute():
    centres = CENTRES
    d = geometry.build(centres, 1.0, geometry.Params(**KW))
    op = solve.Operator(d)
    ctx = mfs.Context(0)
    ctx.set_spheres(centres)
    ctx.build(**KW, **FAR)
    yield centres, d, op, ctx
    ctx.close()


def _krylov_like(op, mu, steps=4):
    x = mu.copy()
    for _ in range(steps):
        x = op.apply(x)
        x /= np.abs(x).max()
    return x


def test_far_field_is_used(dilute):
    _, d, _, ctx = dilute
    s = ctx.sizes()
    assert s.pairs_far_eq > 0 and 0 < s.pairs_near_fp < s.pairs_fp
    assert s.n_contacts >= 1


def test_pass_operator_matches_exact_oracle(dilute):
    centres, d, op, ctx = dilute
    v, om = workloads.rigid_velocities(len(d.spheres), seed=3)
    mu = np.concatenate(solve.rhs(d, v, om))
    for vec in (mu, _krylov_like(op, mu)):
        ref = op.apply(vec)
        scale = np.abs(ref).max()
        out = ctx.apply_operator(vec, mfs.MIXED_PASS)
        assert np.abs(out - ref).max() <= 1e-5 * scale
    # control: every sphere near (no far field) -> the all-pairs pass operator
    with mfs.Context(0) as c2:
        c2.set_spheres(centres)
        c2.build(**KW, **dict(FAR, far_dist=1e3))
        assert c2.sizes().pairs_far_eq == 0
        with mfs.Context(0) as c3:
            c3.set_spheres(centres)
            c3.build(**KW)
            for vec in (mu, _krylov_like(op, mu)):
                a = c2.apply_operator(vec, mfs.MIXED_PASS)
                b = c3.apply_operator(vec, mfs.MIXED_PASS)
                assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
                assert np.abs(a - op.apply(vec)).max() <= 1e-7 * np.abs(a).max()


def test_far_field_solve_matches_oracle(dilute):
    centres, d, op, ctx = dilute
    v, om = workloads.rigid_velocities(len(d.spheres), seed=8)
    sol = solve.solve_o3(d, v, om, op=op, tol=1e-9)
    ctx.set_rigid_velocities(v, om)
    ctx.set_profiling(True)
    ctx.timing(reset=True)
    info = ctx.solve(precision="mixed", tol=1e-8)
    t = ctx.timing(reset=True)
    assert info.converged == 1 and info.rel_residual <= 1e-8
    assert t.far_launches > 0 and t.far_pairs > 0
    F, T = ctx.forces_torques()
    Fo, To = solve.forces_torques(d, sol.lam)
    ref = np.abs(np.r_[Fo.ravel(), To.ravel()]).max()
    assert np.abs(np.r_[F.ravel() - Fo.ravel(), T.ravel() - To.ravel()]).max() <= 1e-5 * ref
    x = np.concatenate(d.check)
    u = ctx.eval_velocity(x)
    uo = solve.velocity(d, sol.lam, x)
    assert np.abs(u - uo).max() <= 1e-3 * np.abs(uo).max()
    # the exact-operator MIXED solve needs about as many iterations
    with mfs.Context(0) as c3:
        c3.set_spheres(centres)
        c3.build(**KW)
        c3.set_rigid_velocities(v, om)
        info3 = c3.solve(precision="mixed", tol=1e-8)
        assert info.iters <= 1.3 * info3.iters + 10


def test_far_field_parameters_are_checked():
    with mfs.Context(0) as ctx:
        ctx.set_spheres(workloads.two_spheres(0.5))
        with pytest.raises(mfs.MfsError) as e:
            ctx.build(**KW, **dict(FAR, far_dist=2.5))   # inside check radius + 1
        assert e.value.status == -1
        with pytest.raises(mfs.MfsError) as e:
            ctx.build(**KW, **dict(FAR, far_r_eq=2.5))   # equivalent sphere outside the check sphere
        assert e.value.status == -1


def test_autotuned_shapes_keep_the_operator(dilute):
    centres, d, op, ctx = dilute
    v, om = workloads.rigid_velocities(len(d.spheres), seed=3)
    mu = np.concatenate(solve.rhs(d, v, om))
    before = ctx.apply_operator(mu, mfs.MIXED_PASS)
    shapes = ctx.tune_pairs()
    for nt, parts, ms in ((shapes.all_nodes_per_thread, shapes.all_parts, shapes.all_ms),
                          (shapes.near_nodes_per_thread, shapes.near_parts, shapes.near_ms),
                          (shapes.far_nodes_per_thread, shapes.far_parts, shapes.far_ms)):
        assert nt in (1, 4) and 1 <= parts <= 16 and ms > 0
    after = ctx.apply_operator(mu, mfs.MIXED_PASS)
    # other tiles and source splits only reorder the sums
    assert np.abs(after - before).max() <= 1e-9 * np.abs(before).max()
    assert np.abs(after - op.apply(mu)).max() <= 1e-5 * np.abs(before).max()


def test_far_field_with_512_node_tiles():
    # 343 contact-free spheres on a lattice 3 radii apart: enough 512-node tiles that the far
    # kernel runs 4 nodes per thread (packed two-lane FP32 by default); the pass operator against
    # the exact double-float operator, which the other tests tie to the oracle
    g = np.arange(7) * 3.0
    centres = np.array([[x, y, z] for x in g for y in g for z in g])
    with mfs.Context(0) as ctx:
        ctx.set_spheres(centres)
        ctx.build(n_proxy=160, r_proxy=0.63, m_basic=480, **FAR)
        s = ctx.sizes()
        assert s.pairs_far_eq > 10 * s.pairs_near_fp
        v, om = workloads.rigid_velocities(len(centres), seed=2)
        ctx.set_rigid_velocities(v, om)
        mu = ctx.rhs()
        exact = ctx.apply_operator(mu, mfs.MIXED)
        packed = ctx.apply_operator(mu, mfs.MIXED_PASS)
        assert np.abs(packed - exact).max() <= 1e-5 * np.abs(exact).max()
        shapes = ctx.tune_pairs()
        tuned = ctx.apply_operator(mu, mfs.MIXED_PASS)
        assert np.abs(tuned - exact).max() <= 1e-5 * np.abs(exact).max()
        assert shapes.far_packed in (0, 1)
