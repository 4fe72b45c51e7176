"""Step 1 of the MIXED passes on the tensor cores for the spheres that share the basic factor.

Equal spheres without contacts share one pseudo-inverse (Sec. 2.2), so their products with
Sigma^+ U^T (and, with the far field, with Q) form one matrix product, which the library runs on
the tcgen05 tensor cores in bf16 slices with FP32 accumulation.  Checked through the C ABI:
  * the pass operator with the tensor path matches the one with batched GEMVs to 1e-6 of its
    largest value (both carry FP32-accurate step-1 products) and the oracle's exact operator
    to 1e-6 (smooth data, a Krylov-like vector);
  * a MIXED solve that uses it meets the stated targets against the oracle's O3 solve
    (forces/torques 1e-5, velocity 1e-3);
  * with the far field on, the equivalent strengths of those spheres come from the tensor
    product as well, and the operator still matches the exact oracle to the far-field bound.
Sizes: 26 contact-free spheres on a lattice (one 128-column tile, three 128-row tiles of
Sigma^+ U^T, ragged in both), plus one near-contact pair with images.
"""
import numpy as np
import pytest

from oracle import geometry, solve
from paper_2407_03343_gb300 import mfs, workloads

pytestmark = pytest.mark.gpu

KW = dict(n_proxy=120, r_proxy=0.63, m_basic=240)


def lattice():
    g = np.arange(3) * 3.0
    c = np.array([[x, y, z] for x in g for y in g for z in g])
    c = c[1:]                                     # 26 spheres, 1 radius apart
    pair = np.array([[12.0, 0.0, 0.0], [14.05, 0.0, 0.0]])   # gap 0.05: images and caps
    return np.vstack([c, pair])


@pytest.fixture(scope="module")
def setup():
    centres = lattice()
    d = geometry.build(centres, 1.0, geometry.Params(**KW))
    op = solve.Operator(d)
    ctxs = {}
    for name, kw in (("tensor", dict(tensor_step1=2)), ("gemv", dict(tensor_step1=0)),
                     ("tensor_far", dict(tensor_step1=2, far_dist=4.0))):
        c = mfs.Context(0)
        c.set_spheres(centres)
        c.build(**KW, **kw)
        ctxs[name] = c
    yield centres, d, op, ctxs
    for c in ctxs.values():
        c.close()


def _vectors(d, op):
    v, om = workloads.rigid_velocities(len(d.spheres), seed=5)
    mu = np.concatenate(solve.rhs(d, v, om))
    x = mu.copy()
    for _ in range(4):
        x = op.apply(x)
        x /= np.abs(x).max()
    return mu, x


def test_tensor_pass_operator(setup):
    centres, d, op, ctxs = setup
    assert len(d.contacts) == 1
    for vec in _vectors(d, op):
        ref = op.apply(vec)
        scale = np.abs(ref).max()
        a = ctxs["tensor"].apply_operator(vec, mfs.MIXED_PASS)
        b = ctxs["gemv"].apply_operator(vec, mfs.MIXED_PASS)
        assert not np.array_equal(a, b)            # the two paths really differ
        assert np.abs(a - b).max() <= 1e-6 * scale
        assert np.abs(a - ref).max() <= 1e-6 * scale
        f = ctxs["tensor_far"].apply_operator(vec, mfs.MIXED_PASS)
        assert np.abs(f - ref).max() <= 1e-5 * scale


def test_tensor_solve_matches_oracle(setup):
    centres, d, op, ctxs = setup
    v, om = workloads.rigid_velocities(len(d.spheres), seed=6)
    sol = solve.solve_o3(d, v, om, op=op, tol=1e-9)
    Fo, To = solve.forces_torques(d, sol.lam)
    ref = np.abs(np.r_[Fo.ravel(), To.ravel()]).max()
    x = np.concatenate(d.check)
    uo = solve.velocity(d, sol.lam, x)
    for name in ("tensor", "tensor_far"):
        c = ctxs[name]
        c.set_rigid_velocities(v, om)
        info = c.solve(precision="mixed", tol=1e-8)
        assert info.converged == 1
        F, T = c.forces_torques()
        assert np.abs(np.r_[F.ravel() - Fo.ravel(), T.ravel() - To.ravel()]).max() <= 1e-5 * ref, name
        assert np.abs(c.eval_velocity(x) - uo).max() <= 1e-3 * np.abs(uo).max(), name
