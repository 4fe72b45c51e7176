"""One-body factors shared across contexts, and step 1 on the tensor cores across the problems of
a lockstep batch.

Equal spheres without images have the same self block, so one truncated pseudo-inverse serves
all of them (Sec. 2.2; Sec. 4 needs a single SVD for equal spheres).  The library keeps such
factors in a process-wide store per device: a context whose spheres have the same block (same
radius, viscosity, proxy and collocation grids, truncation and far-field settings) takes the
factor from there instead of computing it, and a lockstep batch puts the spheres of every
problem that hold the same entry into the columns of one tensor-core product (bf16 slices, FP32
accumulation; the other spheres keep the batched GEMV).  Checked through the C ABI:
  * reuse across contexts, no reuse when an input of the block differs, none for spheres with
    images, and the entry outlives the context that computed it;
  * a solve on a taken factor equals one on a freshly computed factor to the solver tolerance;
  * a batch whose problems mix contact-free spheres and a contact pair, and a batch of several
    right-hand sides on one geometry, run their contact-free spheres through the tensor-core
    product (its column counter) and reproduce the single solves to 1e-6 of the largest
    force/torque (both MIXED at tol 1e-9, the single solves through the single-context tensor
    path, which tests/test_gpu_tensor_step1.py ties to the oracle).
"""
import numpy as np
import pytest

from paper_2407_03343_gb300 import mfs, workloads

pytestmark = pytest.mark.gpu

KW = dict(n_proxy=120, r_proxy=0.66, m_basic=260)


def lattice(n, spacing, offset=(0.0, 0.0, 0.0)):
    g = np.arange(n) * spacing
    return np.array([[x, y, z] for x in g for y in g for z in g]) + np.asarray(offset)


def _ctx(centres, **kw):
    c = mfs.Context(0)
    c.set_spheres(centres)
    c.build(**{**KW, **kw})
    return c


def _ft(ctx):
    F, T = ctx.forces_torques()
    return np.concatenate([F.ravel(), T.ravel()])


def test_store_reuse_and_lifetime():
    c1 = _ctx(lattice(2, 3.0))
    s1 = c1.sizes()
    assert s1.n_factors == 1 and s1.n_factors_shared == 1 and s1.n_factors_reused == 0
    # other positions, same block: taken from the store
    c2 = _ctx(lattice(2, 3.5, (0.3, -1.0, 2.0)))
    s2 = c2.sizes()
    assert s2.n_factors_shared == 1 and s2.n_factors_reused == 1
    assert c2.memory_in_use() > 0
    # a different proxy radius is a different block
    c3 = _ctx(lattice(2, 3.0), r_proxy=0.7)
    assert c3.sizes().n_factors_reused == 0
    # spheres with images keep their own factors
    c4 = _ctx(workloads.two_spheres(0.05))
    s4 = c4.sizes()
    assert s4.n_factors == 2 and s4.n_factors_shared == 0 and s4.n_factors_reused == 0
    c3.close()
    c4.close()
    v, w = workloads.rigid_velocities(8, seed=3)
    c2.set_rigid_velocities(v, w)
    assert c2.solve(precision="mixed", tol=1e-10).converged
    ft_shared = _ft(c2)
    # the entry outlives the context that computed it
    c1.close()
    assert c2.solve(precision="mixed", tol=1e-10).converged
    assert np.abs(_ft(c2) - ft_shared).max() <= 1e-12 * np.abs(ft_shared).max()
    c2.close()
    # every holder closed: the next build computes the factor again; same answer to the tolerance
    c5 = _ctx(lattice(2, 3.5, (0.3, -1.0, 2.0)))
    assert c5.sizes().n_factors_reused == 0
    c5.set_rigid_velocities(v, w)
    assert c5.solve(precision="mixed", tol=1e-10).converged
    ft_fresh = _ft(c5)
    c5.close()
    assert np.abs(ft_fresh - ft_shared).max() <= 1e-8 * np.abs(ft_fresh).max()


def _problems():
    pair = workloads.two_spheres(0.05) + np.array([12.0, 0.0, 0.0])
    return [lattice(2, 3.0),                                   # 8 free spheres
            np.vstack([lattice(2, 3.2, (0.5, 0.0, 0.0)), pair]),  # 8 free + a contact pair
            lattice(3, 2.6)[:20]]                              # 20 free spheres, gaps 0.6


def test_batch_tensor_columns_match_single_solves():
    cents = _problems()
    ctxs = [_ctx(c, tensor_step1=2) for c in cents]
    try:
        assert all(c.sizes().n_factors_reused == (0 if i == 0 else 1) for i, c in enumerate(ctxs))
        vel = [workloads.rigid_velocities(c.shape[0], seed=40 + i) for i, c in enumerate(cents)]
        ref = []
        for c, (v, w) in zip(ctxs, vel):
            c.set_rigid_velocities(v, w)
            assert c.solve(precision="mixed", tol=1e-9).converged
            ref.append(_ft(c))
        for c in ctxs:
            c.set_profiling(True)
            c.timing(reset=True)
        infos = mfs.batch_solve(ctxs, precision="mixed", tol=1e-9)
        assert all(i.converged == 1 for i in infos)
        t = ctxs[0].timing(reset=True)
        # the 36 contact-free spheres of the three problems form the columns of each product
        # (every active problem brings at least its 8 contact-free spheres)
        assert t.tc_launches > 0 and 8 * t.tc_launches <= t.tc_columns <= 36 * t.tc_launches
        for c, r in zip(ctxs, ref):
            assert np.abs(_ft(c) - r).max() <= 1e-6 * np.abs(r).max()
    finally:
        for c in ctxs:
            c.close()


def test_batch_rhs_on_one_geometry_uses_tensor_columns():
    # several right-hand sides on one cluster (e.g. the columns of its resistance matrix)
    cent = lattice(3, 2.5)[:18]
    ctx = _ctx(cent, tensor_step1=2)
    try:
        vel = [workloads.rigid_velocities(18, seed=60 + i) for i in range(4)]
        ref = []
        for v, w in vel:
            ctx.set_rigid_velocities(v, w)
            assert ctx.solve(precision="mixed", tol=1e-9).converged
            ref.append(_ft(ctx))
        ctx.set_profiling(True)
        ctx.timing(reset=True)
        infos, outs = mfs.batch_solve_rhs([ctx] * 4, vel, precision="mixed", tol=1e-9)
        assert all(i.converged == 1 for i in infos)
        t = ctx.timing(reset=True)
        assert t.tc_launches > 0 and t.tc_columns > 0
        for (F, T), r in zip(outs, ref):
            got = np.concatenate([F.ravel(), T.ravel()])
            assert np.abs(got - r).max() <= 1e-6 * np.abs(r).max()
    finally:
        ctx.close()


def test_batch_without_tensor_setting_keeps_gemv():
    cents = _problems()[:2]
    ctxs = [_ctx(c, tensor_step1=0) for c in cents]
    try:
        for i, c in enumerate(ctxs):
            c.set_rigid_velocities(*workloads.rigid_velocities(cents[i].shape[0], seed=80 + i))
            c.set_profiling(True)
            c.timing(reset=True)
        infos = mfs.batch_solve(ctxs, precision="mixed", tol=1e-8)
        assert all(i.converged == 1 for i in infos)
        assert ctxs[0].timing(reset=True).tc_launches == 0
    finally:
        for c in ctxs:
            c.close()
