"""Lockstep batched solve (mfs_batch_solve) against one-by-one solves of the same problems.

Each problem keeps its own Krylov coefficients and convergence test inside the batch, so the
results must agree with independent solves to the solver tolerance; a short restart length
exercises the refinement passes that replace GMRES restarts in the batch.
"""
import numpy as np
import pytest

from paper_2407_03343_gb300 import mfs, workloads

pytestmark = pytest.mark.gpu
KW = dict(n_proxy=200, r_proxy=0.63, m_basic=400)


@pytest.fixture(scope="module")
def problems():
    ctxs, P = [], []
    for g in (1e-3, 0.02, 0.3):
        c = mfs.Context(0)
        c.set_spheres(workloads.two_spheres(g))
        c.build(**KW)
        ctxs.append(c)
        P.append(2)
    c = mfs.Context(0)
    centres = workloads.suspension(4, 0.15, seed=2)
    c.set_spheres(centres)
    c.build(**KW)
    ctxs.append(c)
    P.append(4)
    yield ctxs, P
    for c in ctxs:
        c.close()


def ft(ctx):
    F, T = ctx.forces_torques()
    return np.concatenate([F.ravel(), T.ravel()])


@pytest.mark.parametrize("precision,tol,restart", [("fp64", 1e-9, 300), ("mixed", 1e-8, 300), ("mixed", 1e-8, 100)])
def test_batch_matches_single(problems, precision, tol, restart):
    ctxs, P = problems
    rng = np.random.default_rng(4)
    vel = [(rng.normal(size=(p, 3)), rng.normal(size=(p, 3))) for p in P]
    for c, (v, w) in zip(ctxs, vel):
        c.set_rigid_velocities(v, w)
    infos = mfs.batch_solve(ctxs, precision=precision, tol=tol, restart=restart)
    assert all(i.converged == 1 and i.rel_residual <= tol for i in infos)
    batched = [ft(c) for c in ctxs]
    for c, (v, w), fb in zip(ctxs, vel, batched):
        c.set_rigid_velocities(v, w)
        c.solve(precision=precision, tol=tol)
        fs = ft(c)
        assert np.abs(fb - fs).max() <= 1e-5 * np.abs(fs).max()


def test_batch_zero_data_and_outputs(problems):
    ctxs, P = problems
    for c, p in zip(ctxs, P):
        c.set_rigid_velocities(np.zeros((p, 3)), np.zeros((p, 3)))
    infos = mfs.batch_solve(ctxs, precision="mixed")
    assert all(i.converged == 1 and i.iters == 0 for i in infos)
    assert all(np.all(ft(c) == 0) for c in ctxs)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-8)])
def test_repeated_contexts_with_several_right_hand_sides(problems, precision, tol):
    ctxs, P = problems
    rng = np.random.default_rng(9)
    order = [0, 3, 0, 1, 3, 0]            # contexts repeat: several right-hand sides per geometry
    probs = [ctxs[i] for i in order]
    vel = [(rng.normal(size=(P[i], 3)), rng.normal(size=(P[i], 3))) for i in order]
    infos, outs = mfs.batch_solve_rhs(probs, vel, precision=precision, tol=tol)
    assert all(i.converged == 1 for i in infos)
    for c, (v, w), (F, T) in zip(probs, vel, outs):
        c.set_rigid_velocities(v, w)
        c.solve(precision=precision, tol=tol)
        Fs, Ts = c.forces_torques()
        ref = np.abs(np.r_[Fs.ravel(), Ts.ravel()]).max()
        assert np.abs(np.r_[F.ravel() - Fs.ravel(), T.ravel() - Ts.ravel()]).max() <= 1e-5 * ref


def test_repeated_contexts_device_buffers(problems):
    import torch
    ctxs, P = problems
    rng = np.random.default_rng(10)
    order = [1, 1, 2]
    probs = [ctxs[i] for i in order]
    vel = [(rng.normal(size=(P[i], 3)), rng.normal(size=(P[i], 3))) for i in order]
    dv = [torch.tensor(v, dtype=torch.float64, device="cuda:0") for v, _ in vel]
    dw = [torch.tensor(w, dtype=torch.float64, device="cuda:0") for _, w in vel]
    dF = [torch.zeros((P[i], 3), dtype=torch.float64, device="cuda:0") for i in order]
    dT = [torch.zeros((P[i], 3), dtype=torch.float64, device="cuda:0") for i in order]
    torch.cuda.synchronize()
    mfs.batch_solve_rhs_device(probs, [t.data_ptr() for t in dv], [t.data_ptr() for t in dw],
                               [t.data_ptr() for t in dF], [t.data_ptr() for t in dT], precision="mixed", tol=1e-8)
    torch.cuda.synchronize()
    _, outs = mfs.batch_solve_rhs(probs, vel, precision="mixed", tol=1e-8)
    for (F, T), f, t in zip(outs, dF, dT):
        ref = np.abs(np.r_[F.ravel(), T.ravel()]).max()
        assert np.abs(f.cpu().numpy() - F).max() <= 1e-9 * ref and np.abs(t.cpu().numpy() - T).max() <= 1e-9 * ref


def test_batch_of_64_problems_up_to_256_spheres():
    # the shape of the batched workload (64 independent suspensions, sphere counts from 2 to 256,
    # gaps of attached spheres log-uniform in [1e-3, 1e-1]) at a reduced discretisation: 63
    # suspensions with 2 to 12 spheres and one of 256 spheres (a dilute lattice with three
    # near-contact pairs, so most of its spheres share the basic factor and run step 1 on the
    # tensor cores).  The MIXED batch must reproduce one-by-one solves of a sample of its problems
    # to the accuracy their residual allows: both reach 1e-8 (the MIXED floor at this
    # discretisation is ~1.6e-9), and the forces of the gap-2e-3 pair amplify a residual
    # difference ~1/gap (measured 3.3e-5 of the largest force), hence 1e-4 there and 1e-5 elsewhere.
    kw = dict(n_proxy=96, r_proxy=0.63, m_basic=200)
    cents = workloads.batch(n_problems=63, seed=9, p_lo=2, p_hi=12)
    g = np.arange(8) * 3.0
    big = np.array([[x, y, z] for x in g for y in g for z in g[:4]])
    for i, gap in enumerate((2e-3, 2e-2, 8e-2)):
        big[4 * i + 1] = big[4 * i] + np.array([0.0, 0.0, 2.0 + gap])  # bring a neighbour close
    cents.append(big)
    assert big.shape[0] == 256 and max(c.shape[0] for c in cents) == 256
    ctxs = []
    try:
        for c in cents:
            ctx = mfs.Context(0)
            ctx.set_spheres(c)
            ctx.build(**kw)
            ctxs.append(ctx)
        assert ctxs[-1].sizes().n_contacts == 3
        vel = [workloads.rigid_velocities(c.shape[0], seed=300 + i) for i, c in enumerate(cents)]
        for ctx, (v, w) in zip(ctxs, vel):
            ctx.set_rigid_velocities(v, w)
        infos = mfs.batch_solve(ctxs, precision="mixed", tol=1e-8)
        assert len(infos) == 64 and all(i.converged == 1 and i.rel_residual <= 1e-8 for i in infos)
        batched = [ft(c) for c in ctxs]
        for i in (0, 17, 40, 62, 63):
            ctxs[i].set_rigid_velocities(*vel[i])
            assert ctxs[i].solve(precision="mixed", tol=1e-8).converged
            fs = ft(ctxs[i])
            assert np.abs(batched[i] - fs).max() <= (1e-4 if i == 63 else 1e-5) * np.abs(fs).max(), i
    finally:
        for ctx in ctxs:
            ctx.close()
