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
