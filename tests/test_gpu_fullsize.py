"""Parity at full sizes.

* Gap-sweep problems at the benchmark's sizes (N = 800, R_p = 0.63, M0 = 1600, up to 20
  image points per contact) with random rigid motions, solved as one lockstep batch in the
  mixed mode at the tighter tolerance 1e-8 (so the refinement residual uses the native FP64
  operator), against the matrix-free FP64 oracle (O3) solved on the fly.  The benchmarked
  options themselves (tolerance 1e-6, double-float residual) are checked over all 54 sweep
  problems in test_gpu_sweep_bench_config.py.
* The 200-sphere suspension (volume fraction 0.2, ~300 near contacts, N = 800, M0 = 1600):
  its discretisation element by element, and the pair apply on sampled collocation rows that
  the oracle evaluates one by one (every FP64 / double-float / FP32 kernel, 4 nodes per thread).
"""
import numpy as np
import pytest

from oracle import geometry, solve
from paper_2407_03343_gb300 import mfs, workloads
from tests.layout import oracle_to_lib

pytestmark = pytest.mark.gpu
SWEEP = dict(n_proxy=800, r_proxy=0.63, m_basic=1600)


def ft_err(F, T, Fo, To):
    ref = np.abs(np.r_[Fo.ravel(), To.ravel()]).max()
    return np.abs(np.r_[F.ravel() - Fo.ravel(), T.ravel() - To.ravel()]).max() / ref


def test_gap_sweep_batch_full_size_matches_oracle():
    gaps = [1e-3, 0.05, 0.3]
    ctxs = []
    rng = np.random.default_rng(31)
    vel = []
    for g in gaps:
        c = mfs.Context(0)
        c.set_spheres(workloads.two_spheres(g))
        c.build(**SWEEP)
        v, w = workloads.motion("squeeze")
        v = v + 0.3 * rng.normal(size=(2, 3))
        w = w + 0.3 * rng.normal(size=(2, 3))
        c.set_rigid_velocities(v, w)
        ctxs.append(c)
        vel.append((v, w))
    s0 = ctxs[0].sizes()
    assert s0.n_image_nodes == 40 and s0.n_colloc == 2 * (1600 + 36 * 20)
    infos = mfs.batch_solve(ctxs, precision="mixed", tol=1e-8)
    assert all(i.converged == 1 for i in infos)
    for idx in (0, 2):
        d = geometry.build(workloads.two_spheres(gaps[idx]), 1.0, geometry.Params(**SWEEP))
        op = solve.Operator(d)
        v, w = vel[idx]
        sol = solve.solve_o3(d, v, w, op=op, tol=1e-9)
        F, T = ctxs[idx].forces_torques()
        Fo, To = solve.forces_torques(d, sol.lam)
        assert ft_err(F, T, Fo, To) <= 1e-5
        x = np.concatenate(d.check)
        u = ctxs[idx].eval_velocity(x)
        uo = solve.velocity(d, sol.lam, x)
        assert np.abs(u - uo).max() <= 1e-3 * np.abs(uo).max()
    for c in ctxs:
        c.close()


@pytest.fixture(scope="module")
def suspension():
    centres = workloads.suspension(200, 0.2, seed=3)
    ctx = mfs.Context(0)
    ctx.set_spheres(centres)
    ctx.build(build_factors=0, **SWEEP)
    d = geometry.build(centres, 1.0, geometry.Params(**SWEEP))
    yield ctx, d
    ctx.close()


def test_suspension_discretisation_full_size(suspension):
    ctx, d = suspension
    s = ctx.sizes()
    assert s.P == 200 and s.n_contacts == len(d.contacts) and s.n_contacts > 250
    x, w, owner = ctx.collocation()
    X = np.concatenate([sp.colloc for sp in d.spheres])
    W = np.concatenate([sp.weight for sp in d.spheres])
    assert x.shape == X.shape and np.abs(x - X).max() <= 1e-12 and np.allclose(w, W, rtol=1e-13)
    pos, typ = ctx.source_layout()
    ref = np.concatenate([np.concatenate([sp.proxy, np.repeat(sp.image, 3, axis=0)]) for sp in d.spheres])
    assert np.abs(pos - ref).max() <= 1e-12
    with pytest.raises(mfs.MfsError) as e:
        ctx.solve()
    assert e.value.status == -4


def test_suspension_pair_apply_sampled_rows(suspension):
    ctx, d = suspension
    rng = np.random.default_rng(5)
    lam_o = [rng.normal(size=solve.n_unknowns(d, k)) for k in range(len(d.spheres))]
    lam_l = oracle_to_lib(d, lam_o)
    n_nodes = sum(sp.colloc.shape[0] for sp in d.spheres)
    mu = np.zeros(3 * n_nodes)
    offs = np.concatenate([[0], np.cumsum([sp.colloc.shape[0] for sp in d.spheres])])
    rows = rng.choice(n_nodes, size=240, replace=False)
    ref = np.zeros((rows.size, 3))
    for r, i in enumerate(rows):
        k = int(np.searchsorted(offs, i, side="right") - 1)
        xi = d.spheres[k].colloc[i - offs[k]][None, :]
        acc = np.zeros(3)
        for kp in range(len(d.spheres)):
            if kp != k:
                acc += solve.target_from_source(d, xi, kp) @ lam_o[kp]
        ref[r] = np.sqrt(d.spheres[k].weight[i - offs[k]]) * acc
    scale = np.abs(ref).max()
    for prec, tol in ((mfs.FP64, 1e-11), (mfs.MIXED, 1e-11), (mfs.FP32, 1e-4)):
        out = ctx.apply_pairs(lam_l, mu, prec).reshape(-1, 3)[rows]
        assert np.abs(out - ref).max() <= tol * scale, prec
