"""Parity of the benchmarked configuration itself against the oracle.

The 54 gap-sweep problems are solved exactly as bench.py times them: 18 contexts (two unit
spheres, gaps 10^(-3 + 3 i / 17), N = 800, R_p = 0.63, M0 = 1600, images and caps by the
n_im rule), each with the three motions, in one lockstep batch through
mfs_batch_solve_rhs_device with bench.py's options (MIXED, its tolerance and restart,
MFS_RESIDUAL_AUTO, which at that tolerance evaluates the refinement residual with the
double-float operator).  The reference values are the oracle's O3 solutions to 1e-9 stored by
tests/golden/make_gap_sweep_oracle.py.

Checked at the benchmarked tolerance (the paper's GMRES tolerance 1e-6), for every problem: the
disturbance velocity at the stored check points to 1e-3 relative (the stated surface-velocity
target, eq. residual_x), and forces and torques (Sec. 2.3 remark) to 1e-3 relative, which is as
far as a solve to that residual converges them (counter-rotation at gap 1e-3, the slowest
problem, sits near 5e-4; the median is ~1e-7).  The same batch in plain FP64 is held to the
same bounds.  With the tolerance tightened to 1e-9 the same batch meets the stated
force/torque target 1e-5 on all 54 problems.
"""
import json
import os

import numpy as np
import pytest
import torch

import bench
from paper_2407_03343_gb300 import mfs, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sweep():
    if not os.path.exists(bench.GOLDEN):
        pytest.fail("oracle values missing: run tests/golden/make_gap_sweep_oracle.py")
    gold = json.load(open(bench.GOLDEN))
    assert gold["params"] == dict(n_proxy=bench.N_PROXY, r_proxy=bench.R_PROXY, m_basic=bench.M_BASIC)
    gaps = workloads.gap_sweep_gaps()
    assert np.allclose(gold["gaps"], gaps, rtol=0, atol=0)
    ctxs = []
    for g in gaps:
        c = mfs.Context(0)
        c.set_spheres(workloads.two_spheres(g))
        c.build(n_proxy=bench.N_PROXY, r_proxy=bench.R_PROXY, m_basic=bench.M_BASIC)
        ctxs.append(c)
    yield gold, ctxs
    for c in ctxs:
        c.close()


def _run(ctxs, motions, opts):
    dev = torch.device("cuda", 0)
    probs, vp, wp, Fp, Tp, keep, outs = [], [], [], [], [], [], []
    for m in motions:
        v, w = workloads.motion(m)
        tv = torch.tensor(v, dtype=torch.float64, device=dev)
        tw = torch.tensor(w, dtype=torch.float64, device=dev)
        keep += [tv, tw]
        for c in ctxs:
            F = torch.zeros((2, 3), dtype=torch.float64, device=dev)
            T = torch.zeros((2, 3), dtype=torch.float64, device=dev)
            probs.append(c)
            vp.append(tv.data_ptr())
            wp.append(tw.data_ptr())
            Fp.append(F.data_ptr())
            Tp.append(T.data_ptr())
            outs.append((F, T))
    torch.cuda.synchronize()
    infos = mfs.batch_solve_rhs_device(probs, vp, wp, Fp, Tp, opts)
    torch.cuda.synchronize()
    return infos, [(F.cpu().numpy(), T.cpu().numpy()) for F, T in outs]


def _ft_err(F, T, g):
    Fo, To = np.array(g["F"]), np.array(g["T"])
    ref = max(np.abs(Fo).max(), np.abs(To).max())
    return max(np.abs(F - Fo).max(), np.abs(T - To).max()) / ref


def _u_err(ctx, geo, m_index):
    x = np.array(geo["check_points"])
    uo = np.array(geo["problems"][m_index]["u"])
    return np.abs(ctx.eval_velocity(x) - uo).max() / np.abs(uo).max()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_benchmarked_sweep_matches_oracle(sweep, precision):
    gold, ctxs = sweep
    ng = len(ctxs)
    opts = mfs.default_solve_opts(precision=precision, tol=bench.SWEEP_TOL, restart=bench.SWEEP_RESTART)
    assert opts.residual == mfs.RESIDUAL_AUTO
    infos, outs = _run(ctxs, bench.MOTIONS, opts)
    assert all(i.converged == 1 and i.rel_residual <= bench.SWEEP_TOL for i in infos)
    ft = [_ft_err(F, T, gold["geometries"][i % ng]["problems"][i // ng]) for i, (F, T) in enumerate(outs)]
    assert max(ft) <= 1e-3, f"force/torque error {max(ft):.3e} (problem {int(np.argmax(ft))})"
    assert np.median(ft) <= 1e-5
    # each context holds its last problem (the last motion): surface velocity at the check points
    last = len(bench.MOTIONS) - 1
    u = [_u_err(c, gold["geometries"][gi], last) for gi, c in enumerate(ctxs)]
    assert max(u) <= 1e-3, f"velocity error {max(u):.3e}"


def test_tight_tolerance_sweep_meets_force_target(sweep):
    gold, ctxs = sweep
    ng = len(ctxs)
    opts = mfs.default_solve_opts(precision="mixed", tol=1e-9, restart=bench.SWEEP_RESTART)
    infos, outs = _run(ctxs, bench.MOTIONS, opts)
    assert all(i.converged == 1 for i in infos)
    ft = [_ft_err(F, T, gold["geometries"][i % ng]["problems"][i // ng]) for i, (F, T) in enumerate(outs)]
    assert max(ft) <= 1e-5, f"force/torque error {max(ft):.3e} (problem {int(np.argmax(ft))})"
    last = len(bench.MOTIONS) - 1
    assert max(_u_err(c, gold["geometries"][gi], last) for gi, c in enumerate(ctxs)) <= 1e-5


def test_benchmarked_options_per_motion_velocity(sweep):
    # the same options, one motion per batch, so that every problem's velocity field is checked
    gold, ctxs = sweep
    opts = mfs.default_solve_opts(precision="mixed", tol=bench.SWEEP_TOL, restart=bench.SWEEP_RESTART)
    for mi, m in enumerate(bench.MOTIONS[:-1]):
        infos, outs = _run(ctxs, [m], opts)
        assert all(i.converged == 1 for i in infos)
        for gi, c in enumerate(ctxs):
            assert _ft_err(*outs[gi], gold["geometries"][gi]["problems"][mi]) <= 1e-3
            assert _u_err(c, gold["geometries"][gi], mi) <= 1e-3
