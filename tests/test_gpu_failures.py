"""Failure paths made on the host, each followed by a successful call on the same context.

Nothing here faults the GPU: the failures are invalid host data (rejected before any launch),
non-finite device data (caught by the solver's finiteness checks on its FP64 norms), and an
allocation refused by the context's memory cap (which fails exactly like a cudaMalloc
failure).  After each, the context must still solve a valid problem.
"""
import math

import numpy as np
import pytest
import torch

from paper_2407_03343_gb300 import mfs, workloads

pytestmark = pytest.mark.gpu

KW = dict(n_proxy=60, r_proxy=0.63, m_basic=100)
ARG, NUMERIC, OOM = -1, -6, -7


def _solved_ok(ctx):
    v, w = workloads.motion("squeeze")
    ctx.set_rigid_velocities(v, w)
    info = ctx.solve(precision="mixed", tol=1e-6)
    F, _ = ctx.forces_torques()
    return info.converged == 1 and np.all(np.isfinite(F))


def test_non_finite_host_data_is_rejected():
    with mfs.Context(0) as ctx:
        ctx.set_spheres(workloads.two_spheres(0.3))
        ctx.build(**KW)
        v, w = workloads.motion("shear")
        bad = v.copy()
        bad[1, 2] = math.nan
        with pytest.raises(mfs.MfsError) as e:
            ctx.set_rigid_velocities(bad, w)
        assert e.value.status == ARG
        bad_w = w.copy()
        bad_w[0, 0] = math.inf
        with pytest.raises(mfs.MfsError) as e:
            ctx.set_rigid_velocities(v, bad_w)
        assert e.value.status == ARG
        with pytest.raises(mfs.MfsError) as e:
            ctx.set_background_flow(U=[0.0, math.nan, 0.0])
        assert e.value.status == ARG
        with pytest.raises(mfs.MfsError) as e:
            ctx.set_background_flow(E=np.diag([1.0, -1.0, math.inf]))
        assert e.value.status == ARG
        with pytest.raises(mfs.MfsError) as e:
            ctx.set_forces_torques(np.full((2, 3), math.nan), np.zeros((2, 3)))
        assert e.value.status == ARG
        assert _solved_ok(ctx)


def test_non_finite_device_data_gives_numeric_error():
    with mfs.Context(0) as ctx:
        ctx.set_spheres(workloads.two_spheres(0.1))
        ctx.build(**KW)
        v = torch.zeros((2, 3), dtype=torch.float64, device="cuda:0")
        w = torch.zeros((2, 3), dtype=torch.float64, device="cuda:0")
        v[0, 0] = float("nan")
        torch.cuda.synchronize()
        ctx.set_rigid_velocities_device(v.data_ptr(), w.data_ptr())
        for prec in ("fp64", "mixed"):
            with pytest.raises(mfs.MfsError) as e:
                ctx.solve(precision=prec)
            assert e.value.status == NUMERIC
        # the batched solver checks its right-hand sides too
        with pytest.raises(mfs.MfsError) as e:
            mfs.batch_solve_rhs_device([ctx], [v.data_ptr()], [w.data_ptr()], [0], [0], precision="mixed")
        assert e.value.status == NUMERIC
        assert _solved_ok(ctx)


def test_memory_cap_refuses_allocations_and_context_recovers():
    with mfs.Context(0) as ctx:
        ctx.set_spheres(workloads.two_spheres(0.05))
        ctx.set_memory_limit(256 * 1024)  # far below what the discretisation and factors need
        with pytest.raises(mfs.MfsError) as e:
            ctx.build(**KW)
        assert e.value.status == OOM
        assert ctx.memory_in_use() == 0  # the failed build released what it had taken
        ctx.set_memory_limit(0)
        ctx.build(**KW)
        used = ctx.memory_in_use()
        assert used > 256 * 1024
        assert _solved_ok(ctx)
        # a cap between the build's holdings and what the Krylov basis needs: the solve fails
        # cleanly, then succeeds once the cap is lifted
        with mfs.Context(0) as c2:
            c2.set_spheres(workloads.two_spheres(0.05))
            c2.build(**KW)
            c2.set_memory_limit(c2.memory_in_use() + 1024)
            v, w = workloads.motion("rotate")
            c2.set_rigid_velocities(v, w)
            with pytest.raises(mfs.MfsError) as e:
                c2.solve(precision="mixed")
            assert e.value.status == OOM
            c2.set_memory_limit(0)
            assert _solved_ok(c2)
