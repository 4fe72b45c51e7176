"""The step-1 entry point that allocates no device memory, against mfs_apply_precond.

Some callers cannot let a library allocate device memory while they run, for example an
application that hands all GPU memory to its own pool and forbids cudaMalloc/cudaFree
(which also synchronise the device) inside its time-stepping loop.  For them the library
offers mfs_apply_precond_noalloc: the caller passes device buffers in and out, and the
intermediate vector lives in a fixed array the library reserves on the GPU.  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_precond_matches_allocating_entry_point():
    import torch
    from paper_2407_03343_gb300 import mfs, workloads

    with mfs.Context(0) as ctx:
        ctx.set_spheres(workloads.two_spheres(0.05))
        ctx.build(n_proxy=200, r_proxy=0.7, m_basic=300, nim_fixed=6)
        s = ctx.sizes()
        rng = np.random.default_rng(21)
        for call in range(2):   # two calls in a row share the fixed scratch
            mu = rng.normal(size=3 * s.n_colloc)
            ref = ctx.apply_precond(mu, mfs.FP64)
            d_mu = torch.tensor(mu, dtype=torch.float64, device="cuda:0")
            d_out = torch.full((s.n_unknowns,), float("nan"), dtype=torch.float64, device="cuda:0")
            torch.cuda.synchronize()
            ctx.apply_precond_noalloc(d_mu.data_ptr(), d_out.data_ptr())
            out = d_out.cpu().numpy()
            assert np.all(np.isfinite(out))
            assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
