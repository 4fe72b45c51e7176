"""Plain, slow FP64 CPU oracle for the image-enhanced method of fundamental solutions.

TEST INFRASTRUCTURE ONLY.  This package restates the method of Broms, Barnett and
Tornberg (arXiv 2407.03343) step by step in numpy float64 so that the CUDA library can
be checked against it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path (the C-ABI library
and its Python binding) never does, and shares no code with it.

Modules
-------
geometry   discretisation: proxy/collocation grids, contacts, image lines, caps,
           area weights (Sec. 2.1, Sec. 2.3, Sec. 5.1).
kernels    Stokeslet, rotlet and potential-dipole 3x3 blocks (Sec. 2.1 eq. stokeslet,
           Sec. 2.3 rotlet and eq. doublet).
solve      dense target-from-source assembly, one-body truncated pseudo-inverses,
           the three-step preconditioned apply (Sec. 2.2), the three solvers
           O1 (dense Householder-QR least squares, eq. lq / eq. lq2),
           O2 (dense LU of the preconditioned system, eq. resistance),
           O3 (matrix-free GMRES on eq. resistance), and the outputs
           (forces/torques, Sec. 2.3 remark; velocities and residuals, Sec. 3).
brenner    Brenner's series for two squeezing spheres (Sec. 3, eq. Brenner).

Parity status: every function is pinned by a ``-m "not gpu"`` test against closed
forms, invariants or brute force, except the many-sphere physical accuracy of the
discretisation itself (node sets differ from the paper's spherical designs), which is
"parity unpinned" beyond the paper's own accuracy claim.
"""
