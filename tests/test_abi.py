"""The C-ABI library loads on the CPU host and exports every function include/mfs.h declares."""
import ctypes
import os

import pytest

from paper_2407_03343_gb300 import _build, mfs


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(mfs.LIB_PATH):
        _build.build(force=True)
    return mfs.lib()


def test_exports_every_declared_symbol(L):
    names = mfs.declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing


def test_struct_layouts_match_defaults(L):
    p = mfs.default_params()
    assert p.n_proxy == 686 and abs(p.r_proxy - 0.63) < 1e-15 and p.m_basic == 823
    assert p.alpha1 == 6 and p.alpha2 == 6 and p.nim_max == 20 and p.nim_fixed == -1
    assert abs(p.eps_trunc - 5e-12) < 1e-25 and abs(p.nim_a - 8.72) < 1e-15 and abs(p.visc - 1.0) < 1e-15
    assert p.build_factors == 1 and p.nim_min == 0
    o = mfs.default_solve_opts()
    assert o.precision == mfs.MIXED and abs(o.tol - 1e-6) < 1e-20 and o.restart == 300
    assert o.max_iter == 2000 and o.max_refine == 20 and o.residual == mfs.RESIDUAL_AUTO
    with pytest.raises(KeyError):
        mfs.default_solve_opts(tolerance=1e-3)


def test_null_context_is_rejected_without_gpu(L):
    # argument checks run before any device call
    assert L.mfs_create(None, 0, None) == -1
    assert L.mfs_sizes(None, None) == -1
    assert L.mfs_last_error(None) == b"null context"


def test_header_cites_the_paper():
    txt = open(mfs.HEADER).read()
    for tag in ("eq. resistance", "eq. transform", "eq. uAll", "Sec. 2.3 remark", "eq. bc"):
        assert tag in txt
