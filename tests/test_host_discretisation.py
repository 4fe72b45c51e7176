"""The library's host discretisation (the first step of mfs_build, run here without a GPU
through mfs_discretise_host) against the oracle's independent one: collocation nodes,
area weights, owners, and every vector source with its type, in the library's order."""
import numpy as np
import pytest

from oracle import geometry
from paper_2407_03343_gb300 import mfs, workloads

CASES = {
    "plain method, gap 0.1, 10 images": (workloads.two_spheres(0.1), dict(n_proxy=300, r_proxy=0.7, m_basic=600,
                                                                          nim_fixed=10)),
    "gap sweep, gap 1e-3": (workloads.two_spheres(1e-3), dict(n_proxy=800, r_proxy=0.63, m_basic=1600)),
    "gap sweep, gap 0.2 (no images)": (workloads.two_spheres(0.2), dict(n_proxy=800, r_proxy=0.63, m_basic=1600)),
    "tetrahedron, gap 1e-3": (workloads.tetrahedron(1e-3), dict(n_proxy=686, r_proxy=0.63, m_basic=823)),
    "cluster of 20": (workloads.cluster(20, 1e-3, seed=2), dict(n_proxy=686, r_proxy=0.63, m_basic=823)),
    "suspension of 40": (workloads.suspension(40, 0.2, seed=3), dict(n_proxy=400, r_proxy=0.63, m_basic=800)),
    "minimum images below gap 0.3": (workloads.tetrahedron(0.2), dict(n_proxy=400, r_proxy=0.63, m_basic=800,
                                                                       nim_cut=0.3, nim_min=2)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_host_discretisation_matches_oracle(name):
    centres, kw = CASES[name]
    x, w, owner, pos, typ = mfs.discretise_host(centres, **kw)
    d = geometry.build(centres, 1.0, geometry.Params(**kw))
    X = np.concatenate([s.colloc for s in d.spheres])
    W = np.concatenate([s.weight for s in d.spheres])
    O = np.concatenate([np.full(s.colloc.shape[0], k) for k, s in enumerate(d.spheres)])
    assert x.shape == X.shape
    assert np.abs(x - X).max() <= 1e-12 and np.allclose(w, W, rtol=1e-13) and np.array_equal(owner, O)
    ref_pos = np.concatenate([np.concatenate([s.proxy, np.repeat(s.image, 3, axis=0)]) for s in d.spheres])
    ref_typ = np.concatenate([np.concatenate([np.zeros(s.proxy.shape[0], int), np.tile([0, 1, 2], s.image.shape[0])])
                              for s in d.spheres])
    assert pos.shape == ref_pos.shape
    assert np.abs(pos - ref_pos).max() <= 1e-12 and np.array_equal(typ, ref_typ)


def test_radius_scales_the_discretisation():
    c = workloads.two_spheres(0.05)
    kw = dict(n_proxy=200, r_proxy=0.63, m_basic=300)
    x1, w1, _, p1, _ = mfs.discretise_host(c, 1.0, **kw)
    x2, w2, _, p2, _ = mfs.discretise_host(2.5 * c, 2.5, **kw)
    assert np.allclose(x2, 2.5 * x1, atol=1e-12) and np.allclose(w2, 6.25 * w1, rtol=1e-12)
    assert np.allclose(p2, 2.5 * p1, atol=1e-12)


def test_host_discretisation_errors():
    with pytest.raises(mfs.MfsError, match="GEOMETRY"):
        mfs.discretise_host([[0, 0, 0], [1.5, 0, 0]])          # overlapping spheres
    with pytest.raises(mfs.MfsError, match="ARG"):
        mfs.discretise_host([[0, 0, 0]], radius=-1.0)
    with pytest.raises(mfs.MfsError, match="ARG"):
        mfs.discretise_host([[0, 0, 0]], n_proxy=0)
