"""The seeded geometry generators hold the structure the experiments rely on."""
import numpy as np

from paper_2407_03343_gb300 import workloads


def gaps(c):
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2) - 2.0
    np.fill_diagonal(d, np.inf)
    return d


def test_tetrahedron_has_equal_gaps():
    for delta in (0.1, 1e-3):
        g = gaps(workloads.tetrahedron(delta))
        assert np.allclose(g[np.isfinite(g)], delta, rtol=1e-12, atol=1e-14)


def test_cluster_neighbours_sit_at_the_gap():
    c = workloads.cluster(20, 1e-3, seed=2)
    g = gaps(c)
    assert c.shape == (20, 3)
    assert g.min() >= 1e-3 * (1 - 1e-9)
    assert np.all(np.abs(g.min(axis=1) - 1e-3) < 1e-9)
    assert np.array_equal(c, workloads.cluster(20, 1e-3, seed=2))


def test_gap_sweep_and_suspension():
    g = workloads.gap_sweep_gaps()
    assert len(g) == 18 and abs(g[0] - 1e-3) < 1e-15 and abs(g[-1] - 1.0) < 1e-12
    c = workloads.suspension(40, 0.2, seed=3)
    assert gaps(c).min() >= 1e-3 * (1 - 1e-9)
    n, gmin = workloads.count_near_contacts(c)
    assert n > 0 and gmin >= 1e-3 * (1 - 1e-9)
