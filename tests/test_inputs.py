"""Seeded input generators (CPU): sizes, open-axis flags and determinism of
the free-surface workloads; they hold no arithmetic of the method."""
import numpy as np

import fire_inputs as fi


def test_slab_sizes_flags_and_shift():
    c = fi.rgl_slab(ncell=6, nz=4, n_vac=2, sigma=0.0, vacuum=10.0)
    assert c.n == 4 * 6 * 6 * 4 - 2
    assert c.periodic == (1, 1, 0)
    assert np.allclose(c.box, [6 * fi.CU_A, 6 * fi.CU_A, 4 * fi.CU_A + 10.0])
    assert c.x[:, 2].min() >= 0.0 and c.x[:, 2].max() < 4 * fi.CU_A
    d = fi.rgl_slab(ncell=6, nz=4, n_vac=2, sigma=0.0, vacuum=10.0, z_shift=-1.0)
    assert np.allclose(d.x[:, 2], c.x[:, 2] - 1.0) and d.x[:, 2].min() < 0.0


def test_cluster_is_a_sphere_of_lattice_sites():
    c = fi.rgl_cluster(radius=7.0, sigma=0.0, centre=(7.5, 7.5, 7.5), box=15.0)
    assert c.periodic == (0, 0, 0)
    r = np.linalg.norm(c.x - 7.5, axis=1)
    assert r.max() <= 7.0 + 1e-12
    # nearest-neighbour distance of FCC Cu
    d = np.linalg.norm(c.x[:, None] - c.x[None], axis=2) + np.eye(c.n) * 1e9
    assert np.allclose(d.min(axis=1), fi.CU_A / np.sqrt(2.0))


def test_si_slab_matches_the_silicon_vacancy_case_shape():
    c = fi.sw_si_slab()
    assert c.n == 8 * 16 ** 3 - 5 == 32763
    assert c.periodic == (1, 1, 0)
    assert len(c.meta["vacancies"]) == 5


def test_generators_are_deterministic():
    for make in (lambda: fi.rgl_slab(seed=5), lambda: fi.rgl_cluster(seed=5),
                 lambda: fi.sw_si_slab(ncell=4, seed=5)):
        a, b = make(), make()
        assert np.array_equal(a.x, b.x)
