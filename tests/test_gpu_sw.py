"""Stillinger-Weber three-body potential on the GPU (FP64) against the oracle,
through the C ABI."""
import numpy as np
import pytest

import fire_inputs as fi
import oracle
import paper_1908_02038_gb300 as fg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fg.build()
    fg.load_library()
    oracle.build()


def sw_pot(skin=0.3):
    return fg.Potential(fg.FIRE_POT_SW, skin=skin, **fi.SW_SI)


def ora_sw():
    return oracle.Potential("sw", **fi.SW_SI)


@pytest.mark.parametrize("ncell,seed", [(3, 1), (8, 2)])
def test_sw_energy_forces_match_oracle(ncell, seed):
    c = fi.sw_si_vacancy_box(ncell=ncell, seed=seed, n_vac=2, sigma=0.1)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_sw(), mode=oracle.FORCE_CELLS)
    with fg.FireHandle(c.n, fi.SI_MASS, sw_pot(), dt_start=fi.SI_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
    assert np.abs(f - fo).max() / np.abs(fo).max() < 1e-10
    assert e == pytest.approx(eo, rel=1e-12)


def test_sw_perfect_diamond():
    x = fi.diamond_sites(4, fi.SI_A)
    with fg.FireHandle(len(x), fi.SI_MASS, sw_pot(), dt_start=fi.SI_DT) as h:
        e, f = h.energy_forces(x, [4 * fi.SI_A] * 3)
    assert e / len(x) == pytest.approx(-2.0 * fi.SW_SI["eps"], rel=1e-9)
    assert np.abs(f).max() < 1e-11


@pytest.mark.parametrize("ncell", [4, 6])
def test_sw_relaxation_parity(ncell):
    c = fi.sw_si_vacancy_box(ncell=ncell, seed=10 + ncell, n_vac=1, sigma=0.05)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_sw(), oracle.Params(dt_start=fi.SI_DT), fi.SI_MASS,
                             1e-6, 100000, mode=oracle.FORCE_CELLS)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.SI_MASS, sw_pot(), dt_start=fi.SI_DT) as h:
        r = h.minimize(x, c.box, 1e-6, 100000)
    assert ro.stop == oracle.STOP_FTOL and r.stop == fg.FIRE_STOP_FTOL
    assert r.fmax_atom < 1e-6
    assert abs(r.energy - ro.energy) / c.n < 1e-8
    assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations), \
        (r.iterations, ro.iterations)


def test_sw_crowded_neighbourhood_is_an_error():
    rng = np.random.default_rng(3)
    box = np.array([20.0, 20.0, 20.0])
    x = 10.0 + rng.uniform(-1.2, 1.2, size=(60, 3))   # ~60 atoms within a sigma of each other
    with fg.FireHandle(len(x), fi.SI_MASS, sw_pot(), dt_start=fi.SI_DT) as h:
        with pytest.raises(fg.FireError) as e:
            h.energy_forces(x, box)
    assert e.value.status == fg.FIRE_ERR_ARG
    assert "Stillinger-Weber" in str(e.value)
