"""The FP64 half-list passes on shared-memory tiles (fire_set_pair_tiles)
against the FP64 CPU oracle, through the C ABI.

With tiles the neighbour terms of a brick of cells are summed in shared
memory in fixed point and flushed once per staged atom; pairs beyond the
stage (stage_cap), and terms of 15 eV/A or more, take the per-pair FP64
atomics.  Every case here forces the tiles on (FIRE_TILES_ON) on boxes
small enough for the oracle, including ragged bricks at the box edges, a
stage cap small enough that most pairs overflow, a compressed pair that
takes the analytic fall-back and the global path, and an open axis.  Bars
as for the untiled FP64 form: forces within 1e-10 relative, energies
within 1e-12, relaxations within 1e-8 eV/atom and 5 % in iterations.
"""
import numpy as np
import pytest

import fire_inputs as fi
import oracle
import paper_1908_02038_gb300 as fg

pytestmark = pytest.mark.gpu

F_REL = 1e-10
E_REL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    fg.build()
    fg.load_library()


def rgl_pot():
    return fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **fi.RGL_CU)


def ora_rgl():
    return oracle.Potential("rgl", **fi.RGL_CU)


def rel(f, fo):
    return np.abs(f - fo).max() / np.abs(fo).max()


def tiled_eval(c, tiles=fg.FIRE_TILES_ON, stage_cap=0, periodic=(1, 1, 1)):
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT, periodic=periodic) as h:
        h.set_pair_tiles(tiles, stage_cap)
        return h.energy_forces(c.x, c.box)


# 5^3: 3 cells per axis, two tiles; 7^3: one brick of 4 x 4 x 2 cells and a
# ragged one; 9^3: 6 cells per axis, 2 x 2 x 3 bricks
@pytest.mark.parametrize("ncell,nvac,stage_cap", [(5, 3, 0), (7, 10, 0), (9, 7, 0), (9, 7, 64),
                                                  (9, 7, 300)])
def test_tiled_forces_match_oracle(ncell, nvac, stage_cap):
    c = fi.rgl_vacancy_box(ncell=ncell, seed=60 + ncell, n_vac=nvac, sigma=0.08)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl())
    e, f = tiled_eval(c, stage_cap=stage_cap)
    assert rel(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)


def test_tiled_forces_32k_match_oracle_and_untiled():
    c = fi.rgl_vacancy_box(ncell=20, seed=2)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl(), mode=oracle.FORCE_CELLS)
    e, f = tiled_eval(c)
    assert rel(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)
    e0, f0 = tiled_eval(c, tiles=fg.FIRE_TILES_OFF)
    # the two paths differ only in the rounding of their sums
    assert rel(f, f0) < 1e-11
    assert e == pytest.approx(e0, rel=1e-13)


def test_tiled_compressed_pair_takes_the_fallback_paths():
    """A pair pushed to 1.2 A (< r0/2: analytic terms; pair force ~250 eV/A:
    beyond the fixed-point range, so its neighbour term takes the FP64
    atomic)."""
    c = fi.rgl_vacancy_box(ncell=7, seed=66, n_vac=2, sigma=0.05)
    x = c.x.copy()
    d = x[1:] - x[0]
    d -= c.box * np.rint(d / c.box)
    j = 1 + int(np.argmin(np.sum(d * d, 1)))
    u = d[j - 1] / np.linalg.norm(d[j - 1])
    x[j] = x[0] + 1.2 * u
    c = fi.Config("compressed", x, c.box)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl())
    assert np.abs(fo).max() > 100.0
    e, f = tiled_eval(c)
    assert rel(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)


def test_tiled_forces_open_axis_match_oracle():
    c = fi.rgl_slab(ncell=9, nz=8, n_vac=3, sigma=0.08, vacuum=8.0)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl(), periodic=c.periodic)
    e, f = tiled_eval(c, periodic=c.periodic)
    assert rel(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)


@pytest.mark.parametrize("exec_mode,chunk", [(fg.FIRE_EXEC_GRAPH_WHILE, 1),
                                             (fg.FIRE_EXEC_GRAPH_WHILE, 0),
                                             (fg.FIRE_EXEC_CHUNKED, 32)])
def test_tiled_relaxation_32k_parity(exec_mode, chunk, oracle_32k):
    c, xo, ro = oracle_32k
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        h.set_pair_tiles(fg.FIRE_TILES_ON)
        h.set_exec_mode(exec_mode, chunk)
        r = h.minimize(x, c.box, 1e-6, 100000)
    assert r.stop == fg.FIRE_STOP_FTOL and r.fmax_atom < 1e-6
    assert r.force_evals == r.iterations + 1 and r.nbr_builds >= 1
    assert abs(r.energy - ro.energy) / c.n < 1e-8
    assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations), \
        (r.iterations, ro.iterations)


@pytest.fixture(scope="module")
def oracle_32k():
    c = fi.rgl_vacancy_box(ncell=20, seed=2)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT),
                             fi.CU_MASS, 1e-6, 100000, mode=oracle.FORCE_CELLS)
    assert ro.stop == oracle.STOP_FTOL
    return c, xo, ro


def test_tile_setting_rejects_bad_arguments():
    c = fi.rgl_vacancy_box(ncell=5, seed=61, n_vac=1)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        for mode, cap in ((3, 0), (fg.FIRE_TILES_ON, 10), (fg.FIRE_TILES_ON, 5000)):
            with pytest.raises(fg.FireError) as e:
                h.set_pair_tiles(mode, cap)
            assert e.value.status == fg.FIRE_ERR_ARG


def test_tiled_forces_1m_sampled_match_oracle():
    """The 997,450-atom void box (2,541 tiles) on tiles: 2,048 sampled atoms
    against the oracle's forces, the energy against the oracle's total."""
    c = fi.rgl_void_box()
    rng = np.random.default_rng(9)
    which = np.sort(rng.choice(c.n, size=2048, replace=False))
    eo, fo = oracle.energy_forces_subset(c.x, c.box, ora_rgl(), which, mode=oracle.FORCE_CELLS)
    e, f = tiled_eval(c)
    assert rel(f[which], fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)
    assert np.abs(f.sum(0)).max() < 1e-9 * np.abs(f).max() * np.sqrt(c.n)
