"""Open (non-periodic) axes on the cell-list path, GPU vs the FP64 oracle
through the C ABI: Cu slabs periodic in x and y, Cu clusters open on every
axis, atoms lying outside [0, L) on an open axis (they share the edge cells),
the Stillinger-Weber Si slab, and the batched form with an open axis."""
import numpy as np
import pytest

import fire_inputs as fi
import oracle
import paper_1908_02038_gb300 as fg

pytestmark = pytest.mark.gpu

F_REL = 1e-10
F32_ABS = 3e-6       # eV/A, FP32-pair forces against the FP64 oracle
E32_PER_ATOM = 1e-6  # eV/atom


@pytest.fixture(scope="module", autouse=True)
def _built():
    fg.build()
    fg.load_library()


def ora_rgl():
    return oracle.Potential("rgl", **fi.RGL_CU)


FORMS = {
    "fp64_table_half": dict(precision=fg.FIRE_PREC_FP64, pair_eval=fg.FIRE_PAIR_TABLE,
                            newton=fg.FIRE_NEWTON_ON),
    "fp64_table_full": dict(precision=fg.FIRE_PREC_FP64, pair_eval=fg.FIRE_PAIR_TABLE,
                            newton=fg.FIRE_NEWTON_OFF),
    "fp64_exp": dict(precision=fg.FIRE_PREC_FP64, pair_eval=fg.FIRE_PAIR_ANALYTIC),
    "fp32pair": dict(precision=fg.FIRE_PREC_FP32_PAIR, pair_eval=fg.FIRE_PAIR_ANALYTIC),
}


def rgl_pot(form):
    return fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **FORMS[form], **fi.RGL_CU)


def check_forces(form, e, f, eo, fo, n):
    if form == "fp32pair":
        assert np.abs(f - fo).max() < F32_ABS
        assert abs(e - eo) / n < E32_PER_ATOM
    else:
        assert np.abs(f - fo).max() / np.abs(fo).max() < F_REL
        assert e == pytest.approx(eo, rel=1e-12)


CASES = {
    # 862 atoms, 4 x 4 x 5 cells; the lowest layer below z = 0
    "slab": lambda: fi.rgl_slab(ncell=6, n_vac=2, sigma=0.08, z_shift=-1.0),
    # a thick slab: 9 x 9 x 7 cells in the grid
    "slab_thick": lambda: fi.rgl_slab(ncell=9, nz=8, n_vac=3, sigma=0.08, vacuum=8.0),
    # cluster cut by the x = 0 face: a third of it at negative x
    "cluster_edge": lambda: fi.rgl_cluster(radius=11.0, centre=(3.0, 16.0, 15.0), box=32.0),
    # open box smaller than three cells on every axis
    "cluster_small_box": lambda: fi.rgl_cluster(radius=7.0, centre=(7.5, 7.5, 7.5), box=15.0),
}


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("case", list(CASES))
def test_open_axes_energy_forces_match_oracle(case, form):
    c = CASES[case]()
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl(), periodic=c.periodic)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(form), dt_start=fi.CU_DT,
                       periodic=c.periodic) as h:
        e, f = h.energy_forces(c.x, c.box)
    check_forces(form, e, f, eo, fo, c.n)


@pytest.mark.parametrize("case", ["slab", "cluster_edge"])
def test_open_axes_relaxation_parity(case):
    c = CASES[case]()
    prm = oracle.Params(dt_start=fi.CU_DT)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), prm, fi.CU_MASS, 1e-6, 100000,
                             periodic=c.periodic)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot("fp64_table_half"), dt_start=fi.CU_DT,
                       periodic=c.periodic) as h:
        r = h.minimize(x, c.box, 1e-6, 100000)
    assert ro.stop == oracle.STOP_FTOL and r.stop == fg.FIRE_STOP_FTOL
    assert r.fmax_atom < 1e-6
    assert abs(r.energy - ro.energy) / c.n < 1e-8
    assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations)
    assert r.nbr_builds >= 1


def test_atoms_far_outside_open_axis():
    # the whole slab 3 box lengths below z = 0: every atom in the edge cell
    # row, results unchanged apart from the translation
    c = fi.rgl_slab(ncell=6, n_vac=1, sigma=0.08)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl(), periodic=c.periodic)
    x = c.x.copy()
    x[:, 2] -= 3.0 * c.box[2]
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot("fp64_table_half"), dt_start=fi.CU_DT,
                       periodic=c.periodic) as h:
        e, f = h.energy_forces(x, c.box)
    check_forces("fp64_table_half", e, f, eo, fo, c.n)


def test_sw_slab_energy_forces_match_oracle():
    c = fi.sw_si_slab(ncell=6, n_vac=5, sigma=0.1)
    eo, fo = oracle.energy_forces(c.x, c.box, oracle.Potential("sw", **fi.SW_SI),
                                  periodic=c.periodic, mode=oracle.FORCE_CELLS)
    with fg.FireHandle(c.n, fi.SI_MASS, fg.Potential(fg.FIRE_POT_SW, skin=0.3, **fi.SW_SI),
                       dt_start=fi.SI_DT, periodic=c.periodic) as h:
        e, f = h.energy_forces(c.x, c.box)
    assert np.abs(f - fo).max() / np.abs(fo).max() < F_REL
    assert e == pytest.approx(eo, rel=1e-12)


@pytest.mark.parametrize("precision,pair_eval", [
    (fg.FIRE_PREC_FP64, fg.FIRE_PAIR_TABLE), (fg.FIRE_PREC_FP64, fg.FIRE_PAIR_ANALYTIC),
    (fg.FIRE_PREC_FP32_PAIR, fg.FIRE_PAIR_ANALYTIC)])
def test_batch_open_axis_matches_oracle(precision, pair_eval):
    cfgs = [fi.rgl_slab(ncell=n, nz=m, seed=40 + n, n_vac=1, sigma=0.08, vacuum=6.0)
            for n, m in [(3, 3), (4, 6), (6, 4), (5, 5)]]
    x = np.ascontiguousarray(np.concatenate([c.x for c in cfgs]))
    boxes = np.array([c.box for c in cfgs])
    counts = [c.n for c in cfgs]
    pot = fg.Potential(fg.FIRE_POT_RGL, precision=precision, pair_eval=pair_eval,
                       skin=0.3, **fi.RGL_CU)
    with fg.FireBatch(counts, fi.CU_MASS, pot, dt_start=fi.CU_DT, periodic=(1, 1, 0)) as b:
        res, f = b.minimize(x.copy(), boxes, 1e-6, 0, want_forces=True)
    off = np.concatenate([[0], np.cumsum(counts)])
    for s, c in enumerate(cfgs):
        eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl(), periodic=c.periodic)
        check_forces("fp32pair" if precision == fg.FIRE_PREC_FP32_PAIR else "fp64_exp",
                     res[s].energy, f[off[s]:off[s + 1]], eo, fo, c.n)
