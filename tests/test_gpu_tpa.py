"""Several threads per atom in the RGL pair passes (fire_set_threads_per_atom),
GPU vs the FP64 oracle through the C ABI.  Splitting an atom's neighbour list
over 2 to 32 threads only reorders the per-atom sums, so every setting must
meet the one-thread bars: FP64 forces within 1e-10 relative, FP32-pair forces
within a few 1e-6 eV/A, and relaxations to the oracle's energy and iteration
count."""
import numpy as np
import pytest

import fire_inputs as fi
import oracle
import paper_1908_02038_gb300 as fg

pytestmark = pytest.mark.gpu

F_REL = 1e-10
F32_ABS = 3e-6       # eV/A
E32_PER_ATOM = 1e-6  # eV/atom
TPAS = (1, 2, 4, 8, 16, 32)

FORMS = {
    "fp64_half": dict(precision=fg.FIRE_PREC_FP64, pair_eval=fg.FIRE_PAIR_TABLE,
                      newton=fg.FIRE_NEWTON_ON),
    "fp64_full": dict(precision=fg.FIRE_PREC_FP64, pair_eval=fg.FIRE_PAIR_TABLE,
                      newton=fg.FIRE_NEWTON_OFF),
    "fp32pair": dict(precision=fg.FIRE_PREC_FP32_PAIR, pair_eval=fg.FIRE_PAIR_ANALYTIC),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    fg.build()
    fg.load_library()


def rgl_pot(form):
    return fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **FORMS[form], **fi.RGL_CU)


def ora_rgl():
    return oracle.Potential("rgl", **fi.RGL_CU)


@pytest.mark.parametrize("form", list(FORMS))
def test_every_threads_per_atom_matches_oracle(form):
    # 7^3 cells with 5 vacancies and 0.1 A noise: neighbour counts vary from
    # atom to atom, so groups finish their list slices unevenly
    c = fi.rgl_vacancy_box(ncell=7, seed=31, n_vac=5, sigma=0.1)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl())
    got = {}
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(form), dt_start=fi.CU_DT) as h:
        for t in TPAS:
            assert h.set_threads_per_atom(t) == t
            got[t] = h.energy_forces(c.x, c.box)
    for t, (e, f) in got.items():
        if form == "fp32pair":
            assert np.abs(f - fo).max() < F32_ABS, t
            assert abs(e - eo) / c.n < E32_PER_ATOM, t
        else:
            assert np.abs(f - fo).max() / np.abs(fo).max() < F_REL, t
            assert e == pytest.approx(eo, rel=1e-12), t
    # the settings differ only in the order of the per-atom sums; in the
    # FP32-pair form that order also moves the FP32 rounding of rho_i before
    # its square root, by up to an ulp of sqrt(rho) (~3e-7 eV) per atom
    e1, f1 = got[1]
    for t in TPAS[1:]:
        e, f = got[t]
        if form == "fp32pair":
            assert np.abs(f - f1).max() < 1e-6, t
            assert abs(e - e1) / c.n < 1e-7, t
        else:
            assert np.abs(f - f1).max() < 1e-12 * np.abs(f1).max(), t
            assert e == pytest.approx(e1, rel=1e-13), t


@pytest.mark.parametrize("form,tpa", [("fp64_half", 2), ("fp64_full", 4), ("fp32pair", 8)])
def test_relaxation_with_threads_per_atom_matches_oracle(form, tpa):
    c = fi.rgl_vacancy_box(ncell=5, seed=32, n_vac=2, sigma=0.05)
    prm = oracle.Params(dt_start=fi.CU_DT)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), prm, fi.CU_MASS, 1e-6, 100000)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(form), dt_start=fi.CU_DT) as h:
        assert h.set_threads_per_atom(tpa) == tpa
        r = h.minimize(x, c.box, 1e-6, 100000)
    assert ro.stop == oracle.STOP_FTOL and r.stop == fg.FIRE_STOP_FTOL
    assert r.fmax_atom < 1e-6
    assert abs(r.energy - ro.energy) / c.n < 1e-8
    assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations)


def test_full_list_runs_are_identical_for_a_fixed_threads_per_atom():
    # no atomics on the full list: the same setting gives the same run bit for bit
    c = fi.rgl_vacancy_box(ncell=6, seed=33, n_vac=3, sigma=0.08)
    runs = []
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot("fp64_full"), dt_start=fi.CU_DT) as h:
        h.set_threads_per_atom(4)
        for _ in range(2):
            x = c.x.copy()
            runs.append((h.minimize(x, c.box, 1e-6, 100000), x))
    (r1, x1), (r2, x2) = runs
    assert r1.iterations == r2.iterations and r1.energy == r2.energy
    assert np.array_equal(x1, x2)


def test_threads_per_atom_choice_and_errors():
    c = fi.rgl_vacancy_box(ncell=4, seed=34, n_vac=1)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot("fp64_half"), dt_start=fi.CU_DT) as h:
        # a few hundred atoms: the automatic choice is the largest for RGL
        assert h.set_threads_per_atom(0) == 8
        for bad in (-1, 3, 12, 64):
            with pytest.raises(fg.FireError):
                h.set_threads_per_atom(bad)
        assert h.set_threads_per_atom(2) == 2
    # forms that do not split the list report one thread per atom
    sw = fg.Potential(fg.FIRE_POT_SW, skin=0.3, **fi.SW_SI)
    cs = fi.sw_si_vacancy_box(ncell=4, seed=7, n_vac=1, sigma=0.05)
    with fg.FireHandle(cs.n, fi.SI_MASS, sw, dt_start=fi.SI_DT) as h:
        assert h.set_threads_per_atom(4) == 1
    cfgs = [fi.rgl_vacancy_box(ncell=3, seed=35 + k, n_vac=1) for k in range(2)]
    with fg.FireBatch([q.n for q in cfgs], fi.CU_MASS, rgl_pot("fp32pair"),
                      dt_start=fi.CU_DT) as b:
        with pytest.raises(fg.FireError):
            fg.fire_set_threads_per_atom(b.h, 2)


@pytest.mark.parametrize("check", [fg.FIRE_FP64_CHECK_CONFIRM, fg.FIRE_FP64_CHECK_FINISH])
def test_fp32pair_split_lists_graph_and_chunked_runs_are_identical(check):
    # full lists, fixed per-atom sum order: the graph loop and the chunked
    # loop follow the same trajectory bit for bit at 4 threads per atom,
    # through the FP64 confirmations (full-list FP64 passes, also split)
    c = fi.rgl_vacancy_box(ncell=8, seed=36, n_vac=4, sigma=0.1)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot("fp32pair"), dt_start=fi.CU_DT,
                       confirm64=check) as h:
        assert h.set_threads_per_atom(4) == 4
        x1 = c.x.copy()
        r1 = h.minimize(x1, c.box, 1e-6, 100000)
        h.set_exec_mode(fg.FIRE_EXEC_CHUNKED, 16)
        x2 = c.x.copy()
        r2 = h.minimize(x2, c.box, 1e-6, 100000)
    assert r1.stop == r2.stop == fg.FIRE_STOP_FTOL
    assert (r1.iterations, r1.nbr_builds, r1.force_evals) == (r2.iterations, r2.nbr_builds,
                                                               r2.force_evals)
    if check == fg.FIRE_FP64_CHECK_CONFIRM:   # the stop was confirmed in FP64
        assert r1.force_evals > r1.iterations + 1
    assert r1.energy == r2.energy and np.array_equal(x1, x2)


@pytest.mark.parametrize("form", ["fp64_half", "fp32pair"])
def test_frozen_components_with_split_lists(form):
    c = fi.rgl_vacancy_box(ncell=6, seed=37, n_vac=3, sigma=0.05)
    fz = np.zeros(c.n, np.uint8)
    fz[c.x[:, 0] < 4.0] = 3               # frozen in x and y
    fz[c.x[:, 0] > c.box[0] - 3.0] = 4    # frozen in z
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS,
                             1e-6, 100000, frozen=fz)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(form), dt_start=fi.CU_DT) as h:
        assert h.set_threads_per_atom(2) == 2
        h.set_dof_mask(fz)
        r = h.minimize(x, c.box, 1e-6, 100000)
    for d in range(3):
        sel = (fz >> d) & 1 == 1
        assert np.array_equal(x[sel, d], c.x[sel, d]), d
    assert r.stop == fg.FIRE_STOP_FTOL and ro.stop == oracle.STOP_FTOL
    if form == "fp32pair":
        assert abs(r.energy - ro.energy) / c.n < E32_PER_ATOM
    else:
        assert abs(r.energy - ro.energy) / c.n < 1e-8
        assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations)


def test_lj_every_threads_per_atom_matches_oracle():
    """The LJ force pass splits an atom's list the same way (small boxes
    spread their FP64 pair work over more SMs)."""
    c = fi.lj_fcc_vacancy(seed=2)
    opot = oracle.Potential("lj", eps=1.0, sigma=1.0, rc_lj=2.5)
    eo, fo = oracle.energy_forces(c.x, c.box, opot)
    pot = fg.Potential(fg.FIRE_POT_LJ, eps=1.0, sigma=1.0, rc_lj=2.5, skin=0.3)
    with fg.FireHandle(c.n, fi.LJ_MASS, pot, dt_start=fi.LJ_DT) as h:
        assert h.set_threads_per_atom(0) == 32   # 255 atoms: the automatic choice
        for t in TPAS:
            assert h.set_threads_per_atom(t) == t
            e, f = h.energy_forces(c.x, c.box)
            assert np.abs(f - fo).max() / np.abs(fo).max() < F_REL, t
            assert e == pytest.approx(eo, rel=1e-12), t
