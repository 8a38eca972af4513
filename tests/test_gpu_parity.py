"""GPU path vs the FP64 CPU oracle, through the C ABI.

Bars (FP64 path): forces within 1e-10 relative (max-abs difference over the
max-abs oracle force, at the displaced starting configurations where forces
are O(0.1-1)), energies within 1e-12 relative for single evaluations, and for
relaxations the final energy within 1e-8 eV/atom and the iteration count
within 5 % of the oracle's, both runs converged.
"""
import ctypes

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


def lj_pot(**kw):
    return fg.Potential(fg.FIRE_POT_LJ, eps=1.0, sigma=1.0, rc_lj=2.5, skin=kw.pop("skin", 0.3))


def rgl_pot(skin=0.3, precision=fg.FIRE_PREC_FP64):
    return fg.Potential(fg.FIRE_POT_RGL, precision=precision, skin=skin, **fi.RGL_CU)


def ora_lj():
    return oracle.Potential("lj", eps=1.0, sigma=1.0, rc_lj=2.5)


def ora_rgl():
    return oracle.Potential("rgl", **fi.RGL_CU)


def force_rel_err(fg_, fo):
    return np.abs(fg_ - fo).max() / np.abs(fo).max()


# ----------------------------------------------------------------------------
# single evaluations


@pytest.mark.parametrize("seed", [1, 2])
def test_lj_energy_forces_match_oracle(seed):
    c = fi.lj_fcc_vacancy(seed=seed)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_lj())
    with fg.FireHandle(c.n, fi.LJ_MASS, lj_pot(), dt_start=fi.LJ_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
    assert force_rel_err(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)


@pytest.mark.parametrize("ncell,nvac", [(3, 2), (4, 1), (5, 3), (7, 10)])
def test_rgl_energy_forces_match_oracle(ncell, nvac):
    # 3^3 and 4^3 boxes take the all-pairs list build, 5^3 and 7^3 the cell build
    c = fi.rgl_vacancy_box(ncell=ncell, seed=20 + ncell, n_vac=nvac, sigma=0.08)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl())
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
    assert force_rel_err(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)


def test_rgl_32k_energy_forces_match_oracle():
    c = fi.rgl_vacancy_box(ncell=20, seed=2)
    assert c.n == 31680
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl(), mode=oracle.FORCE_CELLS)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
    assert force_rel_err(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)


def test_rgl_1m_sampled_forces_match_oracle():
    c = fi.rgl_void_box()
    assert c.n == 997450
    rng = np.random.default_rng(5)
    which = np.sort(rng.choice(c.n, size=2048, replace=False))
    eo, fo = oracle.energy_forces_subset(c.x, c.box, ora_rgl(), which, mode=oracle.FORCE_CELLS)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
    assert force_rel_err(f[which], fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)
    # properties that hold at any size
    assert np.abs(f.sum(0)).max() < 1e-9 * np.abs(f).max() * np.sqrt(c.n)


def test_perfect_lattice_zero_force_and_cohesive_energy():
    c = fi.perfect_fcc(8, fi.CU_A)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
        res = h.minimize(c.x.copy(), c.box, 1e-6, 100)
    assert np.abs(f).max() < 1e-12
    assert e / c.n == pytest.approx(-3.508821531217027, rel=1e-13)
    assert res.iterations == 0 and res.stop == fg.FIRE_STOP_FTOL


def test_dev_pointer_variants_match_host():
    torch = pytest.importorskip("torch")
    c = fi.rgl_vacancy_box(ncell=5, seed=9, n_vac=2)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
        d_pos = torch.tensor(c.x, dtype=torch.float64, device="cuda")
        d_f = torch.empty_like(d_pos)
        d_e = torch.zeros(1, dtype=torch.float64, device="cuda")
        fg.fire_energy_forces_dev(h.h, d_pos, c.box, d_f, d_e)
        torch.cuda.synchronize()
        assert np.array_equal(d_f.cpu().numpy(), f) or force_rel_err(d_f.cpu().numpy(), f) < 1e-14
        assert d_e.item() == pytest.approx(e, rel=1e-14)
        x = c.x.copy()
        r1 = h.minimize(x, c.box, 1e-6, 5000)
        r2 = h.minimize_dev(d_pos, c.box, 1e-6, 5000)
        assert r2.stop == fg.FIRE_STOP_FTOL
        assert abs(r1.iterations - r2.iterations) <= max(2, 0.05 * r1.iterations)
        assert r2.energy == pytest.approx(r1.energy, abs=1e-8 * c.n)


# ----------------------------------------------------------------------------
# relaxations


def relax_pair(c, pot, opot, mass, dt, ftol, maxiter, mode=oracle.FORCE_BRUTE, periodic=(1, 1, 1)):
    xo, ro, _ = oracle.fire2(c.x, c.box, opot, oracle.Params(dt_start=dt), mass, ftol, maxiter,
                             periodic=periodic, mode=mode)
    x = c.x.copy()
    with fg.FireHandle(c.n, mass, pot, dt_start=dt, periodic=periodic) as h:
        r = h.minimize(x, c.box, ftol, maxiter)
    return x, r, xo, ro


def assert_relax_parity(c, r, ro, ftol):
    assert ro.stop == oracle.STOP_FTOL, "oracle did not converge"
    assert r.stop == fg.FIRE_STOP_FTOL
    assert r.fmax_atom < ftol
    assert r.force_evals == r.iterations + 1
    assert abs(r.energy - ro.energy) / c.n < 1e-8
    assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations), \
        (r.iterations, ro.iterations)


def test_lj_relaxation_parity():
    c = fi.lj_fcc_vacancy(seed=1)
    x, r, xo, ro = relax_pair(c, lj_pot(), ora_lj(), fi.LJ_MASS, fi.LJ_DT, 1e-8, 200000)
    assert_relax_parity(c, r, ro, 1e-8)


@pytest.mark.parametrize("ncell,nvac", [(3, 1), (5, 2)])
def test_rgl_small_relaxation_parity(ncell, nvac):
    c = fi.rgl_vacancy_box(ncell=ncell, seed=30 + ncell, n_vac=nvac)
    x, r, xo, ro = relax_pair(c, rgl_pot(), ora_rgl(), fi.CU_MASS, fi.CU_DT, 1e-6, 100000)
    assert_relax_parity(c, r, ro, 1e-6)


def test_rgl_32k_relaxation_parity():
    c = fi.rgl_vacancy_box(ncell=20, seed=2)
    x, r, xo, ro = relax_pair(c, rgl_pot(), ora_rgl(), fi.CU_MASS, fi.CU_DT, 1e-6, 100000,
                              mode=oracle.FORCE_CELLS)
    assert_relax_parity(c, r, ro, 1e-6)
    assert r.nbr_builds >= 1


def test_lj_dimer_open_boundaries():
    c = fi.Config("dimer", np.array([[5.0, 5.0, 5.0], [6.3, 5.1, 4.9]]), np.array([20.0] * 3),
                  periodic=(0, 0, 0))
    x, r, xo, ro = relax_pair(c, lj_pot(), ora_lj(), 1.0, fi.LJ_DT, 1e-10, 100000,
                              periodic=(0, 0, 0))
    assert r.stop == fg.FIRE_STOP_FTOL
    assert abs(np.linalg.norm(x[1] - x[0]) - 2 ** (1 / 6)) < 1e-10
    assert abs(r.iterations - ro.iterations) <= 2


# ----------------------------------------------------------------------------
# edge cases and error paths


def test_single_atom_is_converged_at_start():
    x = np.array([[1.0, 2.0, 3.0]])
    with fg.FireHandle(1, 1.0, lj_pot(), dt_start=fi.LJ_DT) as h:
        e, f = h.energy_forces(x, [10.0] * 3)
        r = h.minimize(x, [10.0] * 3, 1e-8, 10)
    assert e == 0.0 and np.all(f == 0.0)
    assert r.iterations == 0 and r.stop == fg.FIRE_STOP_FTOL


def test_maxiter_zero_and_vdfmax_zero():
    c = fi.lj_fcc_vacancy(seed=1)
    with fg.FireHandle(c.n, fi.LJ_MASS, lj_pot(), dt_start=fi.LJ_DT) as h:
        x = c.x.copy()
        r = h.minimize(x, c.box, 1e-8, 0)
        assert r.stop == fg.FIRE_STOP_MAXITER and r.iterations == 0
        assert np.array_equal(x, c.x)
    # vdfmax = 0: the first pass has P = 0 and stops with MAXVDOTF, as in the oracle
    with fg.FireHandle(c.n, fi.LJ_MASS, lj_pot(), dt_start=fi.LJ_DT, vdfmax=0) as h:
        r = h.minimize(c.x.copy(), c.box, 1e-8, 100)
    _, ro, _ = oracle.fire2(c.x, c.box, ora_lj(), oracle.Params(dt_start=fi.LJ_DT, vdfmax=0),
                            1.0, 1e-8, 100)
    assert r.stop == fg.FIRE_STOP_MAXVDOTF == ro.stop
    assert r.iterations == ro.iterations == 0


def test_maxiter_stop_matches_oracle_state():
    c = fi.rgl_vacancy_box(ncell=4, seed=3, n_vac=2)
    x, r, xo, ro = relax_pair(c, rgl_pot(), ora_rgl(), fi.CU_MASS, fi.CU_DT, 1e-12, 60)
    assert r.stop == fg.FIRE_STOP_MAXITER == ro.stop
    assert r.iterations == 60
    assert r.dt_final == pytest.approx(ro.dt_final, rel=1e-12)
    assert r.alpha_final == pytest.approx(ro.alpha_final, rel=1e-12)
    assert np.abs(x - xo).max() < 1e-9


@pytest.mark.parametrize("body", [1, 3, 8])
def test_maxiter_stop_with_every_loop_body(body):
    # 61 iterations: not a multiple of the bodies' lengths, so the last body
    # launch runs iterations past the stop, which must leave the state alone
    c = fi.rgl_vacancy_box(ncell=4, seed=3, n_vac=2)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS,
                             1e-12, 61)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        h.set_exec_mode(fg.FIRE_EXEC_GRAPH_WHILE, body)
        r = h.minimize(x, c.box, 1e-12, 61)
    assert r.stop == fg.FIRE_STOP_MAXITER == ro.stop
    assert r.iterations == 61 and r.force_evals == 62
    assert r.dt_final == pytest.approx(ro.dt_final, rel=1e-12)
    assert r.alpha_final == pytest.approx(ro.alpha_final, rel=1e-12)
    assert np.abs(x - xo).max() < 1e-9


def test_nonfinite_positions_rejected_and_untouched():
    c = fi.lj_fcc_vacancy(seed=1)
    x = c.x.copy()
    x[17, 1] = np.nan
    with fg.FireHandle(c.n, fi.LJ_MASS, lj_pot(), dt_start=fi.LJ_DT) as h:
        with pytest.raises(fg.FireError) as e:
            h.minimize(x, c.box, 1e-8, 100)
        assert e.value.status == fg.FIRE_ERR_NONFINITE
        assert np.isnan(x[17, 1]) and np.array_equal(np.delete(x, 17, 0), np.delete(c.x, 17, 0))
        with pytest.raises(fg.FireError) as e:
            h.energy_forces(x, c.box)
        assert e.value.status == fg.FIRE_ERR_NONFINITE
        # the handle stays usable
        r = h.minimize(c.x.copy(), c.box, 1e-8, 200000)
        assert r.stop == fg.FIRE_STOP_FTOL


def test_box_too_small_rejected():
    with fg.FireHandle(4, 1.0, lj_pot(), dt_start=fi.LJ_DT) as h:
        with pytest.raises(fg.FireError) as e:
            h.minimize(np.zeros((4, 3)), [4.0, 10.0, 10.0], 1e-6, 10)
        assert e.value.status == fg.FIRE_ERR_ARG
        with pytest.raises(fg.FireError) as e:
            h.minimize(np.zeros((4, 3)), [10.0, 10.0, 10.0], -1.0, 10)
        assert e.value.status == fg.FIRE_ERR_ARG


def test_time_budget_stops_the_device_loop():
    c = fi.rgl_vacancy_box(ncell=5, seed=9, n_vac=2)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        h.set_time_budget(1e-9)
        x = c.x.copy()
        with pytest.raises(fg.FireError) as e:
            h.minimize(x, c.box, 1e-6, 100000)
        assert e.value.status == fg.FIRE_ERR_TIMEOUT
        assert np.array_equal(x, c.x)
        h.set_time_budget(0)
        r = h.minimize(x, c.box, 1e-6, 100000)
        assert r.stop == fg.FIRE_STOP_FTOL


def test_neighbour_overflow_retry_on_dense_cluster():
    # a dense FCC cluster in a large open box: the mean density underestimates
    # the local one, the first list overflows and the call retries with more room
    c = fi.perfect_fcc(4, fi.LJ_A)
    x = c.x + np.random.default_rng(3).uniform(-0.05, 0.05, c.x.shape) + 20.0
    box = [60.0, 60.0, 60.0]
    eo, fo = oracle.energy_forces(x, box, ora_lj(), periodic=(0, 0, 0))
    with fg.FireHandle(c.n, 1.0, lj_pot(), dt_start=fi.LJ_DT, periodic=(0, 0, 0)) as h:
        e, f = h.energy_forces(x, box)
    assert force_rel_err(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)


def test_graph_reuse_and_box_change():
    c = fi.rgl_vacancy_box(ncell=5, seed=11, n_vac=1)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        r1 = h.minimize(c.x.copy(), c.box, 1e-6, 100000)
        r2 = h.minimize(c.x.copy(), c.box, 1e-6, 100000)
        assert abs(r1.iterations - r2.iterations) <= max(2, 0.05 * r1.iterations)
        box2 = c.box * 1.01
        x3 = c.x * 1.01
        e3, f3 = h.energy_forces(x3, box2)
    eo, fo = oracle.energy_forces(x3, box2, ora_rgl())
    assert force_rel_err(f3, fo) < F_REL


def test_table_exponential_against_libm():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-30.0, 12.0, 200000), np.linspace(-1, 1, 20001),
                        [0.0, -0.0, 1e-300, -1e-17, np.log(2.0), -np.log(2.0), 11.0, -25.0]])
    d_x = torch.tensor(x, dtype=torch.float64, device="cuda")
    d_y = torch.empty_like(d_x)
    fg.fire_diag_exp(d_x, d_y)
    torch.cuda.synchronize()
    y = d_y.cpu().numpy()
    rel = np.abs(y - np.exp(x)) / np.exp(x)
    assert rel.max() < 4.5e-16, rel.max()       # within 2 ulp of the libm value
    assert np.all(y[x == 0.0] == 1.0)


def test_chunked_execution_matches_graph_loop():
    c = fi.rgl_vacancy_box(ncell=5, seed=12, n_vac=2)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        x1 = c.x.copy()
        r1 = h.minimize(x1, c.box, 1e-6, 100000)
        h.set_exec_mode(fg.FIRE_EXEC_CHUNKED, 7)
        x2 = c.x.copy()
        r2 = h.minimize(x2, c.box, 1e-6, 100000)
        r3 = h.minimize(c.x.copy(), c.box, 1e-6, 50)
    assert r2.stop == r1.stop == fg.FIRE_STOP_FTOL
    assert abs(r1.iterations - r2.iterations) <= max(2, 0.05 * r1.iterations)
    assert abs(r1.energy - r2.energy) / c.n < 1e-10
    assert r3.stop == fg.FIRE_STOP_MAXITER and r3.iterations == 50 and r3.force_evals == 51


@pytest.mark.parametrize("check", [fg.FIRE_FP64_CHECK_CONFIRM, fg.FIRE_FP64_CHECK_FINISH])
def test_fp32pair_graph_and_chunked_runs_are_identical(check):
    # The FP32-pair passes write whole forces and sum in a fixed order, so the
    # graph loop with one iteration per body and with several (8, 3 and the
    # largest setting, 64: each iteration's build chain and confirming passes
    # under IF nodes of their own, set by the update kernel's last block;
    # iterations past the stop returning at once) and the chunked loop (build
    # and confirming passes gated in their kernels) must follow the same
    # trajectory bit for bit.
    c = fi.rgl_vacancy_box(ncell=12, seed=14, n_vac=4, sigma=0.1)
    pot = rgl_pot(precision=fg.FIRE_PREC_FP32_PAIR)
    runs = []
    with fg.FireHandle(c.n, fi.CU_MASS, pot, dt_start=fi.CU_DT, confirm64=check) as h:
        for mode, chunk in ((fg.FIRE_EXEC_GRAPH_WHILE, 1), (fg.FIRE_EXEC_GRAPH_WHILE, 8),
                            (fg.FIRE_EXEC_GRAPH_WHILE, 3), (fg.FIRE_EXEC_GRAPH_WHILE, 64),
                            (fg.FIRE_EXEC_CHUNKED, 16)):
            h.set_exec_mode(mode, chunk)
            x = c.x.copy()
            runs.append((x, h.minimize(x, c.box, 1e-6, 100000)))
    x1, r1 = runs[0]
    assert r1.stop == fg.FIRE_STOP_FTOL
    assert r1.nbr_builds > 2
    for x2, r2 in runs[1:]:
        assert r2.stop == fg.FIRE_STOP_FTOL
        assert (r1.iterations, r1.nbr_builds, r1.force_evals) == (r2.iterations, r2.nbr_builds,
                                                                   r2.force_evals)
        assert r1.energy == r2.energy
        assert np.array_equal(x1, x2)


def test_loop_body_setting_rejects_bad_values():
    c = fi.rgl_vacancy_box(ncell=5, seed=12, n_vac=2)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        for mode, chunk in ((fg.FIRE_EXEC_GRAPH_WHILE, -1), (fg.FIRE_EXEC_GRAPH_WHILE, 65),
                            (fg.FIRE_EXEC_CHUNKED, 0), (fg.FIRE_EXEC_CHUNKED, 4097), (2, 1)):
            with pytest.raises(fg.FireError) as e:
                h.set_exec_mode(mode, chunk)
            assert e.value.status == fg.FIRE_ERR_ARG


# ----------------------------------------------------------------------------
# FP32-pair form (pair/embedding math FP32; positions, sums, control FP64)

F32_ABS = 3e-6      # eV/A, max-abs force difference against the FP64 oracle
E32_PER_ATOM = 1e-6  # eV/atom
F32_MARGIN = 6e-7    # eV/A, FP32-pair force error bound at relaxed structures


@pytest.mark.parametrize("ncell,nvac", [(3, 2), (5, 3), (7, 10)])
def test_fp32pair_energy_forces_vs_oracle(ncell, nvac):
    c = fi.rgl_vacancy_box(ncell=ncell, seed=20 + ncell, n_vac=nvac, sigma=0.08)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl())
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(precision=fg.FIRE_PREC_FP32_PAIR),
                       dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
    err = np.abs(f - fo).max()
    print(f"FP32-pair vs FP64 oracle: max|dF| = {err:.3e} eV/A, dE/N = {abs(e - eo) / c.n:.3e} eV")
    assert err < F32_ABS
    assert abs(e - eo) / c.n < E32_PER_ATOM


def test_fp32pair_1m_sampled_forces_vs_oracle():
    c = fi.rgl_void_box()
    which = np.sort(np.random.default_rng(6).choice(c.n, size=2048, replace=False))
    eo, fo = oracle.energy_forces_subset(c.x, c.box, ora_rgl(), which, mode=oracle.FORCE_CELLS)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(precision=fg.FIRE_PREC_FP32_PAIR),
                       dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
    assert np.abs(f[which] - fo).max() < F32_ABS
    assert abs(e - eo) / c.n < E32_PER_ATOM


def test_fp32pair_relaxation_reaches_fp64_converged_state():
    # FIRE_FP64_CHECK_CONFIRM: a stop on the FP32-pair forces is confirmed by
    # one FP64 evaluation at the same positions, so the result meets ftol in FP64
    c = fi.rgl_vacancy_box(ncell=20, seed=2)
    x64, x32 = c.x.copy(), c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h64, \
            fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(precision=fg.FIRE_PREC_FP32_PAIR),
                          dt_start=fi.CU_DT, confirm64=fg.FIRE_FP64_CHECK_CONFIRM) as h32:
        r64 = h64.minimize(x64, c.box, 1e-6, 100000)
        r32 = h32.minimize(x32, c.box, 1e-6, 100000)
        # the FP32 solution judged by FP64 forces
        e_chk, f_chk = h64.energy_forces(x32, c.box)
        _, f32_at32 = h32.energy_forces(x32, c.box)
    fmax64_at32 = np.sqrt((f_chk ** 2).sum(1)).max()
    confirmations = r32.force_evals - r32.iterations - 1
    print(f"iterations FP64 {r64.iterations}, FP32-pair {r32.iterations} "
          f"({confirmations} FP64 confirmations); FP64 max|F| at the FP32-pair minimum "
          f"{fmax64_at32:.3e}; dE/N {abs(e_chk - r64.energy) / c.n:.3e}")
    assert r32.stop == fg.FIRE_STOP_FTOL and confirmations >= 1
    # the reported norm and energy are those of the confirming FP64 evaluation
    assert abs(r32.fmax_atom - fmax64_at32) < 1e-12 and r32.fmax_atom < 1e-6
    assert r32.energy == pytest.approx(e_chk, rel=1e-13)
    assert fmax64_at32 < 1e-6
    assert abs(e_chk - r64.energy) / c.n < 1e-8
    # FP32-pair force error at the relaxed structure
    assert np.sqrt(((f32_at32 - f_chk) ** 2).sum(1)).max() < F32_MARGIN


def test_fp32pair_finishing_in_fp64_converges_in_fp64():
    # FIRE_FP64_CHECK_FINISH: FP32-pair forces while the norm is >= 3 ftol,
    # FP64 forces from there on; the stop is on FP64 forces
    c = fi.rgl_vacancy_box(ncell=20, seed=2)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h64, \
            fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(precision=fg.FIRE_PREC_FP32_PAIR),
                          dt_start=fi.CU_DT, confirm64=fg.FIRE_FP64_CHECK_FINISH) as h32:
        r64 = h64.minimize(c.x.copy(), c.box, 1e-6, 100000)
        r = h32.minimize(x, c.box, 1e-6, 100000)
        e_chk, f_chk = h64.energy_forces(x, c.box)
    fmax64 = np.sqrt((f_chk ** 2).sum(1)).max()
    print(f"FP64 {r64.iterations} iterations; FP32-pair then FP64 {r.iterations}")
    assert r.stop == fg.FIRE_STOP_FTOL and r.force_evals == r.iterations + 1
    assert fmax64 < 1e-6 and abs(r.fmax_atom - fmax64) < 1e-12
    assert r.energy == pytest.approx(e_chk, rel=1e-13)
    assert abs(e_chk - r64.energy) / c.n < 1e-8


def test_fp32pair_without_confirmation_stops_on_fp32_forces():
    # confirm64 = 0: stop on the FP32-pair forces alone; at ftol less their
    # error bound the structure still meets ftol in FP64
    c = fi.rgl_vacancy_box(ncell=8, seed=15, n_vac=3)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h64, \
            fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(precision=fg.FIRE_PREC_FP32_PAIR),
                          dt_start=fi.CU_DT, confirm64=0) as h32:
        r = h32.minimize(x, c.box, 1e-6 - F32_MARGIN, 100000)
        _, f_chk = h64.energy_forces(x, c.box)
    assert r.stop == fg.FIRE_STOP_FTOL and r.force_evals == r.iterations + 1
    assert r.fmax_atom < 1e-6 - F32_MARGIN
    assert np.sqrt((f_chk ** 2).sum(1)).max() < 1e-6


# ----------------------------------------------------------------------------
# integrators (Algorithms 3-6) and the original FIRE (Algorithm 1)

INTEGRATORS = [fg.FIRE_INT_EULER_IMPLICIT, fg.FIRE_INT_EULER_EXPLICIT, fg.FIRE_INT_VERLET,
               fg.FIRE_INT_LEAPFROG]


@pytest.mark.parametrize("integ", INTEGRATORS)
@pytest.mark.parametrize("variant", [fg.FIRE_VARIANT_FIRE2, fg.FIRE_VARIANT_FIRE1])
def test_integrator_variant_state_after_40_iterations(integ, variant):
    c = fi.rgl_vacancy_box(ncell=4, seed=81, n_vac=2)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(),
                             oracle.Params(dt_start=fi.CU_DT, integrator=integ, variant=variant),
                             fi.CU_MASS, 1e-12, 40)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT, integrator=integ,
                       variant=variant) as h:
        r = h.minimize(x, c.box, 1e-12, 40)
    assert r.stop == ro.stop == fg.FIRE_STOP_MAXITER
    assert r.dt_final == pytest.approx(ro.dt_final, rel=1e-12)
    assert r.alpha_final == pytest.approx(ro.alpha_final, rel=1e-12)
    assert np.abs(x - xo).max() < 1e-9
    assert r.energy == pytest.approx(ro.energy, rel=1e-12)


@pytest.mark.parametrize("integ", INTEGRATORS)
@pytest.mark.parametrize("variant", [fg.FIRE_VARIANT_FIRE2, fg.FIRE_VARIANT_FIRE1])
def test_integrator_variant_relaxation_parity(integ, variant):
    c = fi.lj_fcc_vacancy(seed=1)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_lj(),
                             oracle.Params(dt_start=fi.LJ_DT, integrator=integ, variant=variant),
                             fi.LJ_MASS, 1e-6, 200000)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.LJ_MASS, lj_pot(), dt_start=fi.LJ_DT, integrator=integ,
                       variant=variant) as h:
        r = h.minimize(x, c.box, 1e-6, 200000)
    assert_relax_parity(c, r, ro, 1e-6)


def test_fire2_and_fire1_reach_the_same_minimum():
    # Table 2's comparison (FIRE 2.0 vs FIRE) on the 32k vacancy box: both
    # converge to the same structure; the force-evaluation counts are
    # reported (on this short-range problem they are close, see the design notes)
    c = fi.rgl_vacancy_box(ncell=20, seed=2)
    res = {}
    for variant in (fg.FIRE_VARIANT_FIRE2, fg.FIRE_VARIANT_FIRE1):
        for integ in (fg.FIRE_INT_EULER_IMPLICIT, fg.FIRE_INT_EULER_EXPLICIT):
            with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT, variant=variant,
                               integrator=integ) as h:
                r = h.minimize(c.x.copy(), c.box, 1e-6, 100000)
            assert r.stop == fg.FIRE_STOP_FTOL
            res[(variant, integ)] = r
    print("force evaluations to 1e-6 eV/A:",
          {f"{'FIRE2' if v == 0 else 'FIRE'}/{'EI' if i == 0 else 'EE'}": r.force_evals
           for (v, i), r in res.items()})
    e = [r.energy / c.n for r in res.values()]
    assert max(e) - min(e) < 1e-8


@pytest.mark.parametrize("precision", [fg.FIRE_PREC_FP64, fg.FIRE_PREC_FP32_PAIR])
def test_analytic_and_tabulated_pair_functions_agree(precision):
    c = fi.rgl_vacancy_box(ncell=7, seed=91, n_vac=6, sigma=0.1)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl())
    out = {}
    for mode in (fg.FIRE_PAIR_TABLE, fg.FIRE_PAIR_ANALYTIC):
        pot = rgl_pot(precision=precision)
        pot.pair_eval = mode
        with fg.FireHandle(c.n, fi.CU_MASS, pot, dt_start=fi.CU_DT) as h:
            out[mode] = h.energy_forces(c.x, c.box)
    for mode, (e, f) in out.items():
        if precision == fg.FIRE_PREC_FP64:
            assert force_rel_err(f, fo) < F_REL, mode
            assert e == pytest.approx(eo, rel=E_REL), mode
        else:
            assert np.abs(f - fo).max() < F32_ABS, mode
            assert abs(e - eo) / c.n < E32_PER_ATOM, mode


def test_compressed_pairs_fall_back_to_analytic_terms():
    # a dimer at 0.45 r0 lies below the table; forces must still match the oracle
    x = np.array([[5.0, 5.0, 5.0], [5.0 + 0.45 * fi.RGL_CU["r0"], 5.0, 5.0],
                  [8.0, 7.5, 5.5]])
    box = [20.0, 20.0, 20.0]
    eo, fo = oracle.energy_forces(x, box, ora_rgl())
    with fg.FireHandle(3, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(x, box)
    assert force_rel_err(f, fo) < F_REL
    assert e == pytest.approx(eo, rel=E_REL)


# ----------------------------------------------------------------------------
# maximum displacement per step (dmax) and frozen degrees of freedom

@pytest.mark.parametrize("integ", [fg.FIRE_INT_EULER_IMPLICIT, fg.FIRE_INT_VERLET])
def test_dmax_state_after_60_iterations_matches_oracle(integ):
    c = fi.rgl_vacancy_box(ncell=4, seed=91, n_vac=2, sigma=0.1)
    prm = dict(dt_start=fi.CU_DT, integrator=integ, dmax=0.003)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(**prm), fi.CU_MASS, 1e-12, 60)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), **prm) as h:
        r = h.minimize(x, c.box, 1e-12, 60)
    assert r.stop == ro.stop == fg.FIRE_STOP_MAXITER
    assert r.dt_final == pytest.approx(ro.dt_final, rel=1e-12)
    assert np.abs(x - xo).max() < 1e-9
    assert r.energy == pytest.approx(ro.energy, rel=1e-12)


@pytest.mark.parametrize("mode,chunk", [(fg.FIRE_EXEC_GRAPH_WHILE, 0), (fg.FIRE_EXEC_GRAPH_WHILE, 1),
                                        (fg.FIRE_EXEC_CHUNKED, 16)])
def test_dmax_relaxation_parity(mode, chunk):
    c = fi.rgl_vacancy_box(ncell=5, seed=92, n_vac=2, sigma=0.1)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT, dmax=0.002),
                             fi.CU_MASS, 1e-6, 100000)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT, dmax=0.002) as h:
        h.set_exec_mode(mode, chunk)
        r = h.minimize(x, c.box, 1e-6, 100000)
    assert_relax_parity(c, r, ro, 1e-6)


def frozen_slab(c):
    fz = np.zeros(c.n, np.uint8)
    fz[c.x[:, 0] < 4.0] = 3          # frozen in x and y
    fz[c.x[:, 0] > c.box[0] - 3.0] = 4   # frozen in z
    return fz


@pytest.mark.parametrize("precision", [fg.FIRE_PREC_FP64, fg.FIRE_PREC_FP32_PAIR])
def test_frozen_dofs_relaxation_parity(precision):
    c = fi.rgl_vacancy_box(ncell=6, seed=93, n_vac=3, sigma=0.05)
    fz = frozen_slab(c)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS,
                             1e-6, 100000, frozen=fz)
    x = c.x.copy()
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(precision=precision), dt_start=fi.CU_DT) as h:
        h.set_dof_mask(fz)
        r = h.minimize(x, c.box, 1e-6, 100000)
        # forces from an evaluation are the full forces, mask or not
        e_m, f_m = h.energy_forces(x, c.box)
        h.set_dof_mask(None)
        e_u, f_u = h.energy_forces(x, c.box)
    for d in range(3):
        sel = (fz >> d) & 1 == 1
        assert np.array_equal(x[sel, d], c.x[sel, d]), d
    # (equal up to the order of the FP64 atomic sums)
    assert np.abs(f_m - f_u).max() <= 1e-12 * np.abs(f_u).max()
    assert e_m == pytest.approx(e_u, rel=1e-13)
    if precision == fg.FIRE_PREC_FP64:
        assert_relax_parity(c, r, ro, 1e-6)
    else:
        assert r.stop == fg.FIRE_STOP_FTOL
        assert abs(r.energy - ro.energy) / c.n < E32_PER_ATOM


def test_frozen_mask_changes_take_effect_and_bad_masks_are_rejected():
    c = fi.rgl_vacancy_box(ncell=4, seed=94, n_vac=1, sigma=0.05)
    with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as h:
        r0 = h.minimize(c.x.copy(), c.box, 1e-6, 100000)
        h.set_dof_mask(np.full(c.n, 7, np.uint8))     # everything frozen
        x = c.x.copy()
        r1 = h.minimize(x, c.box, 1e-6, 100000)
        assert r1.iterations == 0 and r1.stop == fg.FIRE_STOP_FTOL and np.array_equal(x, c.x)
        bad = np.zeros(c.n, np.uint8)
        bad[5] = 8
        with pytest.raises(fg.FireError) as e:
            h.set_dof_mask(bad)
        assert e.value.status == fg.FIRE_ERR_ARG
        h.set_dof_mask(None)
        r2 = h.minimize(c.x.copy(), c.box, 1e-6, 100000)
    # (FP64 atomics: the two runs may differ in the last bits)
    assert abs(r2.iterations - r0.iterations) <= 2
    assert abs(r2.energy - r0.energy) / c.n < 1e-10


# ----------------------------------------------------------------------------
# FP64 tabulated form: half list with atomics (Newton's third law) or full list

@pytest.mark.parametrize("newton", [fg.FIRE_NEWTON_ON, fg.FIRE_NEWTON_OFF])
def test_fp64_table_newton_settings_match_oracle(newton):
    c = fi.rgl_vacancy_box(ncell=7, seed=95, n_vac=4, sigma=0.08)
    eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl(), mode=oracle.FORCE_CELLS)
    pot = rgl_pot()
    pot.newton = newton
    with fg.FireHandle(c.n, fi.CU_MASS, pot, dt_start=fi.CU_DT) as h:
        e, f = h.energy_forces(c.x, c.box)
        x1 = c.x.copy()
        r1 = h.minimize(x1, c.box, 1e-6, 100000)
        x2 = c.x.copy()
        r2 = h.minimize(x2, c.box, 1e-6, 100000)
    assert np.abs(f - fo).max() / np.abs(fo).max() < 1e-10
    assert e == pytest.approx(eo, rel=1e-12)
    _, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS,
                            1e-6, 100000, mode=oracle.FORCE_CELLS)
    assert_relax_parity(c, r1, ro, 1e-6)
    if newton == fg.FIRE_NEWTON_OFF:   # no atomics: the same run twice, bit for bit
        assert np.array_equal(x1, x2) and r1.energy == r2.energy
