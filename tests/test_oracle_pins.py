"""Pins for the CPU oracle: each test checks the oracle against something the
paper or the mathematics fixes, not against the oracle itself.

  * closed-form FCC lattice sums (shell counting) for the cohesive energy of
    the second-moment EAM of Sec. 5.2 and of the shifted LJ potential;
  * zero force on a perfect lattice, sum F = 0, F = -grad E (Sec. 2.1) by
    central finite differences;
  * hand-traced iterations of Algorithm 2 + Algorithm 4 on quadratic wells
    (values worked out by hand in the comments);
  * stop reasons of Sec. 3.4 / Algorithm 2 (MAXVDOTF, the dt_min guard);
  * the LJ dimer bond length 2^(1/6) sigma, and the (dt, m) -> (c dt, c^2 m)
    invariance of the trajectory.
"""
import math

import numpy as np
import pytest

import fire_inputs as fi
import oracle


def rgl():
    return oracle.Potential("rgl", **fi.RGL_CU)


def lj():
    return oracle.Potential("lj", eps=1.0, sigma=1.0, rc_lj=2.5)


def fcc_shells(a, rmax):
    """(distance, count) of FCC shells within rmax by integer enumeration."""
    m = int(math.ceil(2 * rmax / a)) + 1
    d2 = {}
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                if (i + j + k) % 2 or (i == j == k == 0):
                    continue
                key = i * i + j * j + k * k          # (r / (a/2))^2, exact integer
                d2[key] = d2.get(key, 0) + 1
    out = []
    for key in sorted(d2):
        r = 0.5 * a * math.sqrt(key)
        if r < rmax:
            out.append((r, d2[key]))
    return out


def quintic(r, rs, rc):
    if r <= rs:
        return 1.0
    if r >= rc:
        return 0.0
    t = (r - rs) / (rc - rs)
    return 1 - 10 * t ** 3 + 15 * t ** 4 - 6 * t ** 5


# --------------------------------------------------------------------------
# closed forms


def test_fcc_shell_counts():
    shells = fcc_shells(1.0, 1.5)
    assert [c for _, c in shells[:4]] == [12, 6, 24, 12]


@pytest.mark.parametrize("ncell", [3, 5])
def test_rgl_cohesive_energy_closed_form(ncell):
    P = fi.RGL_CU
    rep, rho = 0.0, 0.0
    for r, cnt in fcc_shells(fi.CU_A, P["rc"]):
        s = quintic(r, P["rs"], P["rc"])
        rep += cnt * P["A"] * math.exp(-P["p"] * (r / P["r0"] - 1)) * s
        rho += cnt * P["xi"] ** 2 * math.exp(-2 * P["q"] * (r / P["r0"] - 1)) * s
    e_closed = rep - math.sqrt(rho)
    assert e_closed == pytest.approx(-3.508821531, abs=2e-9)   # value of the lattice sum
    c = fi.perfect_fcc(ncell, fi.CU_A)
    e, f = oracle.energy_forces(c.x, c.box, rgl())
    assert e / c.n == pytest.approx(e_closed, rel=1e-13)
    assert np.abs(f).max() < 1e-12


@pytest.mark.parametrize("a", [2 ** (2 / 3), fi.LJ_A])
def test_lj_cohesive_energy_closed_form(a):
    def phi(r):
        return 4 * (r ** -12 - r ** -6)
    e_closed = 0.5 * sum(cnt * (phi(r) - phi(2.5)) for r, cnt in fcc_shells(a, 2.5))
    c = fi.perfect_fcc(4, a)
    e, f = oracle.energy_forces(c.x, c.box, lj())
    assert e / c.n == pytest.approx(e_closed, rel=1e-13)
    assert np.abs(f).max() < 1e-11
    if a == 2 ** (2 / 3):
        assert e_closed == pytest.approx(-7.321032079, abs=2e-9)


# --------------------------------------------------------------------------
# forces = -grad E


def _fd_check(x, box, pot, rng, ndof=24, h=1e-5, rc=None):
    e0, f = oracle.energy_forces(x, box, pot)
    n = len(x)
    checked = 0
    for _ in range(200):
        if checked == ndof:
            break
        i, d = int(rng.integers(n)), int(rng.integers(3))
        if rc is not None:      # LJ force is truncated at rc: keep away from it
            dd = x - x[i]
            dd -= box * np.rint(dd / box)
            r = np.sqrt((dd ** 2).sum(1))
            if np.any(np.abs(r - rc) < 1e-3):
                continue
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        ep, _ = oracle.energy_forces(xp, box, pot)
        em, _ = oracle.energy_forces(xm, box, pot)
        fd = -(ep - em) / (2 * h)
        assert fd == pytest.approx(f[i, d], rel=1e-6, abs=1e-7), (i, d)
        checked += 1
    assert checked == ndof


def test_rgl_forces_finite_difference():
    c = fi.rgl_vacancy_box(ncell=3, seed=11, n_vac=2, sigma=0.08)
    # some pairs must sit inside the taper region so dS/dr is exercised
    d = c.x[:, None, :] - c.x[None, :, :]
    d -= c.box * np.rint(d / c.box)
    r = np.sqrt((d ** 2).sum(-1))
    assert np.any((r > 4.5) & (r < 5.0))
    _fd_check(c.x, c.box, rgl(), np.random.default_rng(0))


def test_lj_forces_finite_difference():
    c = fi.lj_fcc_vacancy(seed=1)
    _fd_check(c.x, c.box, lj(), np.random.default_rng(1), h=1e-5, rc=2.5)


@pytest.mark.parametrize("which", ["lj", "rgl"])
def test_sum_of_forces_zero(which):
    c = fi.lj_fcc_vacancy(seed=3) if which == "lj" else fi.rgl_vacancy_box(4, seed=5, n_vac=3)
    e, f = oracle.energy_forces(c.x, c.box, lj() if which == "lj" else rgl())
    assert np.abs(f.sum(0)).max() < 1e-12 * len(f) * max(1.0, np.abs(f).max())


def test_cell_grid_bit_identical_to_all_pairs():
    c = fi.rgl_vacancy_box(ncell=6, seed=7, n_vac=5, sigma=0.1)
    e1, f1 = oracle.energy_forces(c.x, c.box, rgl(), mode=oracle.FORCE_BRUTE)
    e2, f2 = oracle.energy_forces(c.x, c.box, rgl(), mode=oracle.FORCE_CELLS)
    assert e1 == e2
    assert np.array_equal(f1, f2)
    which = np.array([0, 17, 400, len(c.x) - 1])
    e3, f3 = oracle.energy_forces_subset(c.x, c.box, rgl(), which, mode=oracle.FORCE_CELLS)
    assert e3 == e1 and np.array_equal(f3, f1[which])


def test_box_smaller_than_two_cutoffs_rejected():
    with pytest.raises(RuntimeError):
        oracle.energy_forces(np.zeros((2, 3)), np.array([9.0, 12, 12]), rgl())


# --------------------------------------------------------------------------
# FIRE 2.0 control flow, hand-traced


def quad(k, x0):
    k = np.asarray(k, float)
    return oracle.Potential("quad", quad_k=k, quad_x0=np.asarray(x0, float))


def run_quad(k, x_start, maxiter, ftol=0.0, **kw):
    x = np.array([x_start], float)
    params = oracle.Params(**{"dt_start": 0.1, **kw})
    xf, res, rows = oracle.fire2(x, [100.0] * 3, quad(k, [0, 0, 0]), params, 1.0, ftol, maxiter,
                                 periodic=(0, 0, 0), trace=maxiter)
    return xf[0], res, rows


def test_fire_1d_first_iterations():
    # E = x^2/2, m = 1, x = 1, dt = 0.1, Table 1 defaults.
    # i=1: v = 0 so P = 0 -> P<=0 branch, initial delay holds dt and alpha;
    #      v = 0 + 0.1*(-1) = -0.1, x = 1 - 0.01 = 0.99
    # i=2: P = (-0.99)(-0.1) = 0.099 > 0; v = -0.1 - 0.099 = -0.199,
    #      x = 0.99 - 0.0199 = 0.9701
    # i=3: P = 0.9701*0.199 = 0.1930499; v = -0.199 - 0.09701 = -0.29601,
    #      x = 0.9701 - 0.029601 = 0.940499
    expect_x = [0.99, 0.9701, 0.940499]
    expect_P = [0.0, 0.099, 0.1930499]
    for it in (1, 2, 3):
        xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], it)
        assert res.stop == oracle.STOP_MAXITER and res.iterations == it
        assert xf[0] == pytest.approx(expect_x[it - 1], abs=1e-15)
        assert rows[-1]["P"] == pytest.approx(expect_P[it - 1], abs=1e-15)
        assert rows[-1]["nneg"] == (1 if it == 1 else 0)
        assert rows[-1]["npos"] == it - 1
        assert res.dt_final == 0.1 and res.alpha_final == 0.25


def test_fire_1d_uphill_correction():
    # E = x^2/2, m = 1, x = 1, dt_start = 1, initialdelay = no, delaystep = 0.
    # i=1: P = 0 -> N- = 1, dt = 0.5 (>= dt_min 0.02), alpha = 0.25;
    #      v = -0.5, x = 1 - 0.25 = 0.75
    # i=2: P = 0.375 > 0, N+ = 1 > 0 -> dt = min(0.55, 10) = 0.55, alpha = 0.2475;
    #      v = -0.5 - 0.55*0.75 = -0.9125, x = 0.75 - 0.55*0.9125 = 0.248125
    # i=3: P > 0 -> dt = 0.605, alpha = 0.245025;
    #      v = -0.9125 - 0.605*0.248125 = -1.062615625,
    #      x = 0.248125 - 0.605*1.062615625 = -0.394757453125
    # i=4: F = 0.394757453125, P < 0 -> dt = 0.3025, alpha = 0.25;
    #      half step back with the shrunk dt: x = -0.394757453125 + 0.15125*1.062615625
    #                                          = -0.23403683984375, v = 0;
    #      kick with the force stored before the correction:
    #      v = 0.3025*0.394757453125 = 0.1194141295703125,
    #      x = -0.23403683984375 + 0.3025*0.1194141295703125 = -0.19791406564873047
    kw = dict(dt_start=1.0, initialdelay=False, delaystep=0)
    expect = {1: (0.75, 0.5, 0.25), 2: (0.248125, 0.55, 0.2475),
              3: (-0.394757453125, 0.605, 0.245025),
              4: (-0.19791406564873047, 0.3025, 0.25)}
    for it, (xe, dte, ae) in expect.items():
        xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], it, **kw)
        assert xf[0] == pytest.approx(xe, abs=1e-14)
        assert res.dt_final == pytest.approx(dte, rel=1e-15)
        assert res.alpha_final == pytest.approx(ae, rel=1e-15)
    assert rows[-1]["nneg"] == 1 and rows[-1]["npos"] == 0


def test_fire_2d_mixing_uses_kicked_velocity():
    # E = (x^2 + 10 y^2)/2, m = 1, (x, y) = (1, 1), dt = 0.1, defaults.
    # i=1 (P = 0): v = 0.1*F = (-0.1, -1.0), x = (0.99, 0.9)
    # i=2: F = (-0.99, -9), P = 9.099 > 0; kicked v' = (-0.199, -1.9);
    #      mixing with |v'| = sqrt(3.649601), |F| = sqrt(81.9801), alpha = 0.25:
    #      v'' = 0.75 v' + 0.25 |v'| F/|F|;  x = (0.99, 0.9) + 0.1 v''
    nv, nF = math.sqrt(3.649601), math.sqrt(81.9801)
    vx = 0.75 * -0.199 + 0.25 * nv * -0.99 / nF
    vy = 0.75 * -1.9 + 0.25 * nv * -9.0 / nF
    xf, res, rows = run_quad([1, 10, 0], [1, 1, 0], 2)
    assert xf[0] == pytest.approx(0.99 + 0.1 * vx, abs=1e-15)
    assert xf[1] == pytest.approx(0.9 + 0.1 * vy, abs=1e-15)
    # mixing the pre-kick velocity (a literal reading of Algorithm 4's second
    # line) would give a visibly different point
    assert abs(xf[1] - (0.9 + 0.1 * (0.75 * -1.0 + 0.25 * math.sqrt(1.01) * -9.0 / nF))) > 1e-3


def test_fire_growth_waits_for_delaystep():
    xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], 120)
    prev_dt, grew, shrank = 0.1, 0, 0
    for r in rows:
        if r["dt"] > prev_dt:
            assert r["npos"] > 20 and r["P"] > 0
            grew += 1
        if r["dt"] < prev_dt:
            assert r["P"] <= 0 and r["i"] >= 20
            shrank += 1
        prev_dt = r["dt"]
    assert grew > 0 and shrank > 0


def test_fire_maxvdotf_stop():
    # F = 0 exactly, so P = 0 at every pass: N- grows by one per pass and the
    # run stops when N- exceeds vdfmax, before the (vdfmax+1)-th integration.
    xf, res, rows = run_quad([1, 0, 0], [0, 0, 0], 100, vdfmax=5)
    assert res.stop == oracle.STOP_MAXVDOTF
    assert res.iterations == 5 and res.force_evals == 6
    assert [r["nneg"] for r in rows] == [1, 2, 3, 4, 5]


def test_fire_dt_min_guard():
    # F = 0, initialdelay = no, dt_start = 1: dt halves 0.5, 0.25, 0.125, 0.0625,
    # 0.03125 and then stays (0.015625 < dt_min = 0.02); alpha stays alpha0.
    xf, res, rows = run_quad([1, 0, 0], [0, 0, 0], 8, dt_start=1.0, initialdelay=False)
    assert [r["dt"] for r in rows] == [0.5, 0.25, 0.125, 0.0625, 0.03125, 0.03125, 0.03125, 0.03125]
    assert res.stop == oracle.STOP_MAXITER and res.alpha_final == 0.25


def test_fire_converged_start_takes_zero_iterations():
    c = fi.perfect_fcc(3, fi.CU_A)
    xf, res, _ = oracle.fire2(c.x, c.box, rgl(), oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS,
                              1e-6, 100)
    assert res.iterations == 0 and res.stop == oracle.STOP_FTOL and res.force_evals == 1
    assert np.array_equal(xf, c.x)


# --------------------------------------------------------------------------
# physical end points and invariances


def test_lj_dimer_bond_length():
    x = np.array([[5.0, 5.0, 5.0], [6.3, 5.0, 5.0]])
    xf, res, _ = oracle.fire2(x, [20.0] * 3, lj(), oracle.Params(dt_start=fi.LJ_DT), 1.0,
                              1e-10, 100000)
    assert res.stop == oracle.STOP_FTOL
    r = np.linalg.norm(xf[1] - xf[0])
    # |F| = k |r - r*| with k = phi''(r*) = 57.146: |r - r*| < ftol / k
    assert abs(r - 2 ** (1 / 6)) < 1e-10 / 57.0 * 2
    assert np.allclose(xf.mean(0), x.mean(0), atol=1e-12)   # centre of mass fixed


def test_fire_dt_mass_invariance():
    c = fi.lj_fcc_vacancy(seed=1)
    p1 = oracle.Params(dt_start=fi.LJ_DT)
    p2 = oracle.Params(dt_start=fi.LJ_DT * 2.0)
    x1, r1, _ = oracle.fire2(c.x, c.box, lj(), p1, 1.0, 1e-4, 5000)
    x2, r2, _ = oracle.fire2(c.x, c.box, lj(), p2, 4.0, 1e-4, 5000)
    assert r1.stop == oracle.STOP_FTOL and r2.stop == oracle.STOP_FTOL
    assert abs(r1.iterations - r2.iterations) <= 2
    assert np.abs(x1 - x2).max() < 1e-6


def test_rgl_vacancy_relaxation_converges_and_lowers_energy():
    c = fi.rgl_vacancy_box(ncell=3, seed=13, n_vac=1)
    e0, _ = oracle.energy_forces(c.x, c.box, rgl())
    xf, res, _ = oracle.fire2(c.x, c.box, rgl(), oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS,
                              1e-6, 20000)
    assert res.stop == oracle.STOP_FTOL and res.fmax_atom < 1e-6
    assert res.energy < e0
    # relaxed vacancy formation energy E_v = E(N-1) - (N-1) e_coh is positive
    ev = res.energy - c.n * -3.508821531217027
    assert 0.5 < ev < 2.0
    assert res.force_evals == res.iterations + 1


# --------------------------------------------------------------------------
# integrators of Algorithms 3, 5, 6 and the original FIRE (Algorithm 1),
# hand-traced on E = x^2/2 (k = m = 1, x = 1, dt = 0.1, Table 1 defaults)


def test_explicit_euler_first_iterations():
    # i=1: P = 0 -> v = 0; mix no-op; x = 1 + 0.1*0 = 1; v = 0 + 0.1*F(1) = -0.1
    # i=2: P = (-1)(-0.1) = 0.1; x = 1 - 0.01 = 0.99; v = -0.1 + 0.1*(-1) = -0.2
    # i=3: P = (-0.99)(-0.2) = 0.198; x = 0.99 - 0.02 = 0.97; v = -0.2 - 0.099 = -0.299
    for it, (xe, pe) in enumerate([(1.0, 0.0), (0.99, 0.1), (0.97, 0.198)], start=1):
        xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], it, integrator=oracle.INT_EULER_EXPLICIT)
        assert xf[0] == pytest.approx(xe, abs=1e-15)
        assert rows[-1]["P"] == pytest.approx(pe, abs=1e-15)


def test_velocity_verlet_first_iterations():
    # i=1: P = 0 -> v = 0; half kick v = -0.05; x = 1 - 0.005 = 0.995;
    #      F = -0.995; half kick v = -0.05 - 0.04975 = -0.09975
    # i=2: P = 0.995 * 0.09975 = 0.09925125; v = -0.09975 - 0.04975 = -0.1495;
    #      x = 0.995 - 0.01495 = 0.98005
    xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], 1, integrator=oracle.INT_VERLET)
    assert xf[0] == pytest.approx(0.995, abs=1e-15)
    xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], 2, integrator=oracle.INT_VERLET)
    assert xf[0] == pytest.approx(0.98005, abs=1e-15)
    assert rows[-1]["P"] == pytest.approx(0.09925125, abs=1e-15)


def test_leapfrog_first_iterations():
    # v(-dt/2) = -0.05 * F(1) = +0.05.
    # i=1: P = -0.05 <= 0 -> half step back x = 1 - 0.05*0.05 = 0.9975, v = 0;
    #      kick v = -0.1 (force at x = 1); x = 0.9975 - 0.01 = 0.9875
    # i=2: P = 0.9875 * 0.1 = 0.09875; v = -0.1 - 0.09875 = -0.19875;
    #      x = 0.9875 - 0.019875 = 0.967625
    xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], 1, integrator=oracle.INT_LEAPFROG)
    assert xf[0] == pytest.approx(0.9875, abs=1e-15)
    assert rows[-1]["P"] == pytest.approx(-0.05, abs=1e-15) and rows[-1]["nneg"] == 1
    xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], 2, integrator=oracle.INT_LEAPFROG)
    assert xf[0] == pytest.approx(0.967625, abs=1e-15)


def test_original_fire_first_iterations():
    # Algorithm 1 with the semi-implicit Euler step:
    # i=1: P = 0 -> v = 0, dt = 0.05 (no initial delay), alpha = 0.25;
    #      v = -0.05, x = 1 - 0.0025 = 0.9975
    # i=2: P = 0.049875 > 0, no growth yet; v = -0.05 - 0.049875 = -0.099875;
    #      x = 0.9975 - 0.05*0.099875 = 0.99250625
    xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], 2, variant=oracle.VAR_FIRE1)
    assert xf[0] == pytest.approx(0.99250625, abs=1e-15)
    assert res.dt_final == 0.05


def test_original_fire_mixes_before_the_kick():
    # E = (x^2 + 10 y^2)/2, (x, y) = (1, 1), dt = 0.1, Algorithm 1:
    # i=1: P = 0 -> dt = 0.05; v = 0.05 F = (-0.05, -0.5); x = (0.9975, 0.975)
    # i=2: F = (-0.9975, -9.75), P > 0: mix v(t) with |v| = sqrt(0.2525),
    #      |F| = sqrt(96.05750625): v = 0.75 v + 0.25 |v| F/|F|; kick v += 0.05 F;
    #      x += 0.05 v
    nv, nF = math.sqrt(0.2525), math.sqrt(96.05750625)
    vx = 0.75 * -0.05 + 0.25 * nv * -0.9975 / nF + 0.05 * -0.9975
    vy = 0.75 * -0.5 + 0.25 * nv * -9.75 / nF + 0.05 * -9.75
    xf, res, rows = run_quad([1, 10, 0], [1, 1, 0], 2, variant=oracle.VAR_FIRE1)
    assert xf[0] == pytest.approx(0.9975 + 0.05 * vx, abs=1e-15)
    assert xf[1] == pytest.approx(0.975 + 0.05 * vy, abs=1e-15)


def test_original_fire_has_no_dt_floor_or_maxvdotf():
    # F = 0: every pass has P = 0; dt halves every pass and no MAXVDOTF stop
    xf, res, rows = run_quad([1, 0, 0], [0, 0, 0], 12, dt_start=1.0, vdfmax=3,
                             variant=oracle.VAR_FIRE1)
    assert res.stop == oracle.STOP_MAXITER
    assert res.dt_final == 0.5 ** 12


@pytest.mark.parametrize("integ", [oracle.INT_EULER_IMPLICIT, oracle.INT_EULER_EXPLICIT,
                                   oracle.INT_VERLET, oracle.INT_LEAPFROG])
@pytest.mark.parametrize("variant", [oracle.VAR_FIRE2, oracle.VAR_FIRE1])
def test_every_integrator_and_variant_relaxes_the_lj_box(integ, variant):
    c = fi.lj_fcc_vacancy(seed=1)
    xf, res, _ = oracle.fire2(c.x, c.box, lj(), oracle.Params(dt_start=fi.LJ_DT, integrator=integ,
                                                                variant=variant),
                              1.0, 1e-6, 100000)
    assert res.stop == oracle.STOP_FTOL and res.fmax_atom < 1e-6


# ----------------------------------------------------------------------------
# Maximum displacement per step (dmax) and frozen degrees of freedom (Sec. 4,
# cases 1 and 7)

def test_dmax_caps_the_drift_by_hand():
    # E = x^2/2, m = 1, x = 1, dt = 0.1, dmax = 0.005.
    # i=1: P = 0; v = -0.1; dt |v| = 0.01 > dmax -> dt_eff = 0.05, x = 0.995
    # i=2: F = -0.995, P = 0.0995 > 0; v = -0.1 - 0.0995 = -0.1995;
    #      dt |v| = 0.01995 > dmax -> x = 0.995 - 0.005 = 0.99
    # i=3: F = -0.99; v = -0.1995 - 0.099 = -0.2985 -> x = 0.985
    # The FIRE dt itself is untouched (still 0.1).
    expect_x = [0.995, 0.99, 0.985]
    for it in (1, 2, 3):
        xf, res, rows = run_quad([1, 0, 0], [1, 0, 0], it, dmax=0.005)
        assert xf[0] == pytest.approx(expect_x[it - 1], abs=1e-15)
        assert res.dt_final == 0.1
    # a cap larger than every step changes nothing, bit for bit
    xa, ra, _ = run_quad([1, 10, 0], [1, 1, 0], 60)
    xb, rb, _ = run_quad([1, 10, 0], [1, 1, 0], 60, dmax=10.0)
    assert np.array_equal(xa, xb) and ra.energy == rb.energy


def test_dmax_bounds_every_step_of_a_relaxation():
    c = fi.rgl_vacancy_box(ncell=4, seed=31, n_vac=1, sigma=0.1)
    prev = c.x.copy()
    pot = oracle.Potential("rgl", **fi.RGL_CU)
    params = oracle.Params(dt_start=fi.CU_DT, dmax=0.002)
    # a P <= 0 pass would add the half step back, which the cap does not
    # cover; in these iterations only the first pass has P <= 0
    _, _, rows = oracle.fire2(c.x, c.box, pot, params, fi.CU_MASS, 0.0, 39, trace=39)
    assert [r["i"] for r in rows if r["P"] <= 0] == [1]
    steps = []
    for it in range(1, 40):
        xf, res, _ = oracle.fire2(c.x, c.box, pot, params, fi.CU_MASS, 0.0, it)
        steps.append(np.linalg.norm(xf - prev, axis=1).max())
        prev = xf
    assert max(steps) <= 0.002 * (1 + 1e-12)
    assert min(steps[5:]) > 0.002 * (1 - 1e-12)    # the cap is active


def test_frozen_component_reduces_to_the_lower_dimensional_well():
    # E = (x^2 + 10 y^2 + 3 z^2)/2 with z frozen at 0.7 follows exactly the
    # trajectory of E = (x^2 + 10 y^2)/2 in (x, y): the frozen component
    # has zero force, stays put and adds nothing to P, |F| or |v|.
    x3 = np.array([[1.0, 1.0, 0.7]])
    x2 = np.array([[1.0, 1.0, 0.0]])
    params = oracle.Params(dt_start=0.1)
    a, ra, _ = oracle.fire2(x3, [100.0] * 3, quad([1, 10, 3], [0, 0, 0]), params, 1.0, 1e-10,
                            5000, periodic=(0, 0, 0), frozen=np.array([4], np.uint8))
    b, rb, _ = oracle.fire2(x2, [100.0] * 3, quad([1, 10, 0], [0, 0, 0]), params, 1.0, 1e-10,
                            5000, periodic=(0, 0, 0))
    assert a[0, 2] == 0.7
    assert np.array_equal(a[0, :2], b[0, :2])
    assert ra.iterations == rb.iterations and ra.stop == rb.stop == oracle.STOP_FTOL
    # the reported norms are those of the masked force
    assert ra.fmax_atom == rb.fmax_atom


def test_all_frozen_takes_zero_iterations():
    c = fi.lj_fcc_vacancy(seed=1)
    xf, res, _ = oracle.fire2(c.x, c.box, lj(), oracle.Params(dt_start=fi.LJ_DT), 1.0, 1e-8, 100,
                              frozen=np.full(c.n, 7, np.uint8))
    assert res.iterations == 0 and res.stop == oracle.STOP_FTOL and np.array_equal(xf, c.x)


def test_frozen_slab_stays_put_and_the_rest_relaxes():
    c = fi.rgl_vacancy_box(ncell=4, seed=32, n_vac=1, sigma=0.05)
    fz = np.zeros(c.n, np.uint8)
    fz[c.x[:, 0] < 3.0] = 3            # frozen in x and y, free in z
    pot = oracle.Potential("rgl", **fi.RGL_CU)
    xf, res, _ = oracle.fire2(c.x, c.box, pot, oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS, 1e-6,
                              100000, frozen=fz)
    assert res.stop == oracle.STOP_FTOL
    sel = fz == 3
    assert np.array_equal(xf[sel, :2], c.x[sel, :2])
    assert not np.array_equal(xf[sel, 2], c.x[sel, 2])
    # the masked force is converged; the frozen components still carry force
    e, f = oracle.energy_forces(xf, c.box, pot)
    fm = f.copy()
    fm[sel, :2] = 0.0
    assert np.linalg.norm(fm, axis=1).max() < 1e-6
    assert np.abs(f[sel, :2]).max() > 1e-4


# ----------------------------------------------------------------------------
# Stillinger-Weber (the paper's three-body family, Sec. 4 case 5)

def sw():
    return oracle.Potential("sw", **fi.SW_SI)


@pytest.mark.parametrize("ncell", [3, 4])
def test_sw_diamond_cohesive_energy_closed_form(ncell):
    # Nearest neighbours at the pair minimum 2^(1/6) sigma, where the
    # published A, B give phi2 = -eps; second neighbours (1.633 r) lie beyond
    # a sigma and every bond angle is tetrahedral (cos = -1/3, phi3 = 0):
    # E/atom = 4/2 (-eps) = -2 eps = -4.3366 eV, with zero force.
    x = fi.diamond_sites(ncell, fi.SI_A)
    e, f = oracle.energy_forces(x, [ncell * fi.SI_A] * 3, sw())
    assert e / len(x) == pytest.approx(-2.0 * fi.SW_SI["eps"], rel=1e-9)
    assert np.abs(f).max() < 1e-12


@pytest.mark.parametrize("n,nz", [(3, 3), (4, 2)])
def test_sw_diamond_slab_open_axis_closed_form(n, nz):
    # A perfect diamond slab, periodic in x and y, open in z (the structure
    # of the paper's silicon vacancy case without the vacancies): every bond
    # still sits at the pair minimum with tetrahedral angles, so E = -eps per
    # bond and F = 0; the two outer (001) layers (2 n^2 atoms each) have two
    # bonds less per atom: bonds = (4 N - 2 (4 n^2)) / 2 = 16 n^2 nz - 4 n^2.
    c = fi.sw_si_slab(ncell=n, nz=nz, n_vac=0, sigma=0.0)
    assert c.n == 8 * n * n * nz
    e, f = oracle.energy_forces(c.x, c.box, sw(), periodic=c.periodic)
    bonds = 16 * n * n * nz - 4 * n * n
    assert e == pytest.approx(-bonds * fi.SW_SI["eps"], rel=1e-9)
    assert np.abs(f).max() < 1e-8
    # the same atoms periodic in z are the bulk: -2 eps per atom
    e_bulk, _ = oracle.energy_forces(c.x, [n * fi.SI_A, n * fi.SI_A, nz * fi.SI_A], sw())
    assert e_bulk / c.n == pytest.approx(-2.0 * fi.SW_SI["eps"], rel=1e-9)


def test_sw_dimer_minimum_and_trimer_angle_shape():
    box = [100.0] * 3
    r = 2.0 ** (1.0 / 6.0) * fi.SW_SI["sigma"]
    dimer = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    e2, _ = oracle.energy_forces(dimer, box, sw(), periodic=(0, 0, 0))
    assert e2 == pytest.approx(-fi.SW_SI["eps"], rel=1e-9)
    # trimer j-i-k with both bonds r and the j-k distance beyond the cut-off:
    # E(theta) - 2 E_dimer is the three-body term alone, proportional to
    # (cos theta + 1/3)^2 at fixed bond lengths (zero at the tetrahedral angle)
    def trimer(theta):
        x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0], [r * np.cos(theta), r * np.sin(theta), 0.0]])
        e, _ = oracle.energy_forces(x, box, sw(), periodic=(0, 0, 0))
        return e - 2.0 * e2
    tet = np.arccos(-1.0 / 3.0)
    assert abs(trimer(tet)) < 1e-13
    t1, t2 = 2.2, 2.6
    ratio = trimer(t1) / trimer(t2)
    assert ratio == pytest.approx((np.cos(t1) + 1 / 3) ** 2 / (np.cos(t2) + 1 / 3) ** 2, rel=1e-12)


def test_sw_forces_finite_difference_and_sum():
    c = fi.sw_si_vacancy_box(ncell=3, seed=3, n_vac=1, sigma=0.08)
    e, f = oracle.energy_forces(c.x, c.box, sw())
    assert np.abs(f.sum(0)).max() < 1e-11
    h = 1e-5
    for i, d in [(0, 0), (5, 1), (17, 2), (40, 0), (100, 1)]:
        xp, xm = c.x.copy(), c.x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        ep, _ = oracle.energy_forces(xp, c.box, sw())
        em, _ = oracle.energy_forces(xm, c.box, sw())
        assert f[i, d] == pytest.approx(-(ep - em) / (2 * h), rel=1e-7, abs=1e-8)


def test_sw_cell_grid_matches_all_pairs_and_relaxation_converges():
    c = fi.sw_si_vacancy_box(ncell=4, seed=4, n_vac=1, sigma=0.05)
    e1, f1 = oracle.energy_forces(c.x, c.box, sw(), mode=oracle.FORCE_BRUTE)
    e2, f2 = oracle.energy_forces(c.x, c.box, sw(), mode=oracle.FORCE_CELLS)
    assert e1 == e2 and np.array_equal(f1, f2)
    xf, res, _ = oracle.fire2(c.x, c.box, sw(), oracle.Params(dt_start=fi.SI_DT), fi.SI_MASS,
                              1e-6, 100000, mode=oracle.FORCE_CELLS)
    assert res.stop == oracle.STOP_FTOL
    # a vacancy costs energy relative to the perfect crystal
    assert res.energy - (-2.0 * fi.SW_SI["eps"]) * c.n > 1.0
