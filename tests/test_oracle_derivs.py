"""Pins for the oracle's derivatives (differentiable form, RGL only):
central finite differences of E and F in theta = (A, xi, p, q) and in x,
symmetry of the Hessian, its translation zero modes, and the implicit
gradient of a relaxed configuration against finite differences of full
relaxations."""
import numpy as np
import pytest

import fire_inputs as fi
import oracle

THETA = ("A", "xi", "p", "q")


def pot_with(**over):
    kw = dict(fi.RGL_CU)
    kw.update(over)
    return oracle.Potential("rgl", **kw)


@pytest.fixture(scope="module")
def cfg():
    return fi.rgl_vacancy_box(ncell=3, seed=61, n_vac=2, sigma=0.08)


def test_energy_and_force_theta_derivatives(cfg):
    dE, dF = oracle.rgl_param_derivs(cfg.x, cfg.box, pot_with())
    for k, name in enumerate(THETA):
        v = fi.RGL_CU[name]
        h = 1e-6 * v
        ep, fp = oracle.energy_forces(cfg.x, cfg.box, pot_with(**{name: v + h}))
        em, fm = oracle.energy_forces(cfg.x, cfg.box, pot_with(**{name: v - h}))
        assert dE[k] == pytest.approx((ep - em) / (2 * h), rel=1e-7), name
        fd = (fp - fm) / (2 * h)
        assert np.abs(dF[k] - fd).max() < 1e-6 * np.abs(fd).max(), name


def test_hvp_matches_force_differences(cfg):
    rng = np.random.default_rng(3)
    u = rng.normal(size=cfg.x.shape)
    hu = oracle.rgl_hvp(cfg.x, cfg.box, pot_with(), u)
    eps = 1e-6
    _, fp = oracle.energy_forces(cfg.x + eps * u, cfg.box, pot_with())
    _, fm = oracle.energy_forces(cfg.x - eps * u, cfg.box, pot_with())
    fd = -(fp - fm) / (2 * eps)
    assert np.abs(hu - fd).max() < 1e-6 * np.abs(fd).max()


def test_hvp_symmetric_and_translation_free(cfg):
    rng = np.random.default_rng(4)
    u, v = rng.normal(size=cfg.x.shape), rng.normal(size=cfg.x.shape)
    hu = oracle.rgl_hvp(cfg.x, cfg.box, pot_with(), u)
    hv = oracle.rgl_hvp(cfg.x, cfg.box, pot_with(), v)
    assert np.sum(v * hu) == pytest.approx(np.sum(u * hv), rel=1e-11)
    t = np.zeros_like(cfg.x)
    t[:, 1] = 1.0
    assert np.abs(oracle.rgl_hvp(cfg.x, cfg.box, pot_with(), t)).max() < 1e-11


def test_cell_mode_matches_all_pairs():
    c = fi.rgl_vacancy_box(ncell=6, seed=62, n_vac=3, sigma=0.06)
    u = np.random.default_rng(5).normal(size=c.x.shape)
    h1 = oracle.rgl_hvp(c.x, c.box, pot_with(), u, mode=oracle.FORCE_BRUTE)
    h2 = oracle.rgl_hvp(c.x, c.box, pot_with(), u, mode=oracle.FORCE_CELLS)
    assert np.array_equal(h1, h2)


def vacancy_loss_setup(c, radius=6.0):
    site = c.meta["vacancy_sites"][0]
    d = c.meta["lattice"] - site
    d -= c.box * np.rint(d / c.box)
    return np.flatnonzero(np.sum(d * d, 1) < radius * radius)


def loss_and_grad(x, c, sel):
    d = x[sel] - c.meta["lattice"][sel]
    d -= c.box * np.rint(d / c.box)
    g = np.zeros_like(x)
    g[sel] = 2.0 * d
    return float(np.sum(d * d)), g


def test_implicit_gradient_matches_relaxation_differences():
    c = fi.rgl_vacancy_box(ncell=4, seed=63, n_vac=1, sigma=0.05)
    sel = vacancy_loss_setup(c)
    assert 10 < len(sel) < 80
    par = oracle.Params(dt_start=fi.CU_DT)

    def relax(pot):
        x, r, _ = oracle.fire2(c.x, c.box, pot, par, fi.CU_MASS, 1e-11, 200000)
        assert r.stop == oracle.STOP_FTOL
        return x

    xs = relax(pot_with())
    _, g = loss_and_grad(xs, c, sel)
    grad, it = oracle.implicit_grad(xs, c.box, pot_with(), g, tol=1e-12)
    assert it > 0
    for k, name in enumerate(THETA):
        v = fi.RGL_CU[name]
        h = 1e-5 * v
        lp, _ = loss_and_grad(relax(pot_with(**{name: v + h})), c, sel)
        lm, _ = loss_and_grad(relax(pot_with(**{name: v - h})), c, sel)
        fd = (lp - lm) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-4, abs=1e-9), (name, grad[k], fd)
