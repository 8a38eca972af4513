"""Differentiable form on the GPU (FP64): dE/dtheta, forces and Hessian-vector
products against the oracle, and the implicit gradient of a relaxed vacancy
configuration against the oracle's and against central finite differences
of full relaxations (h = 1e-5 relative), through the C ABI and torch.autograd."""
import numpy as np
import pytest

import fire_inputs as fi
import oracle
import paper_1908_02038_gb300 as fg

pytestmark = pytest.mark.gpu
THETA = ("A", "xi", "p", "q")
THETA0 = [fi.RGL_CU[k] for k in THETA]


@pytest.fixture(scope="module")
def torch():
    import torch
    fg.build()
    fg.load_library()
    return torch


def ora_pot(theta=THETA0):
    kw = dict(fi.RGL_CU)
    kw.update(dict(zip(THETA, theta)))
    return oracle.Potential("rgl", **kw)


def handle(n):
    return fg.FireHandle(n, fi.CU_MASS, fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **fi.RGL_CU),
                         dt_start=fi.CU_DT)


def test_energy_gradient_and_forces_match_oracle(torch):
    c = fi.rgl_vacancy_box(ncell=5, seed=71, n_vac=2, sigma=0.08)
    theta = [0.09, 1.2, 10.5, 2.3]
    dEo, _ = oracle.rgl_param_derivs(c.x, c.box, ora_pot(theta))
    eo, fo = oracle.energy_forces(c.x, c.box, ora_pot(theta))
    d_pos = torch.tensor(c.x, dtype=torch.float64, device="cuda")
    d_f = torch.empty_like(d_pos)
    with handle(c.n) as h:
        e, de = fg.fire_rgl_energy_grad_dev(h.h, d_pos, c.box, theta, d_f)
    assert e == pytest.approx(eo, rel=1e-12)
    np.testing.assert_allclose(de, dEo, rtol=1e-10)
    f = d_f.cpu().numpy()
    assert np.abs(f - fo).max() / np.abs(fo).max() < 1e-10


def test_hvp_matches_oracle(torch):
    c = fi.rgl_vacancy_box(ncell=6, seed=72, n_vac=3, sigma=0.06)
    u = np.random.default_rng(8).normal(size=c.x.shape)
    hu_o = oracle.rgl_hvp(c.x, c.box, ora_pot(), u, mode=oracle.FORCE_CELLS)
    d_pos = torch.tensor(c.x, dtype=torch.float64, device="cuda")
    d_u = torch.tensor(u, dtype=torch.float64, device="cuda")
    d_hu = torch.empty_like(d_u)
    with handle(c.n) as h:
        fg.fire_rgl_hvp_dev(h.h, d_pos, c.box, THETA0, d_u, d_hu)
    hu = d_hu.cpu().numpy()
    assert np.abs(hu - hu_o).max() / np.abs(hu_o).max() < 1e-10


def vacancy_loss(c, radius=6.0):
    site = c.meta["vacancy_sites"][0]
    d = c.meta["lattice"] - site
    d -= c.box * np.rint(d / c.box)
    sel = np.flatnonzero(np.sum(d * d, 1) < radius * radius)

    def loss_grad(x):
        dd = x[sel] - c.meta["lattice"][sel]
        dd -= c.box * np.rint(dd / c.box)
        g = np.zeros_like(x)
        g[sel] = 2.0 * dd
        return float(np.sum(dd * dd)), g
    return sel, loss_grad


def test_implicit_gradient_small_box_matches_oracle(torch):
    c = fi.rgl_vacancy_box(ncell=6, seed=73, n_vac=1, sigma=0.05)
    sel, loss_grad = vacancy_loss(c)
    xo, ro, _ = oracle.fire2(c.x, c.box, ora_pot(), oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS,
                             1e-11, 200000, mode=oracle.FORCE_CELLS)
    assert ro.stop == oracle.STOP_FTOL
    _, go = loss_grad(xo)
    grad_o, _ = oracle.implicit_grad(xo, c.box, ora_pot(), go, tol=1e-12,
                                     mode=oracle.FORCE_CELLS)
    # the GPU gradient at the oracle's own minimum (same input, two implementations)
    d_pos = torch.tensor(xo, dtype=torch.float64, device="cuda")
    d_g = torch.tensor(go, dtype=torch.float64, device="cuda")
    with handle(c.n) as h:
        grad, it = fg.fire_rgl_implicit_grad_dev(h.h, d_pos, c.box, THETA0, d_g, tol=1e-12)
    assert it > 10
    np.testing.assert_allclose(grad, grad_o, rtol=1e-7)


def test_implicit_gradient_32k_matches_finite_differences(torch):
    from paper_1908_02038_gb300.autograd import RGLRelax, theta_tensor
    c = fi.rgl_vacancy_box(ncell=20, seed=5, n_vac=1)
    assert c.n == 31999
    sel, loss_grad = vacancy_loss(c)
    x0 = torch.tensor(c.x, dtype=torch.float64, device="cuda")
    with handle(c.n) as h:
        theta = theta_tensor(fi.RGL_CU)
        xs = RGLRelax.apply(x0, theta, h, c.box, 1e-12, 400000, 1e-12)
        lat = torch.tensor(c.meta["lattice"][sel], dtype=torch.float64, device="cuda")
        box = torch.tensor(c.box, dtype=torch.float64, device="cuda")
        dd = xs[sel] - lat
        dd = dd - box * torch.round(dd / box)
        loss = (dd * dd).sum()
        loss.backward()
        grad = theta.grad.numpy().copy()

        def relaxed_loss(th):
            fg.fire_set_rgl_params(h.h, th)
            x = x0.clone()
            r = fg.fire_minimize_dev(h.h, x, c.box, 1e-12, 400000)
            assert r.stop == fg.FIRE_STOP_FTOL
            return loss_grad(x.cpu().numpy())[0]

        for k in range(4):
            step = 1e-5 * THETA0[k]
            tp, tm = list(THETA0), list(THETA0)
            tp[k] += step
            tm[k] -= step
            fd = (relaxed_loss(tp) - relaxed_loss(tm)) / (2 * step)
            print(f"dL/d{THETA[k]}: implicit {grad[k]:.8e}  finite difference {fd:.8e}")
            assert grad[k] == pytest.approx(fd, rel=1e-4), THETA[k]


def test_autograd_energy_backward(torch):
    from paper_1908_02038_gb300.autograd import RGLEnergy, theta_tensor
    c = fi.rgl_vacancy_box(ncell=4, seed=74, n_vac=1, sigma=0.07)
    pos = torch.tensor(c.x, dtype=torch.float64, device="cuda", requires_grad=True)
    theta = theta_tensor(fi.RGL_CU)
    with handle(c.n) as h:
        e = RGLEnergy.apply(pos, theta, h, c.box)
        e.backward()
    eo, fo = oracle.energy_forces(c.x, c.box, ora_pot())
    dEo, _ = oracle.rgl_param_derivs(c.x, c.box, ora_pot())
    assert e.item() == pytest.approx(eo, rel=1e-12)
    assert np.abs(pos.grad.cpu().numpy() + fo).max() < 1e-10 * np.abs(fo).max()
    np.testing.assert_allclose(theta.grad.numpy(), dEo, rtol=1e-10)


def test_implicit_gradient_reports_unconverged_solve(torch):
    """A CG solve cut off by maxit returns FIRE_ERR_NOT_CONVERGED (with the
    residual in the message), not FIRE_OK; a zero right-hand side is solved
    in 0 iterations."""
    c = fi.rgl_vacancy_box(ncell=5, seed=75, n_vac=1, sigma=0.05)
    d_pos = torch.tensor(c.x, dtype=torch.float64, device="cuda")
    with handle(c.n) as h:
        fg.fire_minimize_dev(h.h, d_pos, c.box, 1e-10, 100000)
        g = torch.zeros_like(d_pos)
        g[0, 0] = 1.0
        with pytest.raises(fg.FireError) as e:
            fg.fire_rgl_implicit_grad_dev(h.h, d_pos, c.box, THETA0, g, tol=1e-12, maxit=1)
        assert e.value.status == fg.FIRE_ERR_NOT_CONVERGED
        assert "maxit" in str(e.value) and "residual" in str(e.value)
        grad, it = fg.fire_rgl_implicit_grad_dev(h.h, d_pos, c.box, THETA0,
                                                 torch.zeros_like(d_pos), tol=1e-12)
        assert it == 0 and np.all(grad == 0.0)


def test_implicit_gradient_32k_matches_oracle_golden(torch):
    """The differentiation workload itself (31,999-atom vacancy box, seed 5):
    the GPU relaxes to max|F_i| < 1e-12 eV/A and solves for dL/dtheta; the
    oracle's gradient of the same workload (relaxed by the oracle to the same
    ftol, its own CG to 1e-12) is stored in tests/golden, written by
    tests/golden/make_implicit_grad_rgl32k.py from oracle/ alone."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "implicit_grad_rgl32k.json")))
    c = fi.rgl_vacancy_box(ncell=20, seed=5, n_vac=1)
    assert c.n == gold["n_atoms"] == 31999
    sel, loss_grad = vacancy_loss(c, gold["radius_A"])
    assert len(sel) == gold["loss_atoms"]
    d_pos = torch.tensor(c.x, dtype=torch.float64, device="cuda")
    with handle(c.n) as h:
        r = fg.fire_minimize_dev(h.h, d_pos, c.box, gold["ftol"], 400000)
        assert r.stop == fg.FIRE_STOP_FTOL
        loss, g = loss_grad(d_pos.cpu().numpy())
        d_g = torch.tensor(g, dtype=torch.float64, device="cuda")
        grad, it = fg.fire_rgl_implicit_grad_dev(h.h, d_pos, c.box, THETA0, d_g,
                                                 tol=gold["cg_tol"])
    print(f"GPU {r.iterations} FIRE iterations, {it} CG iterations; oracle "
          f"{gold['oracle_fire_iterations']} / {gold['oracle_cg_iterations']}")
    assert loss == pytest.approx(gold["loss"], rel=1e-8)
    np.testing.assert_allclose(grad, gold["dL_dtheta"], rtol=1e-6)
