"""Pins of the oracle's nudged elastic band (the paper's cases 7 and 8: FIRE
2.0 on an ensemble of images with modified forces).  Closed forms on a
double-well test surface (saddle position and height, symmetry, equal
spacing, the minimum energy path from the saddle), and on a Cu vacancy hop
the defining properties of a first-order saddle (vanishing true force,
negative curvature along the path)."""
import numpy as np
import pytest

import fire_inputs as fi
import oracle

H, A, C, KY, KZ = 1.0, 1.0, 0.5, 5.0, 2.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def dwell():
    return oracle.Potential("dwell", dwell=(H, A, C, KY, KZ))


def dwell_path(m, bend=0.3):
    e0, e1 = np.array([[-A, C * A * A, 0.0]]), np.array([[A, C * A * A, 0.0]])
    path = np.array([e0 + (e1 - e0) * t for t in np.linspace(0.0, 1.0, m + 2)])
    path[1:-1, 0, 1] += bend
    path[1:-1, 0, 2] += 0.1
    return path


def run_dwell(m, climb, k=2.0, ftol=1e-10):
    return oracle.neb(dwell_path(m), [100.0] * 3, dwell(), oracle.Params(dt_start=0.01), 1.0, k,
                      climb, ftol, 200000, periodic=(0, 0, 0))


def test_dwell_surface_forces_finite_difference():
    x = np.array([[0.3, -0.2, 0.15], [-1.2, 0.8, -0.4]])
    e, f = oracle.energy_forces(x, [100.0] * 3, dwell(), periodic=(0, 0, 0))
    h = 1e-6
    for i in range(2):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            ep, _ = oracle.energy_forces(xp, [100.0] * 3, dwell(), periodic=(0, 0, 0))
            em, _ = oracle.energy_forces(xm, [100.0] * 3, dwell(), periodic=(0, 0, 0))
            assert f[i, d] == pytest.approx(-(ep - em) / (2 * h), abs=1e-8)
    # the closed-form stationary points
    e_min, f_min = oracle.energy_forces(np.array([[A, C * A * A, 0.0]]), [100.0] * 3, dwell(),
                                        periodic=(0, 0, 0))
    e_sad, f_sad = oracle.energy_forces(np.zeros((1, 3)), [100.0] * 3, dwell(), periodic=(0, 0, 0))
    assert e_min == 0.0 and np.all(f_min == 0.0)
    assert e_sad == H and np.all(f_sad == 0.0)


def test_climbing_image_lands_on_the_saddle():
    # 7 movable images on a symmetric path: the middle one climbs to the
    # saddle (0, 0, 0) of height h; the end states do not move
    path0 = dwell_path(7)
    out, r, E, cl = run_dwell(7, True)
    assert r.stop == oracle.STOP_FTOL and cl == 4
    # the true force there is the NEB force up to the sign of its tangent
    # component, so it is below ftol; curvature 4h/a^2 along x, 2 ky along y
    assert np.abs(out[4, 0]).max() < 1e-9
    assert E[4] == pytest.approx(H, abs=1e-15)
    assert np.array_equal(out[0], path0[0]) and np.array_equal(out[-1], path0[-1])
    assert E[0] == 0.0 and E[-1] == 0.0
    np.testing.assert_allclose(E, E[::-1], atol=1e-12)


def test_plain_band_is_symmetric_equally_spaced_and_below_the_saddle():
    out, r, E, cl = run_dwell(6, False, k=3.0)
    assert r.stop == oracle.STOP_FTOL and cl == 0
    seg = np.linalg.norm(np.diff(out[:, 0, :], axis=0), axis=1)
    # converged: k (|t+| - |t-|) = 0 at every image, so equal spacing
    np.testing.assert_allclose(seg, seg.mean(), rtol=1e-8)
    np.testing.assert_allclose(E, E[::-1], atol=1e-12)
    np.testing.assert_allclose(out[1:-1, 0, 0], -out[-2:0:-1, 0, 0], atol=1e-9)
    assert E.max() < H
    assert np.abs(out[1:-1, 0, 2]).max() < 1e-9          # z relaxed to 0


def test_band_follows_the_minimum_energy_path():
    # the minimum energy path: steepest descent from the saddle along its
    # unstable direction (x), integrated independently of the oracle with
    # the closed-form gradient
    from scipy.integrate import solve_ivp

    def grad(_, p):
        x, y = p
        w = x * x / (A * A) - 1.0
        g = np.array([4 * H * w * x / (A * A) - 4 * KY * C * x * (y - C * x * x),
                      2 * KY * (y - C * x * x)])
        return -g / max(np.linalg.norm(g), 1e-300)

    def near_minimum(_, p):
        return np.hypot(p[0] - A, p[1] - C * A * A) - 1e-3
    near_minimum.terminal = True

    sol = solve_ivp(grad, (0.0, 3.0), [1e-7, 0.0], rtol=1e-10, atol=1e-12, max_step=1e-3,
                    events=near_minimum)
    assert sol.status == 1                     # reached the minimum
    curve = sol.y.T
    worst = {}
    for m in (9, 19):
        out, r, E, cl = run_dwell(m, True)
        assert r.stop == oracle.STOP_FTOL
        worst[m] = max(np.min(np.linalg.norm(curve - np.array([abs(p[0]), p[1]]), axis=1))
                       for p in out[1:-1, 0, :2])
    # the images sit on the path up to the discretisation of the tangent,
    # which shrinks as the band gets finer
    assert worst[9] < 1.5e-2 and worst[19] < 0.6 * worst[9], worst


def test_vacancy_hop_climbing_image_is_a_first_order_saddle():
    c = fi.neb_vacancy_hop(ncell=3, seed=6, n_img=5)
    pot = oracle.Potential("rgl", **fi.RGL_CU)
    params = oracle.Params(dt_start=fi.CU_DT)
    path = c.x.copy()
    for end in (0, -1):
        xr, rr, _ = oracle.fire2(path[end], c.box, pot, params, fi.CU_MASS, 1e-8, 100000)
        assert rr.stop == oracle.STOP_FTOL
        path[end] = xr
    t = np.linspace(0.0, 1.0, 7)[:, None, None]
    path = path[0][None] + t * (path[-1] - path[0])[None]
    out, r, E, cl = oracle.neb(path, c.box, pot, params, fi.CU_MASS, 1.0, True, 1e-6, 200000)
    assert r.stop == oracle.STOP_FTOL and cl == 3
    # symmetric hop between equivalent sites: symmetric profile, a barrier
    np.testing.assert_allclose(E - E[0], (E - E[0])[::-1], atol=1e-6)
    assert E[3] - E[0] > 0.5
    # at the climbing image the true force is below ftol ...
    _, f = oracle.energy_forces(out[3], c.box, pot)
    assert np.linalg.norm(f, axis=1).max() < 1e-6
    # ... and the curvature along the band is negative: tau.H.tau < 0
    tau = out[4] - out[2]
    tau /= np.linalg.norm(tau)
    hu = oracle.rgl_hvp(out[3], c.box, pot, tau)
    assert float(np.sum(tau * hu)) < -0.1
    # the neighbouring images are not saddles: their true force is finite
    _, f2 = oracle.energy_forces(out[2], c.box, pot)
    assert np.linalg.norm(f2, axis=1).max() > 1e-2
