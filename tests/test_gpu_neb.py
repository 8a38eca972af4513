"""Nudged elastic band on the GPU (fire_neb_*) against the oracle's NEB on the
same seeded vacancy-hop paths, through the C ABI."""
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


def rgl_pot(precision=fg.FIRE_PREC_FP64, pair_eval=fg.FIRE_PAIR_TABLE):
    return fg.Potential(fg.FIRE_POT_RGL, precision=precision, skin=0.3, pair_eval=pair_eval,
                        **fi.RGL_CU)


def ora_rgl():
    return oracle.Potential("rgl", **fi.RGL_CU)


def hop_path(ncell, n_img, seed=6, mode=oracle.FORCE_BRUTE):
    """Relaxed end states (oracle) and the straight-line path between them."""
    c = fi.neb_vacancy_hop(ncell=ncell, seed=seed, n_img=n_img)
    ends = []
    for e in (0, -1):
        xr, rr, _ = oracle.fire2(c.x[e], c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT),
                                 fi.CU_MASS, 1e-8, 100000, mode=mode)
        assert rr.stop == oracle.STOP_FTOL
        ends.append(xr)
    t = np.linspace(0.0, 1.0, n_img + 2)[:, None, None]
    return c, np.ascontiguousarray(ends[0][None] + t * (ends[1] - ends[0])[None])


def assert_neb_parity(c, r, E, cl, ro, Eo, clo, n_img):
    n = c.x.shape[1]
    assert ro.stop == oracle.STOP_FTOL and r.stop == fg.FIRE_STOP_FTOL
    assert cl == clo
    assert np.abs(E - Eo).max() / n < 1e-8, np.abs(E - Eo).max()
    assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations), \
        (r.iterations, ro.iterations)


@pytest.mark.parametrize("climb", [True, False])
def test_neb_small_box_matches_oracle(climb):
    c, path = hop_path(3, 5)
    po, ro, Eo, clo = oracle.neb(path, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT),
                                 fi.CU_MASS, 1.0, climb, 1e-6, 100000)
    p = path.copy()
    with fg.FireNEB(5, path.shape[1], fi.CU_MASS, rgl_pot(), 1.0, climb, dt_start=fi.CU_DT) as h:
        r, E, cl = h.minimize(p, c.box, 1e-6, 100000)
    assert_neb_parity(c, r, E, cl, ro, Eo, clo, 5)
    assert np.array_equal(p[0], path[0]) and np.array_equal(p[-1], path[-1])
    assert np.abs(p - po).max() < 1e-5
    assert (E[3] - E[0] > 0.5) if climb else (E.max() - E[0] > 0.5)


@pytest.mark.parametrize("mode,chunk", [(fg.FIRE_EXEC_GRAPH_WHILE, 0), (fg.FIRE_EXEC_GRAPH_WHILE, 1),
                                        (fg.FIRE_EXEC_CHUNKED, 16)])
def test_neb_cell_list_box_matches_oracle(mode, chunk):
    # 6^3 cells: the list build runs in cell mode, each image in its own cells
    c, path = hop_path(6, 7, seed=8, mode=oracle.FORCE_CELLS)
    po, ro, Eo, clo = oracle.neb(path, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT),
                                 fi.CU_MASS, 2.0, True, 1e-6, 100000, mode=oracle.FORCE_CELLS)
    p = path.copy()
    with fg.FireNEB(7, path.shape[1], fi.CU_MASS, rgl_pot(), 2.0, True, dt_start=fi.CU_DT) as h:
        h.set_exec_mode(mode, chunk)
        r, E, cl = h.minimize(p, c.box, 1e-6, 100000)
    assert_neb_parity(c, r, E, cl, ro, Eo, clo, 7)
    assert cl == 4
    # the climbing image is a saddle of the true potential: its force is below ftol
    _, f = oracle.energy_forces(p[cl], c.box, ora_rgl(), mode=oracle.FORCE_CELLS)
    assert np.linalg.norm(f, axis=1).max() < 1e-6


def test_neb_device_path_and_frozen_layer():
    c, path = hop_path(4, 5, seed=9)
    n = path.shape[1]
    fz = np.zeros(n, np.uint8)
    fz[path[0][:, 2] < 2.0] = 7          # a frozen layer, away from the hop
    assert not fz[c.meta["hopper"]]
    po, ro, Eo, clo = oracle.neb(path, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT),
                                 fi.CU_MASS, 1.0, True, 1e-6, 100000, frozen=fz)
    import torch
    d = torch.tensor(path, dtype=torch.float64, device="cuda")
    with fg.FireNEB(5, n, fi.CU_MASS, rgl_pot(), 1.0, True, dt_start=fi.CU_DT) as h:
        h.set_dof_mask(fz)
        r, E, cl = h.minimize_dev(d, c.box, 1e-6, 100000)
    torch.cuda.synchronize()
    p = d.cpu().numpy()
    assert_neb_parity(c, r, E, cl, ro, Eo, clo, 5)
    sel = fz == 7
    assert np.array_equal(p[:, sel], path[:, sel])


@pytest.mark.parametrize("check", [fg.FIRE_FP64_CHECK_CONFIRM, fg.FIRE_FP64_CHECK_FINISH])
def test_neb_fp32pair_reaches_the_fp64_barrier(check):
    c, path = hop_path(6, 5, seed=10, mode=oracle.FORCE_CELLS)
    res = {}
    for prec in (fg.FIRE_PREC_FP64, fg.FIRE_PREC_FP32_PAIR):
        p = path.copy()
        with fg.FireNEB(5, path.shape[1], fi.CU_MASS, rgl_pot(prec, fg.FIRE_PAIR_ANALYTIC), 1.0,
                        True, dt_start=fi.CU_DT, confirm64=check) as h:
            r, E, cl = h.minimize(p, c.box, 1e-5, 100000)
        assert r.stop == fg.FIRE_STOP_FTOL and cl == 3
        res[prec] = (E[cl] - E[0], p)
    b64, b32 = res[fg.FIRE_PREC_FP64][0], res[fg.FIRE_PREC_FP32_PAIR][0]
    assert abs(b32 - b64) < 1e-4, (b64, b32)
    # the FP32-pair saddle checked in FP64: below ten times ftol
    _, f = oracle.energy_forces(res[fg.FIRE_PREC_FP32_PAIR][1][3], c.box, ora_rgl(),
                                mode=oracle.FORCE_CELLS)
    assert np.linalg.norm(f, axis=1).max() < 1e-4


def test_neb_rejects_wrong_calls():
    c, path = hop_path(3, 3)
    with fg.FireNEB(3, path.shape[1], fi.CU_MASS, rgl_pot(), 1.0, True, dt_start=fi.CU_DT) as h:
        with pytest.raises(fg.FireError) as e:
            fg.fire_minimize(h.h, path[1].copy(), c.box, 1e-6, 10)
        assert e.value.status == fg.FIRE_ERR_STATE
        with pytest.raises(ValueError):
            h.minimize(path[:3].copy(), c.box, 1e-6, 10)
    with pytest.raises(fg.FireError) as e:
        fg.FireNEB(0, 10, fi.CU_MASS, rgl_pot(), 1.0, dt_start=fi.CU_DT)
    assert e.value.status == fg.FIRE_ERR_ARG
