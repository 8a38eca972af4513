"""Batched form (one persistent launch, one CTA per system at a time) against
the FP64 oracle and against the single-system path, through the C ABI."""
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


def rgl_pot(precision=fg.FIRE_PREC_FP64, pair_eval=fg.FIRE_PAIR_TABLE):
    # FP64: the table form (double-float pair terms) by default, the IEEE-FP64
    # exponentials with FIRE_PAIR_ANALYTIC
    return fg.Potential(fg.FIRE_POT_RGL, precision=precision, pair_eval=pair_eval, skin=0.3,
                        **fi.RGL_CU)


FP64_FORMS = [fg.FIRE_PAIR_TABLE, fg.FIRE_PAIR_ANALYTIC]


def ora_rgl():
    return oracle.Potential("rgl", **fi.RGL_CU)


def pack(cfgs):
    x = np.ascontiguousarray(np.concatenate([c.x for c in cfgs]))
    boxes = np.array([c.box for c in cfgs])
    counts = [c.n for c in cfgs]
    return x, boxes, counts


def small_batch(n_sys=10, seed=50):
    # sizes 3^3..6^3 cells: both the all-pairs and the cell-list build paths
    return fi.rgl_batch(n_sys=n_sys, seed=seed, nmin=3, nmax=6)


@pytest.mark.parametrize("pair_eval", FP64_FORMS)
def test_batch_fp64_forces_match_oracle(pair_eval):
    cfgs = small_batch()
    x, boxes, counts = pack(cfgs)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(pair_eval=pair_eval), dt_start=fi.CU_DT) as b:
        res, f = b.minimize(x.copy(), boxes, 1e-6, 0, want_forces=True)
    off = np.concatenate([[0], np.cumsum(counts)])
    for s, c in enumerate(cfgs):
        eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl())
        fs = f[off[s]:off[s + 1]]
        assert np.abs(fs - fo).max() / np.abs(fo).max() < 1e-10, s
        assert res[s].energy == pytest.approx(eo, rel=1e-12)
        assert res[s].iterations == 0 and res[s].stop == fg.FIRE_STOP_MAXITER


@pytest.mark.parametrize("pair_eval", FP64_FORMS)
def test_batch_fp64_relaxations_match_oracle(pair_eval):
    cfgs = small_batch(n_sys=8, seed=51)
    x, boxes, counts = pack(cfgs)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(pair_eval=pair_eval), dt_start=fi.CU_DT) as b:
        res, _ = b.minimize(x, boxes, 1e-6, 100000)
    for s, c in enumerate(cfgs):
        _, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT),
                                fi.CU_MASS, 1e-6, 100000)
        r = res[s]
        assert ro.stop == oracle.STOP_FTOL and r.stop == fg.FIRE_STOP_FTOL, s
        assert r.fmax_atom < 1e-6
        assert abs(r.energy - ro.energy) / c.n < 1e-8, s
        assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations), \
            (s, r.iterations, ro.iterations)


def test_batch_matches_single_system_path_and_tuning_does_not_change_results():
    cfgs = small_batch(n_sys=6, seed=52)
    x, boxes, counts = pack(cfgs)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(fg.FIRE_PREC_FP32_PAIR),
                      dt_start=fi.CU_DT) as b:
        tuned = b.autotune(x, boxes, iters=10)
        assert tuned["threads_per_block"] in (64, 128, 192, 256, 384, 512, 768, 1024)
        r1, _ = b.minimize(x.copy(), boxes, 1e-6, 100000)
        b.set_tuning(64, 1)
        r2, _ = b.minimize(x.copy(), boxes, 1e-6, 100000)
    for s, c in enumerate(cfgs):
        # like the batch, the single-system path stopping on the FP32-pair
        # forces (no FP64 confirmation), so both report FP32-pair energies
        with fg.FireHandle(c.n, fi.CU_MASS, rgl_pot(fg.FIRE_PREC_FP32_PAIR),
                           dt_start=fi.CU_DT, confirm64=0) as h:
            rs = h.minimize(c.x.copy(), c.box, 1e-6, 100000)
        for r in (r1[s], r2[s]):
            assert r.stop == fg.FIRE_STOP_FTOL
            assert abs(r.energy - rs.energy) / c.n < 1e-7


@pytest.mark.parametrize("check", [fg.FIRE_FP64_CHECK_CONFIRM, fg.FIRE_FP64_CHECK_FINISH])
def test_batch_fp32pair_stops_meet_ftol_in_fp64(check):
    # every system's stop is checked in FP64 (confirmation, or the FP64
    # finish below 3 ftol): the structures meet ftol with FP64 forces
    cfgs = fi.rgl_batch(n_sys=24, seed=57, nmin=3, nmax=8)
    x, boxes, counts = pack(cfgs)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(fg.FIRE_PREC_FP32_PAIR),
                      dt_start=fi.CU_DT, confirm64=check) as b:
        res, _ = b.minimize(x, boxes, 1e-6, 100000)
    assert all(r.stop == fg.FIRE_STOP_FTOL for r in res)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as b64:
        chk, _ = b64.minimize(x.copy(), boxes, 1e-6, 0)
    for s, (r, rc) in enumerate(zip(res, chk)):
        assert rc.fmax_atom < 1e-6, (s, rc.fmax_atom)
        # the reported norm and energy come from the FP64 evaluation
        assert abs(r.fmax_atom - rc.fmax_atom) < 1e-10, s
        assert abs(r.energy - rc.energy) / counts[s] < 1e-12, s


def test_batch_512_fp32_all_converge_and_sample_matches_oracle():
    cfgs = fi.rgl_batch()           # 512 systems, 3^3..12^3 cells, 1-3 vacancies
    x, boxes, counts = pack(cfgs)
    assert len(cfgs) == 512
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(fg.FIRE_PREC_FP32_PAIR),
                      dt_start=fi.CU_DT) as b:
        b.autotune(x, boxes, iters=10)
        xr = x.copy()
        res, _ = b.minimize(xr, boxes, 1e-6, 100000)
    assert all(r.stop == fg.FIRE_STOP_FTOL for r in res)
    assert max(r.fmax_atom for r in res) < 1e-6
    off = np.concatenate([[0], np.cumsum(counts)])
    rng = np.random.default_rng(0)
    for s in rng.choice(512, size=6, replace=False):
        c = cfgs[s]
        eo, fo = oracle.energy_forces(xr[off[s]:off[s + 1]], c.box, ora_rgl(),
                                      mode=oracle.FORCE_CELLS)
        # the FP32-pair minimum judged by FP64 oracle forces
        assert np.sqrt((fo ** 2).sum(1)).max() < 2e-6, s
        assert abs(res[s].energy - eo) / c.n < 1e-6, s


def test_batch_rejects_single_system_calls():
    cfgs = small_batch(n_sys=2)
    x, boxes, counts = pack(cfgs)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as b:
        with pytest.raises(fg.FireError) as e:
            fg.fire_energy_forces(b.h, x, boxes[0])
        assert e.value.status == fg.FIRE_ERR_STATE
        xbad = x.copy()
        xbad[3, 0] = np.inf
        with pytest.raises(fg.FireError) as e:
            b.minimize(xbad, boxes, 1e-6, 100)
        assert e.value.status == fg.FIRE_ERR_NONFINITE
        assert np.isinf(xbad[3, 0])


def test_batch_dmax_relaxations_match_oracle():
    cfgs = small_batch(n_sys=5, seed=53)
    x, boxes, counts = pack(cfgs)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT, dmax=0.002) as b:
        res, _ = b.minimize(x, boxes, 1e-6, 100000)
    for s, c in enumerate(cfgs):
        _, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(),
                                oracle.Params(dt_start=fi.CU_DT, dmax=0.002), fi.CU_MASS, 1e-6,
                                100000)
        r = res[s]
        assert ro.stop == oracle.STOP_FTOL and r.stop == fg.FIRE_STOP_FTOL, s
        assert abs(r.energy - ro.energy) / c.n < 1e-8, s
        assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations), \
            (s, r.iterations, ro.iterations)


@pytest.mark.parametrize("cluster", [2, 4])
def test_batch_clusters_share_systems_and_match_oracle(cluster):
    # clusters of CTAs split every system's atoms and combine the reductions
    # through distributed shared memory; FP64 parity per system as for one CTA
    cfgs = small_batch(n_sys=7, seed=54)
    x, boxes, counts = pack(cfgs)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as b:
        b.set_tuning(256, 2, cluster)
        res, f = b.minimize(x.copy(), boxes, 1e-6, 100000, want_forces=True)
        r0, f0 = b.minimize(x.copy(), boxes, 1e-6, 0, want_forces=True)
    off = np.concatenate([[0], np.cumsum(counts)])
    for s, c in enumerate(cfgs):
        eo, fo = oracle.energy_forces(c.x, c.box, ora_rgl())
        assert np.abs(f0[off[s]:off[s + 1]] - fo).max() / np.abs(fo).max() < 1e-10, s
        assert r0[s].energy == pytest.approx(eo, rel=1e-12)
        _, ro, _ = oracle.fire2(c.x, c.box, ora_rgl(), oracle.Params(dt_start=fi.CU_DT),
                                fi.CU_MASS, 1e-6, 100000)
        r = res[s]
        assert r.stop == fg.FIRE_STOP_FTOL and r.fmax_atom < 1e-6, s
        assert abs(r.energy - ro.energy) / c.n < 1e-8, s
        assert abs(r.iterations - ro.iterations) <= max(2, 0.05 * ro.iterations), \
            (s, r.iterations, ro.iterations)


def test_batch_512_fp32_with_clusters_converges():
    cfgs = fi.rgl_batch()
    x, boxes, counts = pack(cfgs)
    with fg.FireBatch(counts, fi.CU_MASS, rgl_pot(fg.FIRE_PREC_FP32_PAIR),
                      dt_start=fi.CU_DT) as b:
        b.set_tuning(512, 1, 2)
        res, _ = b.minimize(x, boxes, 0.9e-6, 200000)
    assert all(r.stop == fg.FIRE_STOP_FTOL for r in res)
    with pytest.raises(fg.FireError):
        with fg.FireBatch(counts[:4], fi.CU_MASS, rgl_pot(), dt_start=fi.CU_DT) as b:
            b.set_tuning(256, 1, 3)
