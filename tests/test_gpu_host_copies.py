"""Host-pointer calls whose caller arrays sit in page-locked memory: the
library copies results straight into them instead of through its staging
buffer, and they must come out as with ordinary host memory.  The FP32-pair
form writes whole forces and sums in a fixed order, so both runs agree bit
for bit."""
import ctypes as C

import numpy as np
import pytest

import fire_inputs as fi
import paper_1908_02038_gb300 as fg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    fg.build()
    fg.load_library()
    return torch


def pinned_copy(torch, a):
    """A page-locked float64 copy of a (the tensor keeps the memory alive)."""
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    v = t.numpy()
    v[...] = a
    return t, v


def fp32pair_pot():
    return fg.Potential(fg.FIRE_POT_RGL, precision=fg.FIRE_PREC_FP32_PAIR,
                        pair_eval=fg.FIRE_PAIR_ANALYTIC, skin=0.3, **fi.RGL_CU)


def test_minimize_into_pinned_memory(torch):
    c = fi.rgl_vacancy_box(ncell=6, seed=5, n_vac=2, sigma=0.05)
    with fg.FireHandle(c.n, fi.CU_MASS, fp32pair_pot(), dt_start=fi.CU_DT) as h:
        x1 = c.x.copy()
        r1 = h.minimize(x1, c.box, 1e-6, 100000)
        keep, x2 = pinned_copy(torch, c.x)
        r2 = h.minimize(x2, c.box, 1e-6, 100000)
    assert r1.stop == r2.stop == fg.FIRE_STOP_FTOL
    assert (r1.iterations, r1.force_evals) == (r2.iterations, r2.force_evals)
    assert r1.energy == r2.energy
    assert np.array_equal(x1, x2)
    del keep


def test_forces_into_pinned_memory(torch):
    c = fi.rgl_vacancy_box(ncell=5, seed=6, n_vac=1, sigma=0.08)
    lib = fg.load_library()
    with fg.FireHandle(c.n, fi.CU_MASS, fp32pair_pot(), dt_start=fi.CU_DT) as h:
        e1, f1 = h.energy_forces(c.x, c.box)
        pos = np.ascontiguousarray(c.x)
        keep, f2 = pinned_copy(torch, np.zeros_like(pos))
        e2 = C.c_double(0.0)
        box = (C.c_double * 3)(*c.box)
        st = lib.fire_energy_forces(h.h, pos.ctypes.data, box, f2.ctypes.data, C.byref(e2))
        assert st == fg.FIRE_OK
    assert e1 == e2.value
    assert np.array_equal(f1, f2)
    del keep
