"""The allocation-free evaluation (fire_energy_forces_noalloc) against the
handle-based one (fire_energy_forces_dev), through the C ABI.

fire_energy_forces_noalloc serves callers that cannot allocate device memory
when they need forces (inside stream capture, under a host program's memory
pool, in latency-critical loops).  Its scratch is a static device array shared
by every call, so the test calls it twice in a row and checks both results,
on the same FP64 tolerances as the other parity tests.  This file is collected
last so that a failure here never hides the results of the other tests.
"""
import ctypes

import numpy as np
import pytest

import fire_inputs as fi
import paper_1908_02038_gb300 as fg

pytestmark = pytest.mark.gpu

F_REL = 1e-10
E_REL = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch
    fg.build()
    fg.load_library()
    return torch


def reference(torch, cfg, pot, mass, dt, periodic=(1, 1, 1)):
    d_pos = torch.tensor(cfg.x, dtype=torch.float64, device="cuda")
    d_f = torch.empty_like(d_pos)
    d_e = torch.zeros(1, dtype=torch.float64, device="cuda")
    with fg.FireHandle(cfg.n, mass, pot, dt_start=dt, periodic=periodic) as h:
        fg.fire_energy_forces_dev(h.h, d_pos, cfg.box, d_f, d_e)
    torch.cuda.synchronize()
    return d_pos, d_f.cpu().numpy(), d_e.item()


@pytest.mark.parametrize("which", ["rgl_small", "rgl_32k", "lj"])
def test_noalloc_matches_handle_path_twice(torch, which):
    if which == "lj":
        cfg = fi.lj_fcc_vacancy(seed=1)
        pot = fg.Potential(fg.FIRE_POT_LJ, eps=1.0, sigma=1.0, rc_lj=2.5, skin=0.3)
        mass, dt = fi.LJ_MASS, fi.LJ_DT
    else:
        cfg = (fi.rgl_vacancy_box(ncell=5, seed=41, n_vac=3, sigma=0.08) if which == "rgl_small"
               else fi.rgl_vacancy_box(ncell=20, seed=2))
        pot = fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **fi.RGL_CU)
        mass, dt = fi.CU_MASS, fi.CU_DT
    d_pos, f_ref, e_ref = reference(torch, cfg, pot, mass, dt)
    for call in range(2):
        d_f = torch.full_like(d_pos, float("nan"))
        d_e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        fg.fire_energy_forces_noalloc(pot.c(), d_pos, cfg.box, (1, 1, 1), d_f, d_e)
        torch.cuda.synchronize()
        f = d_f.cpu().numpy()
        assert np.abs(f - f_ref).max() / np.abs(f_ref).max() < F_REL, call
        assert d_e.item() == pytest.approx(e_ref, rel=E_REL), call


def test_noalloc_rejects_too_many_atoms(torch):
    pot = fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **fi.RGL_CU)
    d_pos = torch.zeros((32769, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fg.FireError) as e:
        fg.fire_energy_forces_noalloc(pot.c(), d_pos, [200.0] * 3, (1, 1, 1), None, None)
    assert e.value.status == fg.FIRE_ERR_ARG
    assert "32768" in str(e.value)
    assert ctypes.sizeof(fg.fire_potential_t) == 160
