"""The allocation-free evaluation (fire_energy_forces_noalloc) through the C
ABI, against the FP64 CPU oracle and against the handle-based entry point
(fire_energy_forces_dev).

fire_energy_forces_noalloc serves callers that cannot allocate device memory
when they need forces: plug-ins whose host program's memory pool owns all
device memory, and latency-critical loops where an allocation could
synchronise the device.  Its scratch is a static device array shared by every
call, so each test calls it twice in a row and checks both results, on the
same FP64 tolerances as the other parity tests (forces 1e-10 relative,
energy 1e-12).  This file is collected last so that a failure here never
hides the results of the other tests.
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


def workload(which):
    if which == "lj":
        cfg = fi.lj_fcc_vacancy(seed=1)
        return (cfg, fg.Potential(fg.FIRE_POT_LJ, eps=1.0, sigma=1.0, rc_lj=2.5, skin=0.3),
                oracle.Potential("lj", eps=1.0, sigma=1.0, rc_lj=2.5), fi.LJ_MASS, fi.LJ_DT)
    cfg = (fi.rgl_vacancy_box(ncell=5, seed=41, n_vac=3, sigma=0.08) if which == "rgl_small"
           else fi.rgl_vacancy_box(ncell=20, seed=2))
    return (cfg, fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **fi.RGL_CU),
            oracle.Potential("rgl", **fi.RGL_CU), fi.CU_MASS, fi.CU_DT)


def call_twice(torch, pot, d_pos, box):
    out = []
    for _ in range(2):
        d_f = torch.full_like(d_pos, float("nan"))
        d_e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        fg.fire_energy_forces_noalloc(pot.c(), d_pos, box, (1, 1, 1), d_f, d_e)
        torch.cuda.synchronize()
        out.append((d_f.cpu().numpy(), d_e.item()))
    return out


@pytest.mark.parametrize("which", ["rgl_small", "rgl_32k", "lj"])
def test_noalloc_matches_handle_path_twice(torch, which):
    cfg, pot, _, mass, dt = workload(which)
    d_pos, f_ref, e_ref = reference(torch, cfg, pot, mass, dt)
    for call, (f, e) in enumerate(call_twice(torch, pot, d_pos, cfg.box)):
        assert np.abs(f - f_ref).max() / np.abs(f_ref).max() < F_REL, call
        assert e == pytest.approx(e_ref, rel=E_REL), call


@pytest.mark.parametrize("which", ["rgl_small", "lj"])
def test_noalloc_matches_oracle_twice(torch, which):
    cfg, pot, opot, _, _ = workload(which)
    eo, fo = oracle.energy_forces(cfg.x, cfg.box, opot)
    d_pos = torch.tensor(cfg.x, dtype=torch.float64, device="cuda")
    for call, (f, e) in enumerate(call_twice(torch, pot, d_pos, cfg.box)):
        assert np.abs(f - fo).max() / np.abs(fo).max() < F_REL, call
        assert e == pytest.approx(eo, rel=E_REL), call


def test_noalloc_rejects_too_many_atoms(torch):
    pot = fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **fi.RGL_CU)
    d_pos = torch.zeros((32769, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fg.FireError) as e:
        fg.fire_energy_forces_noalloc(pot.c(), d_pos, [200.0] * 3, (1, 1, 1), None, None)
    assert e.value.status == fg.FIRE_ERR_ARG
    assert "32768" in str(e.value)
    assert ctypes.sizeof(fg.fire_potential_t) == 160
