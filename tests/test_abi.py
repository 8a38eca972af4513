"""The C-ABI library builds for sm_103a, loads, and exports every function the
public header declares.  No compute call is made (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import fire_inputs as fi
import paper_1908_02038_gb300 as fg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "fire2.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fire_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    fg.build()
    return fg.load_library()


def test_header_declares_expected_set():
    assert header_functions() == sorted(fg.EXPORTED)


def test_library_exports_every_header_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", fg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fire_[a-z_]+)$", out, flags=re.M))
    missing = set(header_functions()) - exported
    assert not missing, missing


def test_abi_version_and_defaults(lib):
    assert fg.fire_abi_version() == 9
    p = fg.fire_default_params(0.001)
    assert (p.tmax, p.tmin, p.dtgrow, p.dtshrink, p.alpha0, p.alphashrink) == \
        (10.0, 0.02, 1.1, 0.5, 0.25, 0.99)
    assert (p.delaystep, p.vdfmax, p.halfstepback, p.initialdelay, p.integrator, p.norm) == \
        (20, 2000, 1, 1, 0, 0)
    assert p.confirm64 == fg.FIRE_FP64_CHECK_FINISH
    with pytest.raises(fg.FireError) as e:
        fg.fire_default_params(0.0)
    assert e.value.status == fg.FIRE_ERR_ARG


def test_struct_layouts_match_header(lib):
    # sizes of the C structs as the header lays them out on LP64
    assert ctypes.sizeof(fg.fire_system_t) == 8 + 8 + 12 + 4
    assert ctypes.sizeof(fg.fire_potential_t) == 4 + 4 + 8 * 11 + 8 + 8 * 7
    assert ctypes.sizeof(fg.fire_params_t) == 7 * 8 + 8 * 4 + 8
    assert ctypes.sizeof(fg.fire_result_t) == 8 + 8 * 3 + 4 + 4 + 8 * 5


def test_init_rejects_bad_arguments_before_touching_the_gpu(lib):
    pot = fg.Potential(fg.FIRE_POT_LJ).c()
    par = fg.fire_default_params(0.005)
    sys = fg.fire_system_t(0, 1.0, (ctypes.c_int32 * 3)(1, 1, 1), 0)
    with pytest.raises(fg.FireError) as e:
        fg.fire_init(sys, pot, par)
    assert e.value.status == fg.FIRE_ERR_ARG and "n_atoms" in str(e.value)
    sys = fg.fire_system_t(10, -1.0, (ctypes.c_int32 * 3)(1, 1, 1), 0)
    with pytest.raises(fg.FireError):
        fg.fire_init(sys, pot, par)


def test_init_rejects_unknown_fp64_check_setting(lib):
    pot = fg.Potential(fg.FIRE_POT_RGL, precision=fg.FIRE_PREC_FP32_PAIR, **fi.RGL_CU).c()
    sys = fg.fire_system_t(10, 1.0, (ctypes.c_int32 * 3)(1, 1, 1), 0)
    par = fg.fire_default_params(0.001)
    par.confirm64 = 3
    with pytest.raises(fg.FireError) as e:
        fg.fire_init(sys, pot, par)
    assert e.value.status == fg.FIRE_ERR_ARG and "confirm64" in str(e.value)


def test_fp32pair_rejected_for_lj(lib):
    pot = fg.Potential(fg.FIRE_POT_LJ, precision=fg.FIRE_PREC_FP32_PAIR).c()
    sys = fg.fire_system_t(10, 1.0, (ctypes.c_int32 * 3)(1, 1, 1), 0)
    with pytest.raises(fg.FireError) as e:
        fg.fire_init(sys, pot, fg.fire_default_params(0.005))
    assert e.value.status == fg.FIRE_ERR_ARG and "FP32-pair" in str(e.value)


def test_batch_init_rejects_bad_offsets(lib):
    pot = fg.Potential(fg.FIRE_POT_RGL, A=0.0855, xi=1.224, p=10.96, q=2.278, r0=2.556,
                       rs=4.5, rc=5.0).c()
    sys = fg.fire_system_t(0, 1.0, (ctypes.c_int32 * 3)(1, 1, 1), 0)
    par = fg.fire_default_params(0.001)
    for off in ([1, 5], [0, 5, 5], [0]):
        with pytest.raises(fg.FireError) as e:
            fg.fire_batch_init(off, sys, pot, par)
        assert e.value.status == fg.FIRE_ERR_ARG
    lj = fg.Potential(fg.FIRE_POT_LJ).c()
    with pytest.raises(fg.FireError) as e:
        fg.fire_batch_init([0, 4], sys, lj, par)
    assert "RGL" in str(e.value)


def test_pair_function_table_matches_oracle(lib):
    """The quintic Hermite tables of the RGL pair functions (host copy of what
    the kernels use) against the oracle's analytic phi, g and derivatives."""
    import fire_inputs as fi
    import numpy as np
    import oracle
    pot = fg.Potential(fg.FIRE_POT_RGL, **fi.RGL_CU).c()
    r = np.concatenate([np.linspace(1.0, 4.999999, 200001),
                        [fi.RGL_CU["r0"], fi.RGL_CU["rs"], 4.5 + 1e-9, 4.5 - 1e-9]])
    tab = fg.fire_diag_rgl_table(pot, r)
    ref = oracle.rgl_pair_terms(oracle.Potential("rgl", **fi.RGL_CU), r)
    near = r > 2.0          # pairs no more compressed than ~0.8 r0
    for k in range(4):
        err = np.abs(tab[:, k] - ref[:, k])
        assert err.max() / np.abs(ref[:, k]).max() < 5e-11, k
        assert err[near].max() / np.abs(ref[near, k]).max() < 5e-12, k
    # beyond rc everything vanishes
    assert np.all(fg.fire_diag_rgl_table(pot, np.array([5.0, 6.0])) == 0.0)


def test_device_wrappers_reject_bad_shapes_on_the_host():
    """The *_dev wrappers check shapes and dtypes before any library call, so
    a flat 3N position tensor or a mis-shaped output never reaches a kernel
    (which would read or write past the tensors)."""
    import torch
    pot = fg.Potential(fg.FIRE_POT_RGL, **fi.RGL_CU).c()
    flat = torch.zeros(30, dtype=torch.float64)
    pos = torch.zeros((10, 3), dtype=torch.float64)
    box = [20.0] * 3
    cases = [
        (lambda: fg.fire_energy_forces_noalloc(pot, flat, box), "shape (n, 3)"),
        (lambda: fg.fire_energy_forces_noalloc(pot, pos, box, d_forces=torch.zeros(
            (9, 3), dtype=torch.float64)), "d_forces"),
        (lambda: fg.fire_energy_forces_noalloc(pot, pos, box, d_forces=torch.zeros(
            (10, 3), dtype=torch.float32)), "d_forces"),
        (lambda: fg.fire_energy_forces_noalloc(pot, pos, box, d_energy=torch.zeros(
            0, dtype=torch.float64)), "d_energy"),
        (lambda: fg.fire_energy_forces_dev(None, flat, box), "shape (n, 3)"),
        (lambda: fg.fire_minimize_dev(None, flat, box, 1e-6, 10), "shape (n, 3)"),
        (lambda: fg.fire_rgl_hvp_dev(None, pos, box, [1, 1, 1, 1], pos, flat), "d_hu"),
        (lambda: fg.fire_rgl_implicit_grad_dev(None, pos, box, [1, 1, 1, 1], flat), "d_g"),
        (lambda: fg.fire_energy_forces_noalloc(pot, pos, box), "CUDA"),
    ]
    for call, what in cases:
        with pytest.raises(ValueError) as e:
            call()
        assert what in str(e.value), (what, str(e.value))


def test_not_converged_status_is_named():
    assert fg.FIRE_ERR_NOT_CONVERGED == 8
    assert fg.STATUS_NAMES[8] == "FIRE_ERR_NOT_CONVERGED"
    txt = open(os.path.join(ROOT, "include", "fire2.h")).read()
    assert "FIRE_ERR_NOT_CONVERGED = 8" in txt
