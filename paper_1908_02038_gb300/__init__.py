"""Python binding of the GB300 FIRE 2.0 library (C ABI in include/fire2.h).

Argument marshalling only: every step of a relaxation runs in the CUDA
library ``_lib/libfire2gb300.so``.  The functions keep the C names
(``fire_init``, ``fire_minimize``, ``fire_minimize_dev``, ``fire_energy_forces``,
``fire_energy_forces_dev``, ...); ``FireHandle`` is a small owner object over
them.  Importing this package never falls back to another implementation:
if the library is missing or fails to load, the functions raise.

Host-pointer entry points take numpy float64 arrays; the ``*_dev`` entry points
take CUDA tensors (torch is used only for device memory and streams).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from ._build import LIB_PATH, build  # noqa: F401

FIRE_OK, FIRE_ERR_ARG, FIRE_ERR_CUDA, FIRE_ERR_NOMEM = 0, 1, 2, 3
FIRE_ERR_NONFINITE, FIRE_ERR_NBR_OVERFLOW, FIRE_ERR_TIMEOUT, FIRE_ERR_STATE = 4, 5, 6, 7
FIRE_ERR_NOT_CONVERGED = 8
FIRE_STOP_FTOL, FIRE_STOP_MAXITER, FIRE_STOP_MAXVDOTF = 0, 1, 2
FIRE_NORM_MAX_ATOM, FIRE_NORM_TWO, FIRE_NORM_INF = 0, 1, 2
FIRE_POT_LJ, FIRE_POT_RGL, FIRE_POT_SW = 0, 1, 2
FIRE_PREC_FP64, FIRE_PREC_FP32_PAIR = 0, 1
FIRE_PAIR_TABLE, FIRE_PAIR_ANALYTIC = 0, 1
FIRE_NEWTON_AUTO, FIRE_NEWTON_ON, FIRE_NEWTON_OFF = 0, 1, 2
FIRE_INT_EULER_IMPLICIT, FIRE_INT_EULER_EXPLICIT, FIRE_INT_VERLET, FIRE_INT_LEAPFROG = 0, 1, 2, 3
FIRE_VARIANT_FIRE2, FIRE_VARIANT_FIRE1 = 0, 1
FIRE_FP64_CHECK_OFF, FIRE_FP64_CHECK_CONFIRM, FIRE_FP64_CHECK_FINISH = 0, 1, 2

STATUS_NAMES = {0: "FIRE_OK", 1: "FIRE_ERR_ARG", 2: "FIRE_ERR_CUDA", 3: "FIRE_ERR_NOMEM",
                4: "FIRE_ERR_NONFINITE", 5: "FIRE_ERR_NBR_OVERFLOW", 6: "FIRE_ERR_TIMEOUT",
                7: "FIRE_ERR_STATE", 8: "FIRE_ERR_NOT_CONVERGED"}

# Every symbol include/fire2.h declares (checked by the ABI test).
EXPORTED = ("fire_abi_version", "fire_default_params", "fire_init", "fire_minimize",
            "fire_minimize_dev", "fire_energy_forces", "fire_energy_forces_dev",
            "fire_set_pair_tiles",
            "fire_set_time_budget", "fire_profile_stages", "fire_diag_fma_peak",
            "fire_energy_forces_noalloc", "fire_set_exec_mode", "fire_set_threads_per_atom",
            "fire_diag_exp",
            "fire_batch_init", "fire_minimize_batch", "fire_minimize_batch_dev",
            "fire_batch_set_tuning", "fire_batch_autotune", "fire_set_rgl_params",
            "fire_rgl_energy_grad_dev", "fire_rgl_hvp_dev", "fire_rgl_implicit_grad_dev",
            "fire_diag_rgl_table", "fire_set_dof_mask", "fire_neb_init", "fire_neb_minimize",
            "fire_neb_minimize_dev", "fire_last_error", "fire_destroy")
FIRE_EXEC_GRAPH_WHILE, FIRE_EXEC_CHUNKED = 0, 1
FIRE_TILES_AUTO, FIRE_TILES_ON, FIRE_TILES_OFF = 0, 1, 2
STAGES = ("build", "density", "embed", "force", "reduce", "control", "update")


class fire_system_t(C.Structure):
    _fields_ = [("n_atoms", C.c_int64), ("mass", C.c_double), ("periodic", C.c_int32 * 3),
                ("reserved", C.c_int32)]


class fire_potential_t(C.Structure):
    _fields_ = [("kind", C.c_int32), ("precision", C.c_int32),
                ("eps", C.c_double), ("sigma", C.c_double), ("rc_lj", C.c_double),
                ("A", C.c_double), ("xi", C.c_double), ("p", C.c_double), ("q", C.c_double),
                ("r0", C.c_double), ("rs", C.c_double), ("rc", C.c_double),
                ("skin", C.c_double), ("pair_eval", C.c_int32), ("newton", C.c_int32),
                ("sw_A", C.c_double), ("sw_B", C.c_double), ("sw_p", C.c_double),
                ("sw_q", C.c_double), ("sw_a", C.c_double), ("sw_lambda", C.c_double),
                ("sw_gamma", C.c_double)]


class fire_params_t(C.Structure):
    _fields_ = [("dt_start", C.c_double), ("tmax", C.c_double), ("tmin", C.c_double),
                ("dtgrow", C.c_double), ("dtshrink", C.c_double), ("alpha0", C.c_double),
                ("alphashrink", C.c_double), ("delaystep", C.c_int32), ("vdfmax", C.c_int32),
                ("halfstepback", C.c_int32), ("initialdelay", C.c_int32),
                ("integrator", C.c_int32), ("norm", C.c_int32), ("variant", C.c_int32),
                ("confirm64", C.c_int32), ("dmax", C.c_double)]


class fire_batch_tuning_t(C.Structure):
    _fields_ = [("threads_per_block", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("cluster_size", C.c_int32), ("reserved", C.c_int32)]


class fire_result_t(C.Structure):
    _fields_ = [("energy", C.c_double), ("iterations", C.c_int64), ("force_evals", C.c_int64),
                ("nbr_builds", C.c_int64), ("stop", C.c_int32), ("reserved", C.c_int32),
                ("fmax_atom", C.c_double), ("f2norm", C.c_double), ("finf", C.c_double),
                ("dt_final", C.c_double), ("alpha_final", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


_lib = None


def load_library(path: str | None = None):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"FIRE CUDA library not built ({path}); run "
                           "paper_1908_02038_gb300.build() first")
    lib = C.CDLL(path)
    H = C.c_void_p
    lib.fire_abi_version.restype = C.c_int32
    lib.fire_default_params.argtypes = [C.POINTER(fire_params_t), C.c_double]
    lib.fire_init.argtypes = [C.POINTER(H), C.POINTER(fire_system_t), C.POINTER(fire_potential_t),
                              C.POINTER(fire_params_t)]
    lib.fire_minimize.argtypes = [H, C.c_void_p, C.POINTER(C.c_double), C.c_double, C.c_int64,
                                  C.POINTER(fire_result_t)]
    lib.fire_minimize_dev.argtypes = [H, C.c_void_p, C.POINTER(C.c_double), C.c_double,
                                      C.c_int64, C.POINTER(fire_result_t), C.c_void_p]
    lib.fire_energy_forces.argtypes = [H, C.c_void_p, C.POINTER(C.c_double), C.c_void_p,
                                       C.POINTER(C.c_double)]
    lib.fire_energy_forces_dev.argtypes = [H, C.c_void_p, C.POINTER(C.c_double), C.c_void_p,
                                           C.c_void_p, C.c_void_p]
    lib.fire_set_time_budget.argtypes = [H, C.c_double]
    lib.fire_set_exec_mode.argtypes = [H, C.c_int32, C.c_int32]
    lib.fire_set_threads_per_atom.argtypes = [H, C.c_int32, C.POINTER(C.c_int32)]
    lib.fire_set_pair_tiles.argtypes = [H, C.c_int32, C.c_int32]
    lib.fire_set_dof_mask.argtypes = [H, C.c_void_p]
    lib.fire_neb_init.argtypes = [C.POINTER(H), C.c_int32, C.POINTER(fire_system_t),
                                  C.POINTER(fire_potential_t), C.POINTER(fire_params_t),
                                  C.c_double, C.c_int32]
    lib.fire_neb_minimize.argtypes = [H, C.c_void_p, C.POINTER(C.c_double), C.c_double, C.c_int64,
                                      C.POINTER(fire_result_t), C.c_void_p,
                                      C.POINTER(C.c_int32)]
    lib.fire_neb_minimize_dev.argtypes = [H, C.c_void_p, C.POINTER(C.c_double), C.c_double,
                                          C.c_int64, C.POINTER(fire_result_t), C.c_void_p,
                                          C.POINTER(C.c_int32), C.c_void_p]
    lib.fire_diag_exp.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.fire_batch_init.argtypes = [C.POINTER(H), C.c_int32, C.c_void_p, C.POINTER(fire_system_t),
                                    C.POINTER(fire_potential_t), C.POINTER(fire_params_t)]
    lib.fire_minimize_batch.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.c_int64,
                                        C.c_void_p, C.c_void_p]
    lib.fire_minimize_batch_dev.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.c_int64,
                                            C.c_void_p, C.c_void_p, C.c_void_p]
    lib.fire_batch_set_tuning.argtypes = [H, C.POINTER(fire_batch_tuning_t)]
    D4 = C.POINTER(C.c_double)
    lib.fire_set_rgl_params.argtypes = [H, D4]
    lib.fire_diag_rgl_table.argtypes = [C.POINTER(fire_potential_t), C.c_int64, C.c_void_p,
                                        C.c_void_p]
    lib.fire_rgl_energy_grad_dev.argtypes = [H, C.c_void_p, D4, D4, C.c_void_p, D4, D4, C.c_void_p]
    lib.fire_rgl_hvp_dev.argtypes = [H, C.c_void_p, D4, D4, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.fire_rgl_implicit_grad_dev.argtypes = [H, C.c_void_p, D4, D4, C.c_void_p, C.c_double,
                                               C.c_int64, D4, C.c_void_p,
                                               C.POINTER(C.c_int64), C.c_void_p]
    lib.fire_batch_autotune.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int32,
                                        C.POINTER(fire_batch_tuning_t)]
    lib.fire_profile_stages.argtypes = [H, C.c_void_p, C.POINTER(C.c_double), C.c_int32,
                                        C.POINTER(C.c_double)]
    lib.fire_diag_fma_peak.argtypes = [C.c_int32, C.POINTER(C.c_double)]
    lib.fire_energy_forces_noalloc.argtypes = [C.POINTER(fire_potential_t), C.c_int64,
                                               C.POINTER(C.c_int32), C.c_void_p,
                                               C.POINTER(C.c_double), C.c_void_p, C.c_void_p,
                                               C.c_void_p]
    lib.fire_last_error.restype = C.c_char_p
    lib.fire_last_error.argtypes = [H]
    lib.fire_destroy.argtypes = [H]
    lib.fire_destroy.restype = None
    for name in EXPORTED:
        if name not in ("fire_last_error", "fire_destroy", "fire_abi_version"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class FireError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, handle) -> None:
    if status != FIRE_OK:
        raise FireError(status, fire_last_error(handle))


def _box(box):
    b = (C.c_double * 3)(*[float(v) for v in box])
    return b


# --- same-name wrappers ------------------------------------------------------

def fire_abi_version() -> int:
    return int(load_library().fire_abi_version())


def fire_default_params(dt_start: float) -> fire_params_t:
    p = fire_params_t()
    _check(load_library().fire_default_params(C.byref(p), float(dt_start)), None)
    return p


def fire_init(sys: fire_system_t, pot: fire_potential_t, params: fire_params_t):
    h = C.c_void_p()
    st = load_library().fire_init(C.byref(h), C.byref(sys), C.byref(pot), C.byref(params))
    _check(st, None)
    return h


def fire_last_error(handle) -> str:
    msg = load_library().fire_last_error(handle)
    return msg.decode() if msg else ""


def fire_destroy(handle) -> None:
    if handle:
        load_library().fire_destroy(handle)


def fire_set_time_budget(handle, seconds: float) -> None:
    _check(load_library().fire_set_time_budget(handle, float(seconds)), handle)


def fire_set_dof_mask(handle, mask) -> None:
    """Frozen degrees of freedom of later relaxations: one uint8 per atom,
    bit d set = component d frozen; None frees them all."""
    if mask is None:
        _check(load_library().fire_set_dof_mask(handle, None), handle)
        return
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    _check(load_library().fire_set_dof_mask(handle, m.ctypes.data_as(C.c_void_p)), handle)


def fire_set_exec_mode(handle, mode: int, chunk: int | None = None) -> None:
    """chunk: iterations per graph launch (chunked mode, default 32) or per
    WHILE-body launch (graph mode, default 0 = automatic)."""
    if chunk is None:
        chunk = 32 if mode == FIRE_EXEC_CHUNKED else 0
    _check(load_library().fire_set_exec_mode(handle, int(mode), int(chunk)), handle)


def fire_set_threads_per_atom(handle, tpa: int = 0) -> int:
    """Threads per atom of the splitting RGL pair passes (0 = automatic);
    returns the value in effect."""
    out = C.c_int32(0)
    _check(load_library().fire_set_threads_per_atom(handle, int(tpa), C.byref(out)), handle)
    return out.value


def fire_set_pair_tiles(handle, mode: int = FIRE_TILES_AUTO, stage_cap: int = 0) -> None:
    """Shared-memory tiles of the FP64 half-list passes: FIRE_TILES_AUTO,
    FIRE_TILES_ON or FIRE_TILES_OFF; stage_cap 0 = the largest stage."""
    _check(load_library().fire_set_pair_tiles(handle, int(mode), int(stage_cap)), handle)


def fire_minimize(handle, pos: np.ndarray, box, ftol: float, maxiter: int) -> fire_result_t:
    """Relaxes pos (float64, N x 3, C-contiguous) in place."""
    if pos.dtype != np.float64 or not pos.flags.c_contiguous:
        raise ValueError("pos must be a C-contiguous float64 array")
    res = fire_result_t()
    st = load_library().fire_minimize(handle, pos.ctypes.data, _box(box), float(ftol),
                                      int(maxiter), C.byref(res))
    _check(st, handle)
    return res


def fire_minimize_dev(handle, d_pos, box, ftol: float, maxiter: int, stream=None) -> fire_result_t:
    """d_pos: CUDA float64 tensor (N x 3, contiguous), relaxed in place."""
    _check_dev(d_pos, "d_pos", rows3=True)
    res = fire_result_t()
    st = load_library().fire_minimize_dev(handle, d_pos.data_ptr(), _box(box), float(ftol),
                                          int(maxiter), C.byref(res), _stream(stream))
    _check(st, handle)
    return res


def fire_energy_forces(handle, pos: np.ndarray, box, want_forces: bool = True):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    f = np.empty_like(pos) if want_forces else None
    e = C.c_double(0.0)
    st = load_library().fire_energy_forces(handle, pos.ctypes.data, _box(box),
                                           f.ctypes.data if f is not None else None, C.byref(e))
    _check(st, handle)
    return float(e.value), f


def fire_energy_forces_dev(handle, d_pos, box, d_forces=None, d_energy=None, stream=None):
    _check_outputs(d_pos, d_forces, d_energy)
    st = load_library().fire_energy_forces_dev(
        handle, d_pos.data_ptr(), _box(box),
        d_forces.data_ptr() if d_forces is not None else None,
        d_energy.data_ptr() if d_energy is not None else None, _stream(stream))
    _check(st, handle)


def fire_profile_stages(handle, pos: np.ndarray, box, reps: int = 10) -> dict:
    """Mean device milliseconds per stage of one iteration (diagnostic)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = (C.c_double * len(STAGES))()
    _check(load_library().fire_profile_stages(handle, pos.ctypes.data, _box(box), int(reps), out),
           handle)
    return dict(zip(STAGES, list(out)))


def fire_diag_fma_peak(which: int) -> float:
    """Measured FMA issue rate in flop/s (which: 0 = FP64, 1 = FP32)."""
    v = C.c_double(0.0)
    _check(load_library().fire_diag_fma_peak(int(which), C.byref(v)), None)
    return float(v.value)


def fire_energy_forces_noalloc(pot: fire_potential_t, d_pos, box, periodic=(1, 1, 1),
                               d_forces=None, d_energy=None, stream=None) -> None:
    """Allocation-free evaluation into caller-owned CUDA tensors (enqueued on
    `stream`; synchronise before reading the results)."""
    _check_outputs(d_pos, d_forces, d_energy)
    per = (C.c_int32 * 3)(*[int(bool(p)) for p in periodic])
    st = load_library().fire_energy_forces_noalloc(
        C.byref(pot), int(d_pos.shape[0]), per, d_pos.data_ptr(), _box(box),
        d_forces.data_ptr() if d_forces is not None else None,
        d_energy.data_ptr() if d_energy is not None else None, _stream(stream))
    _check(st, None)


def fire_diag_exp(d_x, d_out, stream=None) -> None:
    """The library's FP64 exponential at the points of d_x (CUDA float64)."""
    _check_dev(d_x, "d_x")
    _check_dev(d_out, "d_out", like=d_x)
    _check(load_library().fire_diag_exp(int(d_x.numel()), d_x.data_ptr(), d_out.data_ptr(),
                                        _stream(stream)), None)


def fire_batch_init(offsets, sys: fire_system_t, pot: fire_potential_t, params: fire_params_t):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    h = C.c_void_p()
    st = load_library().fire_batch_init(C.byref(h), int(len(off) - 1), off.ctypes.data,
                                        C.byref(sys), C.byref(pot), C.byref(params))
    _check(st, None)
    return h


def fire_minimize_batch(handle, pos: np.ndarray, boxes, ftol: float, maxiter: int,
                        want_forces: bool = False):
    """Relaxes the packed positions in place; returns (results, forces or None)."""
    if pos.dtype != np.float64 or not pos.flags.c_contiguous:
        raise ValueError("pos must be a C-contiguous float64 array")
    bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
    out = (fire_result_t * len(bx))()
    f = np.empty_like(pos) if want_forces else None
    st = load_library().fire_minimize_batch(handle, pos.ctypes.data, bx.ctypes.data, float(ftol),
                                            int(maxiter), C.cast(out, C.c_void_p),
                                            f.ctypes.data if f is not None else None)
    _check(st, handle)
    return list(out), f


def fire_minimize_batch_dev(handle, d_pos, boxes, ftol: float, maxiter: int, d_forces=None,
                            stream=None):
    _check_dev(d_pos, "d_pos", rows3=True)
    if d_forces is not None:
        _check_dev(d_forces, "d_forces", like=d_pos)
    bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
    out = (fire_result_t * len(bx))()
    st = load_library().fire_minimize_batch_dev(
        handle, d_pos.data_ptr(), bx.ctypes.data, float(ftol), int(maxiter),
        C.cast(out, C.c_void_p), d_forces.data_ptr() if d_forces is not None else None,
        _stream(stream))
    _check(st, handle)
    return list(out)


def fire_batch_set_tuning(handle, threads_per_block: int, ctas_per_sm: int,
                          cluster_size: int = 1) -> None:
    t = fire_batch_tuning_t(int(threads_per_block), int(ctas_per_sm), int(cluster_size), 0)
    _check(load_library().fire_batch_set_tuning(handle, C.byref(t)), handle)


def fire_batch_autotune(handle, pos: np.ndarray, boxes, iters: int = 20):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
    t = fire_batch_tuning_t()
    _check(load_library().fire_batch_autotune(handle, pos.ctypes.data, bx.ctypes.data,
                                              int(iters), C.byref(t)), handle)
    return {"threads_per_block": t.threads_per_block, "ctas_per_sm": t.ctas_per_sm,
            "cluster_size": max(1, t.cluster_size)}


def _theta(theta):
    return (C.c_double * 4)(*[float(v) for v in theta])


def fire_set_rgl_params(handle, theta) -> None:
    _check(load_library().fire_set_rgl_params(handle, _theta(theta)), handle)


def fire_rgl_energy_grad_dev(handle, d_pos, box, theta, d_forces=None, stream=None):
    """Returns (E, dE/dtheta as a numpy (4,)); fills d_forces if given."""
    _check_outputs(d_pos, d_forces, None)
    e = C.c_double(0.0)
    de = (C.c_double * 4)()
    st = load_library().fire_rgl_energy_grad_dev(
        handle, d_pos.data_ptr(), _box(box), _theta(theta),
        d_forces.data_ptr() if d_forces is not None else None, C.byref(e), de, _stream(stream))
    _check(st, handle)
    return float(e.value), np.array(list(de))


def fire_rgl_hvp_dev(handle, d_pos, box, theta, d_u, d_hu, stream=None) -> None:
    for cuda in (False, True):
        _check_dev(d_pos, "d_pos", rows3=True, cuda=cuda)
        _check_dev(d_u, "d_u", like=d_pos, cuda=cuda)
        _check_dev(d_hu, "d_hu", like=d_pos, cuda=cuda)
    st = load_library().fire_rgl_hvp_dev(handle, d_pos.data_ptr(), _box(box), _theta(theta),
                                         d_u.data_ptr(), d_hu.data_ptr(), _stream(stream))
    _check(st, handle)


def fire_rgl_implicit_grad_dev(handle, d_pos, box, theta, d_g, tol=1e-10, maxit=20000,
                               d_lambda=None, stream=None):
    """Returns (dL/dtheta as numpy (4,), CG iterations).  Raises FireError
    with status FIRE_ERR_NOT_CONVERGED when CG stopped before tol (maxit
    reached, or a breakdown away from a minimum)."""
    for cuda in (False, True):
        _check_dev(d_pos, "d_pos", rows3=True, cuda=cuda)
        _check_dev(d_g, "d_g", like=d_pos, cuda=cuda)
        if d_lambda is not None:
            _check_dev(d_lambda, "d_lambda", like=d_pos, cuda=cuda)
    out = (C.c_double * 4)()
    it = C.c_int64(0)
    st = load_library().fire_rgl_implicit_grad_dev(
        handle, d_pos.data_ptr(), _box(box), _theta(theta), d_g.data_ptr(), float(tol),
        int(maxit), out, d_lambda.data_ptr() if d_lambda is not None else None, C.byref(it),
        _stream(stream))
    _check(st, handle)
    return np.array(list(out)), int(it.value)


def fire_diag_rgl_table(pot: fire_potential_t, r) -> np.ndarray:
    """Host evaluation of the pair-function table: (n, 4) = phi, g, phi', g'."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros((len(r), 4))
    _check(load_library().fire_diag_rgl_table(C.byref(pot), len(r), r.ctypes.data,
                                              out.ctypes.data), None)
    return out


def _check_dev(t, name="tensor", rows3=False, like=None, min_numel=1, cuda=True):
    """Raises ValueError unless t is a contiguous float64 CUDA tensor; with
    rows3 it must be shaped (n, 3); with like, it must have like's shape and
    device; it must hold at least min_numel elements.  The checks that need
    no GPU come first (cuda=False: only those)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float64 tensor")
    if rows3 and (t.dim() != 2 or t.shape[1] != 3):
        raise ValueError(f"{name}: expected shape (n, 3), got {tuple(t.shape)}")
    if like is not None and t.shape != like.shape:
        raise ValueError(f"{name}: expected shape {tuple(like.shape)}, got {tuple(t.shape)}")
    if t.numel() < min_numel:
        raise ValueError(f"{name}: expected at least {min_numel} element(s)")
    if not cuda:
        return
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if like is not None and t.device != like.device:
        raise ValueError(f"{name}: on {t.device}, expected {like.device}")


def _check_outputs(d_pos, d_forces, d_energy):
    """Positions (n, 3); forces, if given, shaped like them on the same
    device; energy, if given, one double or more on the same device."""
    for cuda in (False, True):   # every layout check before the device checks
        _check_dev(d_pos, "d_pos", rows3=True, cuda=cuda)
        if d_forces is not None:
            _check_dev(d_forces, "d_forces", like=d_pos, cuda=cuda)
        if d_energy is not None:
            _check_dev(d_energy, "d_energy", cuda=cuda)
    if d_energy is not None and d_energy.device != d_pos.device:
        raise ValueError(f"d_energy: on {d_energy.device}, expected {d_pos.device}")


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# --- owner object ------------------------------------------------------------

@dataclass
class Potential:
    kind: int
    precision: int = FIRE_PREC_FP64
    eps: float = 1.0
    sigma: float = 1.0
    rc_lj: float = 2.5
    A: float = 0.0
    xi: float = 0.0
    p: float = 0.0
    q: float = 0.0
    r0: float = 1.0
    rs: float = 0.0
    rc: float = 0.0
    skin: float = 0.3
    pair_eval: int = FIRE_PAIR_TABLE
    newton: int = FIRE_NEWTON_AUTO
    sw_A: float = 0.0
    sw_B: float = 0.0
    sw_p: float = 0.0
    sw_q: float = 0.0
    sw_a: float = 0.0
    sw_lambda: float = 0.0
    sw_gamma: float = 0.0

    def c(self) -> fire_potential_t:
        return fire_potential_t(self.kind, self.precision, self.eps, self.sigma, self.rc_lj,
                                self.A, self.xi, self.p, self.q, self.r0, self.rs, self.rc,
                                self.skin, self.pair_eval, self.newton, self.sw_A, self.sw_B,
                                self.sw_p, self.sw_q, self.sw_a, self.sw_lambda, self.sw_gamma)


class FireBatch:
    """Owns one batched fire_handle_t (fire_batch_init)."""

    def __init__(self, counts, mass: float, pot: Potential, params=None, periodic=(1, 1, 1),
                 dt_start: float | None = None, **param_overrides):
        if params is None:
            params = fire_default_params(dt_start)
        for k, v in param_overrides.items():
            setattr(params, k, int(v) if isinstance(getattr(params, k), int) else float(v))
        self.offsets = np.concatenate([[0], np.cumsum(np.asarray(counts, dtype=np.int64))])
        sys = fire_system_t(int(self.offsets[-1]), float(mass), (C.c_int32 * 3)(*periodic), 0)
        self.h = fire_batch_init(self.offsets, sys, pot.c(), params)

    def minimize(self, pos, boxes, ftol, maxiter, want_forces=False):
        return fire_minimize_batch(self.h, pos, boxes, ftol, maxiter, want_forces)

    def minimize_dev(self, d_pos, boxes, ftol, maxiter, d_forces=None, stream=None):
        return fire_minimize_batch_dev(self.h, d_pos, boxes, ftol, maxiter, d_forces, stream)

    def set_tuning(self, threads_per_block, ctas_per_sm, cluster_size=1):
        fire_batch_set_tuning(self.h, threads_per_block, ctas_per_sm, cluster_size)

    def autotune(self, pos, boxes, iters=20):
        return fire_batch_autotune(self.h, pos, boxes, iters)

    def set_time_budget(self, seconds):
        fire_set_time_budget(self.h, seconds)

    def close(self):
        if getattr(self, "h", None):
            fire_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FireHandle:
    """Owns one fire_handle_t; closes it on exit / garbage collection."""

    def __init__(self, n_atoms: int, mass: float, pot: Potential, params=None,
                 periodic=(1, 1, 1), dt_start: float | None = None, **param_overrides):
        if params is None:
            params = fire_default_params(dt_start)
        for k, v in param_overrides.items():
            setattr(params, k, int(v) if isinstance(getattr(params, k), int) else float(v))
        sys = fire_system_t(int(n_atoms), float(mass), (C.c_int32 * 3)(*periodic), 0)
        self.n = int(n_atoms)
        self.h = fire_init(sys, pot.c(), params)

    def minimize(self, pos, box, ftol, maxiter):
        return fire_minimize(self.h, pos, box, ftol, maxiter)

    def minimize_dev(self, d_pos, box, ftol, maxiter, stream=None):
        return fire_minimize_dev(self.h, d_pos, box, ftol, maxiter, stream)

    def energy_forces(self, pos, box, want_forces=True):
        return fire_energy_forces(self.h, pos, box, want_forces)

    def profile_stages(self, pos, box, reps=10):
        return fire_profile_stages(self.h, pos, box, reps)

    def set_rgl_params(self, theta):
        fire_set_rgl_params(self.h, theta)

    def set_exec_mode(self, mode, chunk=None):
        fire_set_exec_mode(self.h, mode, chunk)

    def set_threads_per_atom(self, tpa=0):
        return fire_set_threads_per_atom(self.h, tpa)

    def set_pair_tiles(self, mode=FIRE_TILES_AUTO, stage_cap=0):
        fire_set_pair_tiles(self.h, mode, stage_cap)

    def set_time_budget(self, seconds):
        fire_set_time_budget(self.h, seconds)

    def set_dof_mask(self, mask):
        if mask is not None and np.asarray(mask).shape != (self.n,):
            raise ValueError("the mask holds one byte per atom")
        fire_set_dof_mask(self.h, mask)

    def close(self):
        if getattr(self, "h", None):
            fire_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FireNEB:
    """Nudged elastic band handle (fire_neb_init): n_img movable images of a
    system of n_atoms atoms, relaxed together with FIRE 2.0."""

    def __init__(self, n_img: int, n_atoms: int, mass: float, pot: Potential, k_spring: float,
                 climb: bool = True, params=None, periodic=(1, 1, 1),
                 dt_start: float | None = None, **param_overrides):
        if params is None:
            params = fire_default_params(dt_start)
        for k, v in param_overrides.items():
            setattr(params, k, int(v) if isinstance(getattr(params, k), int) else float(v))
        sys = fire_system_t(int(n_atoms), float(mass), (C.c_int32 * 3)(*periodic), 0)
        self.n_img, self.n = int(n_img), int(n_atoms)
        h = C.c_void_p()
        st = load_library().fire_neb_init(C.byref(h), int(n_img), C.byref(sys), C.byref(pot.c()),
                                          C.byref(params), float(k_spring), int(bool(climb)))
        _check(st, None)
        self.h = h

    def _shape_ok(self, path):
        if tuple(path.shape) != (self.n_img + 2, self.n, 3):
            raise ValueError(f"path must be ({self.n_img + 2}, {self.n}, 3)")

    def minimize(self, path, box, ftol, maxiter):
        """path: float64 (n_img + 2, n_atoms, 3), relaxed in place; returns
        (result, energies (n_img + 2), climbing-image index or 0)."""
        if not (isinstance(path, np.ndarray) and path.dtype == np.float64
                and path.flags.c_contiguous):
            raise ValueError("path must be a C-contiguous float64 array")
        self._shape_ok(path)
        out, E, cl = fire_result_t(), np.zeros(self.n_img + 2), C.c_int32(0)
        _check(load_library().fire_neb_minimize(self.h, path.ctypes.data, _box(box), float(ftol),
                                                int(maxiter), C.byref(out), E.ctypes.data,
                                                C.byref(cl)), self.h)
        return out, E, int(cl.value)

    def minimize_dev(self, d_path, box, ftol, maxiter, stream=None):
        """d_path: CUDA float64 tensor (n_img + 2, n_atoms, 3), relaxed in place."""
        _check_dev(d_path)
        self._shape_ok(d_path)
        out, E, cl = fire_result_t(), np.zeros(self.n_img + 2), C.c_int32(0)
        _check(load_library().fire_neb_minimize_dev(self.h, d_path.data_ptr(), _box(box),
                                                    float(ftol), int(maxiter), C.byref(out),
                                                    E.ctypes.data, C.byref(cl),
                                                    _stream(stream)), self.h)
        return out, E, int(cl.value)

    def set_dof_mask(self, mask):
        if mask is not None and np.asarray(mask).shape != (self.n,):
            raise ValueError("the mask holds one byte per atom of an image")
        fire_set_dof_mask(self.h, mask)

    def set_exec_mode(self, mode, chunk=None):
        fire_set_exec_mode(self.h, mode, chunk)

    def set_threads_per_atom(self, tpa=0):
        return fire_set_threads_per_atom(self.h, tpa)

    def close(self):
        if getattr(self, "h", None):
            fire_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
