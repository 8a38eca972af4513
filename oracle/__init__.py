"""FIRE 2.0 reference oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU implementation (``fire_oracle.c``) of the energy/force
evaluation and of the FIRE 2.0 relaxation loop (Algorithm 2 with the
semi-implicit Euler integrator of Algorithm 4).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with the CUDA library and never imports it.

Parity status: ``energy_forces`` and ``fire2`` are pinned by the tests in
``tests/test_oracle_pins.py`` (finite differences, sum F = 0, zero force on a
perfect lattice, closed-form cohesive energies, hand-traced FIRE iterations,
the LJ dimer bond length); ``rgl_param_derivs``, ``rgl_hvp``, ``rgl_cg`` and
``implicit_grad`` by ``tests/test_oracle_derivs.py`` (central differences in
theta and x, Hessian symmetry and translation modes, finite differences of
full relaxations).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fire_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfire_oracle.so")

POT_LJ, POT_RGL, POT_QUAD, POT_DWELL, POT_SW = 0, 1, 2, 3, 4
FORCE_BRUTE, FORCE_CELLS = 0, 1
STOP_FTOL, STOP_MAXITER, STOP_MAXVDOTF = 0, 1, 2
NORM_MAX_ATOM, NORM_TWO, NORM_INF = 0, 1, 2
INT_EULER_IMPLICIT, INT_EULER_EXPLICIT, INT_VERLET, INT_LEAPFROG = 0, 1, 2, 3
VAR_FIRE2, VAR_FIRE1 = 0, 1


class _Sys(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double * 3), ("periodic", C.c_int32 * 3),
                ("mass", C.c_double)]


class _Pot(C.Structure):
    _fields_ = [("kind", C.c_int32),
                ("eps", C.c_double), ("sigma", C.c_double), ("rc_lj", C.c_double),
                ("A", C.c_double), ("xi", C.c_double), ("p", C.c_double), ("q", C.c_double),
                ("r0", C.c_double), ("rs", C.c_double), ("rc", C.c_double),
                ("quad_k", C.POINTER(C.c_double)), ("quad_x0", C.POINTER(C.c_double)),
                ("dwell", C.POINTER(C.c_double)),
                ("sw_A", C.c_double), ("sw_B", C.c_double), ("sw_p", C.c_double),
                ("sw_q", C.c_double), ("sw_a", C.c_double), ("sw_lambda", C.c_double),
                ("sw_gamma", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("dt_start", C.c_double), ("tmax", C.c_double), ("tmin", C.c_double),
                ("dtgrow", C.c_double), ("dtshrink", C.c_double), ("alpha0", C.c_double),
                ("alphashrink", C.c_double), ("delaystep", C.c_int32), ("vdfmax", C.c_int32),
                ("halfstepback", C.c_int32), ("initialdelay", C.c_int32),
                ("integrator", C.c_int32), ("norm", C.c_int32), ("variant", C.c_int32),
                ("pad", C.c_int32), ("dmax", C.c_double), ("frozen", C.c_void_p)]


class _Result(C.Structure):
    _fields_ = [("energy", C.c_double), ("iterations", C.c_int64), ("force_evals", C.c_int64),
                ("stop", C.c_int32), ("pad", C.c_int32), ("fmax_atom", C.c_double),
                ("f2norm", C.c_double), ("finf", C.c_double), ("dt_final", C.c_double),
                ("alpha_final", C.c_double)]


class _Trace(C.Structure):
    _fields_ = [("i", C.c_int64), ("npos", C.c_int64), ("nneg", C.c_int64),
                ("P", C.c_double), ("dt", C.c_double), ("alpha", C.c_double),
                ("energy", C.c_double), ("fnorm", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.ora_energy_forces.restype = C.c_int
        lib.ora_energy_forces.argtypes = [C.POINTER(_Sys), C.POINTER(_Pot), C.c_void_p,
                                          C.c_void_p, C.POINTER(C.c_double), C.c_int]
        lib.ora_energy_forces_subset.restype = C.c_int
        lib.ora_energy_forces_subset.argtypes = [C.POINTER(_Sys), C.POINTER(_Pot), C.c_void_p,
                                                 C.c_void_p, C.c_int64, C.c_void_p,
                                                 C.POINTER(C.c_double), C.c_int]
        lib.ora_densities.restype = C.c_int
        lib.ora_densities.argtypes = [C.POINTER(_Sys), C.POINTER(_Pot), C.c_void_p, C.c_void_p]
        lib.ora_neb.restype = C.c_int
        lib.ora_neb.argtypes = [C.POINTER(_Sys), C.POINTER(_Pot), C.POINTER(_Params), C.c_int64,
                                C.c_void_p, C.c_double, C.c_int, C.c_double, C.c_int64, C.c_int,
                                C.POINTER(_Result), C.c_void_p, C.POINTER(C.c_int64)]
        lib.ora_fire2.restype = C.c_int
        lib.ora_fire2.argtypes = [C.POINTER(_Sys), C.POINTER(_Pot), C.POINTER(_Params), C.c_void_p,
                                  C.c_double, C.c_int64, C.c_int, C.POINTER(_Result),
                                  C.c_void_p, C.c_int64]
        lib.ora_rgl_param_derivs.restype = C.c_int
        lib.ora_rgl_param_derivs.argtypes = [C.POINTER(_Sys), C.POINTER(_Pot), C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_int]
        lib.ora_rgl_hvp.restype = C.c_int
        lib.ora_rgl_hvp.argtypes = [C.POINTER(_Sys), C.POINTER(_Pot), C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int]
        lib.ora_rgl_cg.restype = C.c_int64
        lib.ora_rgl_cg.argtypes = [C.POINTER(_Sys), C.POINTER(_Pot), C.c_void_p, C.c_void_p,
                                   C.c_double, C.c_int64, C.c_void_p, C.c_int]
        lib.ora_rgl_pair_terms.restype = C.c_int
        lib.ora_rgl_pair_terms.argtypes = [C.POINTER(_Pot), C.c_int64, C.c_void_p, C.c_void_p]
        lib.ora_set_threads.argtypes = [C.c_int]
        lib.ora_max_threads.restype = C.c_int
        _lib = lib
    return _lib


def set_threads(k: int) -> None:
    _load().ora_set_threads(int(k))


def max_threads() -> int:
    return int(_load().ora_max_threads())


@dataclass
class Potential:
    """Potential description.  kind: 'lj', 'rgl', 'sw' (Stillinger-Weber with
    eps, sigma and the sw_* fields), 'quad' (test well) or 'dwell' (double-well
    test surface, dwell = (h, a, c, ky, kz))."""
    kind: str
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
    quad_k: np.ndarray | None = None
    quad_x0: np.ndarray | None = None
    dwell: tuple | None = None
    sw_A: float = 0.0
    sw_B: float = 0.0
    sw_p: float = 0.0
    sw_q: float = 0.0
    sw_a: float = 0.0
    sw_lambda: float = 0.0
    sw_gamma: float = 0.0


@dataclass
class Params:
    """FIRE 2.0 parameters, Table 1 names and defaults (dt_start is the MD timestep)."""
    dt_start: float
    tmax: float = 10.0
    tmin: float = 0.02
    dtgrow: float = 1.1
    dtshrink: float = 0.5
    alpha0: float = 0.25
    alphashrink: float = 0.99
    delaystep: int = 20
    vdfmax: int = 2000
    halfstepback: bool = True
    initialdelay: bool = True
    integrator: int = 0
    norm: int = NORM_MAX_ATOM
    variant: int = 0
    pad: int = 0
    dmax: float = 0.0


@dataclass
class Result:
    energy: float
    iterations: int
    force_evals: int
    stop: int
    fmax_atom: float
    f2norm: float
    finf: float
    dt_final: float
    alpha_final: float


def _sys(n, box, periodic, mass):
    s = _Sys()
    s.n = int(n)
    for d in range(3):
        s.box[d] = float(box[d])
        s.periodic[d] = int(bool(periodic[d]))
    s.mass = float(mass)
    return s


def _pot(pot: Potential, keep: list):
    kinds = {"lj": POT_LJ, "rgl": POT_RGL, "quad": POT_QUAD, "dwell": POT_DWELL, "sw": POT_SW}
    p = _Pot()
    p.kind = kinds[pot.kind]
    for name in ("eps", "sigma", "rc_lj", "A", "xi", "p", "q", "r0", "rs", "rc", "sw_A", "sw_B",
                 "sw_p", "sw_q", "sw_a", "sw_lambda", "sw_gamma"):
        setattr(p, name, float(getattr(pot, name)))
    if pot.kind == "quad":
        k = np.ascontiguousarray(pot.quad_k, dtype=np.float64)
        x0 = np.ascontiguousarray(pot.quad_x0, dtype=np.float64)
        keep += [k, x0]
        p.quad_k = k.ctypes.data_as(C.POINTER(C.c_double))
        p.quad_x0 = x0.ctypes.data_as(C.POINTER(C.c_double))
    if pot.kind == "dwell":
        dw = np.ascontiguousarray(pot.dwell, dtype=np.float64)
        assert dw.shape == (5,)
        keep.append(dw)
        p.dwell = dw.ctypes.data_as(C.POINTER(C.c_double))
    return p


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def energy_forces(x, box, pot: Potential, periodic=(1, 1, 1), mode: int = FORCE_BRUTE):
    """Total energy and forces (N x 3) of positions x (N x 3)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    f = np.zeros_like(x)
    e = C.c_double(0.0)
    keep: list = []
    s, p = _sys(len(x), box, periodic, 1.0), _pot(pot, keep)
    _check(_load().ora_energy_forces(C.byref(s), C.byref(p), x.ctypes.data, f.ctypes.data,
                                     C.byref(e), int(mode)), "energy_forces")
    return float(e.value), f


def energy_forces_subset(x, box, pot: Potential, which, periodic=(1, 1, 1),
                         mode: int = FORCE_CELLS):
    """Total energy and the forces of atoms `which` (len(which) x 3)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(which, dtype=np.int64)
    f = np.zeros((len(w), 3))
    e = C.c_double(0.0)
    keep: list = []
    s, p = _sys(len(x), box, periodic, 1.0), _pot(pot, keep)
    _check(_load().ora_energy_forces_subset(C.byref(s), C.byref(p), x.ctypes.data, w.ctypes.data,
                                            len(w), f.ctypes.data, C.byref(e), int(mode)),
           "energy_forces_subset")
    return float(e.value), f


def densities(x, box, pot: Potential, periodic=(1, 1, 1)):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    rho = np.zeros(len(x))
    keep: list = []
    s, p = _sys(len(x), box, periodic, 1.0), _pot(pot, keep)
    _check(_load().ora_densities(C.byref(s), C.byref(p), x.ctypes.data, rho.ctypes.data),
           "densities")
    return rho


def rgl_pair_terms(pot: Potential, r):
    """(n, 4): phi(r), g(r), phi'(r), g'(r) of the RGL pair functions."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros((len(r), 4))
    keep: list = []
    p = _pot(pot, keep)
    _check(_load().ora_rgl_pair_terms(C.byref(p), len(r), r.ctypes.data, out.ctypes.data),
           "rgl_pair_terms")
    return out


def rgl_param_derivs(x, box, pot: Potential, periodic=(1, 1, 1), mode: int = FORCE_BRUTE):
    """dE/dtheta (4,) and dF/dtheta (4, N, 3) for theta = (A, xi, p, q)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    dE = np.zeros(4)
    dF = np.zeros((4, len(x), 3))
    keep: list = []
    s, p = _sys(len(x), box, periodic, 1.0), _pot(pot, keep)
    _check(_load().ora_rgl_param_derivs(C.byref(s), C.byref(p), x.ctypes.data, dE.ctypes.data,
                                        dF.ctypes.data, int(mode)), "rgl_param_derivs")
    return dE, dF


def rgl_hvp(x, box, pot: Potential, u, periodic=(1, 1, 1), mode: int = FORCE_BRUTE):
    """Hessian-vector product (d^2 E/dx^2) u, N x 3."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
    hu = np.zeros_like(x)
    keep: list = []
    s, p = _sys(len(x), box, periodic, 1.0), _pot(pot, keep)
    _check(_load().ora_rgl_hvp(C.byref(s), C.byref(p), x.ctypes.data, u.ctypes.data,
                               hu.ctypes.data, int(mode)), "rgl_hvp")
    return hu


def rgl_cg(x, box, pot: Potential, b, tol=1e-12, maxit=10000, periodic=(1, 1, 1),
           mode: int = FORCE_BRUTE):
    """Solves H lambda = b (translations projected out); returns (lambda, iterations)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1, 3)
    lam = np.zeros_like(x)
    keep: list = []
    s, p = _sys(len(x), box, periodic, 1.0), _pot(pot, keep)
    it = _load().ora_rgl_cg(C.byref(s), C.byref(p), x.ctypes.data, b.ctypes.data, float(tol),
                            int(maxit), lam.ctypes.data, int(mode))
    if it < 0:
        raise RuntimeError("oracle CG failed")
    return lam, int(it)


def implicit_grad(x_star, box, pot: Potential, g, tol=1e-12, maxit=10000, periodic=(1, 1, 1),
                  mode: int = FORCE_BRUTE):
    """dL/dtheta at a minimum x*: lambda^T dF/dtheta with H lambda = dL/dx."""
    lam, it = rgl_cg(x_star, box, pot, g, tol, maxit, periodic, mode)
    _, dF = rgl_param_derivs(x_star, box, pot, periodic, mode)
    return np.einsum("kna,na->k", dF, lam), it


def fire2(x, box, pot: Potential, params: Params, mass: float, ftol: float, maxiter: int,
          periodic=(1, 1, 1), mode: int = FORCE_BRUTE, trace: int = 0, frozen=None):
    """Relaxes x (copied) with FIRE 2.0; returns (x_final, Result, trace_rows).
    frozen: None or one uint8 per atom, bit d set = component d frozen."""
    x = np.array(x, dtype=np.float64).reshape(-1, 3)
    keep: list = []
    s, p = _sys(len(x), box, periodic, mass), _pot(pot, keep)
    pr = _Params()
    for name, _ in _Params._fields_:
        if name == "frozen":
            continue
        setattr(pr, name, int(getattr(params, name)) if isinstance(getattr(pr, name), int)
                else float(getattr(params, name)))
    if frozen is not None:
        fz = np.ascontiguousarray(frozen, dtype=np.uint8)
        if fz.shape != (len(x),):
            raise ValueError("frozen must hold one byte per atom")
        keep.append(fz)
        pr.frozen = fz.ctypes.data
    res = _Result()
    tr = (_Trace * max(int(trace), 1))()
    _check(_load().ora_fire2(C.byref(s), C.byref(p), C.byref(pr), x.ctypes.data, float(ftol),
                             int(maxiter), int(mode), C.byref(res), C.cast(tr, C.c_void_p),
                             int(trace)), "fire2")
    r = Result(res.energy, res.iterations, res.force_evals, res.stop, res.fmax_atom, res.f2norm,
               res.finf, res.dt_final, res.alpha_final)
    rows = [dict(i=t.i, npos=t.npos, nneg=t.nneg, P=t.P, dt=t.dt, alpha=t.alpha,
                 energy=t.energy, fnorm=t.fnorm) for t in tr[:min(int(trace), r.iterations)]]
    return x, r, rows


def neb(path, box, pot: Potential, params: Params, mass: float, k_spring: float, climb: bool,
        ftol: float, maxiter: int, periodic=(1, 1, 1), mode: int = FORCE_BRUTE, frozen=None):
    """Nudged elastic band relaxed with FIRE: path is (m + 2, n, 3) with the
    fixed end states first and last.  Returns (path_out, Result, energies
    (m + 2), climbing-image index or 0)."""
    path = np.array(path, dtype=np.float64)
    if path.ndim != 3 or path.shape[2] != 3 or path.shape[0] < 3:
        raise ValueError("path must be (m + 2, n, 3) with m >= 1")
    m, n = path.shape[0] - 2, path.shape[1]
    keep: list = []
    s, p = _sys(n, box, periodic, mass), _pot(pot, keep)
    pr = _Params()
    for name, _ in _Params._fields_:
        if name == "frozen":
            continue
        setattr(pr, name, int(getattr(params, name)) if isinstance(getattr(pr, name), int)
                else float(getattr(params, name)))
    if frozen is not None:
        fz = np.ascontiguousarray(frozen, dtype=np.uint8)
        if fz.shape != (n,):
            raise ValueError("frozen must hold one byte per atom of an image")
        keep.append(fz)
        pr.frozen = fz.ctypes.data
    res = _Result()
    energies = np.zeros(m + 2)
    climber = C.c_int64(0)
    _check(_load().ora_neb(C.byref(s), C.byref(p), C.byref(pr), int(m), path.ctypes.data,
                           float(k_spring), int(bool(climb)), float(ftol), int(maxiter), int(mode),
                           C.byref(res), energies.ctypes.data, C.byref(climber)), "neb")
    r = Result(res.energy, res.iterations, res.force_evals, res.stop, res.fmax_atom, res.f2norm,
               res.finf, res.dt_final, res.alpha_final)
    return path, r, energies, int(climber.value)
