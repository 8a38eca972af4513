"""Writes implicit_grad_rgl32k.json: the oracle's implicit gradient of the
vacancy loss on the differentiation workload (the 20^3-cell RGL-Cu box with
one vacancy, 31,999 atoms, seed 5).

Calls only the FP64 CPU oracle (oracle/) and the seeded input generator
(fire_inputs); nothing here comes from the CUDA library.  Steps:
  1. relax the box with the oracle's FIRE 2.0 (Algorithm 2 + Algorithm 4,
     Table 1 parameters, cell-grid forces) to max_i |F_i| < 1e-12 eV/A;
  2. loss L = sum over the atoms whose lattice site lies within 6 A of the
     vacancy site (minimum image) of |x*_i - x_lattice,i|^2, and dL/dx*;
  3. solve H lambda = dL/dx* by the oracle's conjugate gradient (relative
     residual 1e-12, translations projected out) and contract lambda with
     dF/dtheta for theta = (A, xi, p, q): dL/dtheta = lambda . dF/dtheta
     (at a minimum F(x*, theta) = 0, so dx*/dtheta = H^-1 dF/dtheta).

Run:  python tests/golden/make_implicit_grad_rgl32k.py   (a few minutes on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import fire_inputs as fi  # noqa: E402
import oracle  # noqa: E402

FTOL = 1e-12
CG_TOL = 1e-12
RADIUS = 6.0
THETA = ("A", "xi", "p", "q")


def main():
    c = fi.rgl_vacancy_box(ncell=20, seed=5, n_vac=1)
    pot = oracle.Potential("rgl", **fi.RGL_CU)
    t0 = time.perf_counter()
    xo, r, _ = oracle.fire2(c.x, c.box, pot, oracle.Params(dt_start=fi.CU_DT), fi.CU_MASS,
                            FTOL, 400000, mode=oracle.FORCE_CELLS)
    t_relax = time.perf_counter() - t0
    assert r.stop == oracle.STOP_FTOL, r
    site = c.meta["vacancy_sites"][0]
    d = c.meta["lattice"] - site
    d -= c.box * np.rint(d / c.box)
    sel = np.flatnonzero(np.sum(d * d, 1) < RADIUS * RADIUS)
    dd = xo[sel] - c.meta["lattice"][sel]
    dd -= c.box * np.rint(dd / c.box)
    loss = float(np.sum(dd * dd))
    g = np.zeros_like(xo)
    g[sel] = 2.0 * dd
    t0 = time.perf_counter()
    grad, it = oracle.implicit_grad(xo, c.box, pot, g, tol=CG_TOL, mode=oracle.FORCE_CELLS)
    t_cg = time.perf_counter() - t0
    out = {
        "what": "dL/dtheta of the vacancy loss at the relaxed 31,999-atom RGL-Cu vacancy box "
                "(fire_inputs.rgl_vacancy_box(ncell=20, seed=5, n_vac=1)), FP64 CPU oracle",
        "citation": "FIRE 2.0 relaxation: Algorithm 2 with the semi-implicit Euler integrator "
                    "of Algorithm 4 and the Table 1 parameters; implicit gradient of the "
                    "relaxed configuration: dx*/dtheta = H^-1 dF/dtheta at F(x*, theta) = 0",
        "theta_names": list(THETA),
        "theta": [fi.RGL_CU[k] for k in THETA],
        "dL_dtheta": [float(v) for v in grad],
        "loss": loss,
        "loss_atoms": int(len(sel)),
        "radius_A": RADIUS,
        "n_atoms": int(c.n),
        "ftol": FTOL,
        "cg_tol": CG_TOL,
        "oracle_fire_iterations": int(r.iterations),
        "oracle_final_fmax_atom": float(r.fmax_atom),
        "oracle_energy_per_atom": float(r.energy / c.n),
        "oracle_cg_iterations": int(it),
        "oracle_seconds": {"relax": round(t_relax, 1), "cg": round(t_cg, 1),
                           "threads": oracle.max_threads()},
        "generator": "tests/golden/make_implicit_grad_rgl32k.py",
    }
    path = os.path.join(HERE, "implicit_grad_rgl32k.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
