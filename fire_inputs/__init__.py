"""Seeded synthetic inputs shared by the oracle-side tests and the GPU-side
tests/bench.  This module only builds atom positions and boxes (lattices,
vacancies, strain, voids, random displacements) and holds the workload
constants; it contains none of the relaxation method's arithmetic.

Recipes (one numpy PCG64 generator per config, seeded as stated):
  lj_fcc_vacancy      FCC 4x4x4 cells, a = 1.5874 sigma, 256 sites, one site
                      removed at random, uniform +-0.1 sigma displacement per
                      Cartesian component.
  rgl_vacancy_box     FCC n^3 cells of Cu, a = 3.615 A, a fraction (or count)
                      of sites removed at random, Gaussian displacements
                      (std 0.05 A per component).
  rgl_void_box        FCC 63^3 cells, box and positions stretched by 2 % along
                      x, sites within 20 A of the box centre removed, Gaussian
                      displacements (std 0.02 A).
  rgl_batch           512 periodic FCC Cu boxes with n ~ U{3..12} cells per
                      edge, 1-3 vacancies each, Gaussian 0.05 A displacements.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Workload constants ---------------------------------------------------------
# Lennard-Jones (reduced units), cut and energy-shifted at 2.5 sigma.
LJ = dict(eps=1.0, sigma=1.0, rc=2.5)
LJ_A = 1.5874          # FCC lattice constant in sigma
LJ_MASS = 1.0
LJ_DT = 0.005          # dt_start in tau

# Second-moment (RGL) Cu: A, xi in eV, r0, rs, rc in Angstrom.
RGL_CU = dict(A=0.0855, xi=1.224, p=10.96, q=2.278, r0=2.556, rs=4.5, rc=5.0)
CU_A = 3.615           # FCC lattice constant, Angstrom
CU_MASS_AMU = 63.546
# metal units: a[A/ps^2] = F[eV/A] / m[amu] * 9648.533212...
EV_PER_A_AMU_TO_A_PS2 = 1.602176634e-19 / (1e-10 * 1.66053906660e-27) * 1e-14
CU_MASS = CU_MASS_AMU / EV_PER_A_AMU_TO_A_PS2   # eV ps^2 / A^2, so that a = F / m
CU_DT = 0.001          # ps

# Stillinger-Weber silicon (Stillinger and Weber, Phys. Rev. B 31, 5262
# (1985)): eps [eV], sigma [A] and the dimensionless A, B, p, q, a, lambda,
# gamma of the published parameter set.
SW_SI = dict(eps=2.1683, sigma=2.0951, sw_A=7.049556277, sw_B=0.6022245584, sw_p=4.0,
             sw_q=0.0, sw_a=1.80, sw_lambda=21.0, sw_gamma=1.20)
# diamond lattice constant of the pair minimum: nearest neighbours at 2^(1/6) sigma
SI_A = 4.0 * 2.0 ** (1.0 / 6.0) * SW_SI["sigma"] / np.sqrt(3.0)
SI_MASS_AMU = 28.0855
SI_MASS = SI_MASS_AMU / 9648.533212331001   # eV ps^2 / A^2 (see CU_MASS)
SI_DT = 0.001          # ps

FIRE_TABLE1 = dict(tmax=10.0, tmin=0.02, dtgrow=1.1, dtshrink=0.5, alpha0=0.25,
                   alphashrink=0.99, delaystep=20, vdfmax=2000, halfstepback=True,
                   initialdelay=True)

_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


@dataclass
class Config:
    """One relaxation problem: positions (N x 3, float64), box lengths, flags."""
    name: str
    x: np.ndarray
    box: np.ndarray
    periodic: tuple = (1, 1, 1)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def fcc_sites(nx: int, ny: int, nz: int, a: float) -> np.ndarray:
    """FCC sites of an nx x ny x nz block of cubic cells, cell-major order."""
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    corners = np.stack([ix, iy, iz], axis=-1).reshape(-1, 1, 3).astype(np.float64)
    return ((corners + _FCC_BASIS[None]) * a).reshape(-1, 3)


def lj_fcc_vacancy(seed: int = 1, ncell: int = 4, a: float = LJ_A, amp: float = 0.1) -> Config:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = fcc_sites(ncell, ncell, ncell, a)
    vac = int(rng.integers(len(x)))
    x = np.delete(x, vac, axis=0)
    x = x + rng.uniform(-amp, amp, size=x.shape)
    box = np.full(3, ncell * a)
    return Config("lj_fcc4_vac1", x, box, meta=dict(vacancies=[vac], ncell=ncell))


def rgl_vacancy_box(ncell: int = 20, seed: int = 2, vac_frac: float | None = 0.01,
                    n_vac: int | None = None, sigma: float = 0.05, a: float = CU_A) -> Config:
    rng = np.random.Generator(np.random.PCG64(seed))
    sites = fcc_sites(ncell, ncell, ncell, a)
    k = int(n_vac) if n_vac is not None else int(round(vac_frac * len(sites)))
    vac = np.sort(rng.choice(len(sites), size=k, replace=False)) if k > 0 else np.zeros(0, int)
    keep = np.ones(len(sites), bool)
    keep[vac] = False
    lattice = sites[keep]
    x = lattice + rng.normal(0.0, sigma, size=lattice.shape)
    box = np.full(3, ncell * a)
    return Config(f"rgl_cu{ncell}_vac{k}", x, box,
                  meta=dict(vacancies=vac.tolist(), vacancy_sites=sites[vac], lattice=lattice,
                            ncell=ncell))


def rgl_void_box(ncell: int = 63, seed: int = 3, strain: float = 0.02, void_r: float = 20.0,
                 sigma: float = 0.02, a: float = CU_A) -> Config:
    rng = np.random.Generator(np.random.PCG64(seed))
    sites = fcc_sites(ncell, ncell, ncell, a)
    box = np.full(3, ncell * a)
    sites[:, 0] *= 1.0 + strain
    box[0] *= 1.0 + strain
    centre = 0.5 * box
    keep = np.sum((sites - centre) ** 2, axis=1) >= void_r * void_r
    lattice = sites[keep]
    x = lattice + rng.normal(0.0, sigma, size=lattice.shape)
    return Config(f"rgl_cu{ncell}_strain{strain:g}_void{void_r:g}", x, box,
                  meta=dict(removed=int((~keep).sum()), ncell=ncell))


def rgl_batch(n_sys: int = 512, seed: int = 4, nmin: int = 3, nmax: int = 12,
              sigma: float = 0.05, a: float = CU_A):
    """List of independent periodic Cu boxes of uneven sizes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(n_sys):
        n = int(rng.integers(nmin, nmax + 1))
        k = int(rng.integers(1, 4))
        sites = fcc_sites(n, n, n, a)
        vac = rng.choice(len(sites), size=k, replace=False)
        keep = np.ones(len(sites), bool)
        keep[vac] = False
        x = sites[keep] + rng.normal(0.0, sigma, size=(int(keep.sum()), 3))
        out.append(Config(f"batch{s}_cu{n}_vac{k}", x, np.full(3, n * a),
                          meta=dict(ncell=n, vacancies=np.sort(vac).tolist())))
    return out


def perfect_fcc(ncell: int, a: float) -> Config:
    return Config(f"fcc{ncell}", fcc_sites(ncell, ncell, ncell, a), np.full(3, ncell * a))


def neb_vacancy_hop(ncell: int = 3, seed: int = 6, n_img: int = 5, sigma: float = 0.0,
                    a: float = CU_A) -> Config:
    """End states and straight-line initial path of a nearest-neighbour
    vacancy hop in a periodic Cu FCC box (the NEB workload): site v is
    vacant in state 0; in state 1 the atom of the neighbouring site w has
    moved into v.  Atom order is the same in both states (the hopping atom
    keeps its index).  x holds the (n_img + 2, n, 3) path, images 0 and
    n_img + 1 the (unrelaxed) end states; sigma adds the same seeded
    Gaussian noise to every image."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sites = fcc_sites(ncell, ncell, ncell, a)
    box = np.full(3, ncell * a)
    v = int(rng.integers(len(sites)))
    d = sites - sites[v]
    d -= box * np.rint(d / box)
    r = np.sqrt(np.sum(d * d, axis=1))
    nn = np.flatnonzero(np.abs(r - a / np.sqrt(2.0)) < 1e-6)
    w = int(nn[rng.integers(len(nn))])
    keep = np.ones(len(sites), bool)
    keep[v] = False
    end0 = sites[keep].copy()
    k = int(np.flatnonzero(np.flatnonzero(keep) == w)[0])   # index of the hopping atom
    end1 = end0.copy()
    end1[k] = end0[k] - d[w]          # w -> v along the minimum-image bond
    noise = rng.normal(0.0, sigma, size=end0.shape) if sigma > 0 else np.zeros_like(end0)
    t = np.linspace(0.0, 1.0, n_img + 2)[:, None, None]
    path = end0[None] + t * (end1 - end0)[None] + noise[None]
    return Config(f"neb_cu{ncell}_hop", path, box,
                  meta=dict(vacancy_site=sites[v], target_site=sites[w], hopper=k, ncell=ncell,
                            n_img=n_img))


_DIAMOND_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5],
                           [0.25, 0.25, 0.25], [0.75, 0.75, 0.25], [0.75, 0.25, 0.75],
                           [0.25, 0.75, 0.75]])


def diamond_sites(n: int, a: float) -> np.ndarray:
    """Diamond-lattice sites of an n x n x n block of cubic cells (8 per cell)."""
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    corners = np.stack([ix, iy, iz], axis=-1).reshape(-1, 1, 3).astype(np.float64)
    return ((corners + _DIAMOND_BASIS[None]) * a).reshape(-1, 3)


def sw_si_vacancy_box(ncell: int = 8, seed: int = 7, n_vac: int = 1, sigma: float = 0.05,
                      a: float | None = None) -> Config:
    """Periodic diamond Si box (Stillinger-Weber workload, the paper's
    three-body case): n_vac seeded vacancies, Gaussian noise per component."""
    a = SI_A if a is None else a
    rng = np.random.Generator(np.random.PCG64(seed))
    sites = diamond_sites(ncell, a)
    vac = np.sort(rng.choice(len(sites), size=n_vac, replace=False)) if n_vac > 0 else np.zeros(0, int)
    keep = np.ones(len(sites), bool)
    keep[vac] = False
    lattice = sites[keep]
    x = lattice + rng.normal(0.0, sigma, size=lattice.shape)
    return Config(f"sw_si{ncell}_vac{n_vac}", x, np.full(3, ncell * a),
                  meta=dict(vacancies=vac.tolist(), lattice=lattice, ncell=ncell))


# ---------------------------------------------------------------------------
# Free surfaces (open axes).  The paper's cases include a Si slab periodic in
# x and y only (five vacancies, 32,762 atoms, Stillinger-Weber) and open
# clusters and pillars; these are synthetic stand-ins of that structure.

def rgl_slab(ncell: int = 6, nz: int | None = None, seed: int = 21, n_vac: int = 2,
             sigma: float = 0.05, vacuum: float = 10.0, z_shift: float = 0.0,
             a: float = CU_A) -> Config:
    """Cu FCC slab of ncell x ncell x nz cells, periodic in x and y, open in z:
    box z length = nz a + vacuum; every z moved by z_shift (a negative shift
    puts the lowest layers below z = 0, outside the box on the open axis)."""
    nz = ncell if nz is None else nz
    rng = np.random.Generator(np.random.PCG64(seed))
    sites = fcc_sites(ncell, ncell, nz, a)
    vac = np.sort(rng.choice(len(sites), size=n_vac, replace=False)) if n_vac > 0 else np.zeros(0, int)
    keep = np.ones(len(sites), bool)
    keep[vac] = False
    x = sites[keep] + rng.normal(0.0, sigma, size=(int(keep.sum()), 3))
    x[:, 2] += z_shift
    box = np.array([ncell * a, ncell * a, nz * a + vacuum])
    return Config(f"rgl_slab{ncell}x{nz}_vac{n_vac}", x, box, periodic=(1, 1, 0),
                  meta=dict(vacancies=vac.tolist(), ncell=ncell, nz=nz))


def rgl_cluster(radius: float = 10.0, seed: int = 22, sigma: float = 0.05,
                centre=(15.0, 15.0, 15.0), box: float = 30.0, a: float = CU_A) -> Config:
    """Spherical Cu cluster (FCC sites within `radius` of a lattice site),
    open on every axis, centred at `centre` in a cube of side `box` (a centre
    near a face puts atoms outside the box)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(np.ceil(radius / a)) + 1
    sites = fcc_sites(2 * n, 2 * n, 2 * n, a) - n * a
    sites = sites[np.sum(sites * sites, axis=1) <= radius * radius]
    x = sites + np.asarray(centre, dtype=np.float64) + rng.normal(0.0, sigma, size=sites.shape)
    return Config(f"rgl_cluster_r{radius:g}", x, np.full(3, float(box)), periodic=(0, 0, 0),
                  meta=dict(radius=radius))


def sw_si_slab(ncell: int = 16, nz: int | None = None, seed: int = 23, n_vac: int = 5,
               sigma: float = 0.05, vacuum: float = 10.0, a: float | None = None) -> Config:
    """Diamond Si slab, periodic in x and y, open in z, with n_vac seeded
    vacancies (the structure of the paper's silicon vacancy case)."""
    a = SI_A if a is None else a
    nz = ncell if nz is None else nz
    rng = np.random.Generator(np.random.PCG64(seed))
    ix, iy, iz = np.meshgrid(np.arange(ncell), np.arange(ncell), np.arange(nz), indexing="ij")
    corners = np.stack([ix, iy, iz], axis=-1).reshape(-1, 1, 3).astype(np.float64)
    sites = ((corners + _DIAMOND_BASIS[None]) * a).reshape(-1, 3)
    vac = np.sort(rng.choice(len(sites), size=n_vac, replace=False)) if n_vac > 0 else np.zeros(0, int)
    keep = np.ones(len(sites), bool)
    keep[vac] = False
    x = sites[keep] + rng.normal(0.0, sigma, size=(int(keep.sum()), 3))
    box = np.array([ncell * a, ncell * a, nz * a + vacuum])
    return Config(f"sw_si_slab{ncell}x{nz}_vac{n_vac}", x, box, periodic=(1, 1, 0),
                  meta=dict(vacancies=vac.tolist(), ncell=ncell, nz=nz))
