"""Benchmark: FIRE 2.0 relaxation of the ~1M-atom RGL-Cu configuration on one GB300.

Workload (one "step"): relax the 63x63x63-cell FCC Cu box (2 % uniaxial
strain along x, 20 A void removed at the centre, Gaussian 0.02 A noise,
997,450 atoms) from its initial configuration until max_i |F_i| < 1e-6 eV/A,
with FIRE 2.0 (Algorithm 2) + semi-implicit Euler (Algorithm 4), Table 1
parameters, dt_start = 1 fs, m = 63.546 amu.  The whole relaxation -- list
builds, both RGL force passes, the FP64 reductions, the dt/alpha control and
the integration -- runs inside one CUDA graph launch (fire_minimize_dev).

metric: atom-iterations per second (N x FIRE iterations / wall time), higher is
better; ms_per_step is the time-to-ftol of one relaxation.  The line also
carries the other precision forms on the same workload (`forms`, each
relaxed structure re-checked with the IEEE-FP64 kernels), a nudged-elastic-
band run (`neb`), the roofline of the dominant kernel and the oracle timed on
the host cores (`cpu_baseline`).

`--impl reference` times the FP64 CPU oracle (plain C, OpenMP) on a bounded
sample of the same workload (a few FIRE iterations of the same box).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fire_inputs as fi  # noqa: E402

METRIC = "FIRE2 atom-iters/s & time-to-ftol, EAM 1M atoms, 1 GB300; HBM roofline fraction"
UNIT = "atom-iters/s"
FTOL = 1e-6
MAXITER = 200000
CONFIGS = {
    "rgl1m": lambda: fi.rgl_void_box(),
    "rgl32k": lambda: fi.rgl_vacancy_box(ncell=20, seed=2),
    "lj256": lambda: fi.lj_fcc_vacancy(seed=1),
}
# Algorithmic floating-point operations per unordered pair inside the
# cut-off: the method's own work for one pass (an FMA counts 2, a square
# root, division or exponential 1), whatever the kernel does to get there
# (table interpolation, double-float arithmetic and evaluating a pair from
# both ends are implementation work and not counted):
#   density pass (rho_i = sum_j g(r_ij), E_rep = sum_j phi(r_ij), Sec. 4 /
#   the RGL form): separation 3 + r^2 5 = 8; r 1; s = r/r0 - 1: 2;
#   exp(-p s), exp(-2q s): 2 + 2; prefactors A, xi^2: 2; taper t 2,
#   S and S' 16 (Horner, also for pairs below rs: per-pair average rounded
#   up); phi = e S, g = e S: 2; rho_i, rho_j sums 2; energy 2        39
#   force pass (F = -grad E, Sec. 2.1): separation 8, r 1, s 2, exps 4,
#   prefactors 2, taper 18; phi', g' (e (-a S + S')) 6; fs = (2 phi' +
#   (F'_i + F'_j) g') / r: 5; F_i and F_j: 6 + 6                     56
#   LJ force pass: separation 8; 1/r^2 1; (s/r)^6, ^12: 3; w = 24 eps
#   (2 s12 - s6) / r^2: 4; pair energy 3; F_i and F_j 12              31
METHOD_FLOP_PER_PAIR = {"density": 39, "force": 56, "force_lj": 31}
# the square roots, exponentials and divisions inside those counts, per pair
TRANSCENDENTALS_PER_PAIR = {"density": {"sqrt": 1, "exp": 2}, "force": {"sqrt": 1, "exp": 2},
                            "force_lj": {"div": 1}}
# the kernel each stage runs, per (form, pair evaluation), and the unit it
# issues on ("fp64": FP64 pipe; "ff": double-float arithmetic on the FP32
# pipe; "fp32")
STAGE_KERNELS = {
    ("fp64", "table"): {"density": ("k_density_ff", "ff"), "force": ("k_force_ff", "ff")},
    ("fp64", "analytic"): {"density": ("k_density", "fp64"), "force": ("k_force_rgl", "fp64")},
    ("fp32pair", "analytic"): {"density": ("k_density32", "fp32"),
                               "force": ("k_force32", "fp32")},
    ("fp32pair", "table"): {"density": ("k_density32_tab", "fp32"),
                            "force": ("k_force32_tab", "fp32")},
}
# the FP64 table form on a half list runs its pair passes on shared-memory
# tiles when asked (--tiles on); the library's automatic choice is untiled
TILED_KERNELS = {"density": ("k_density_tile", "ff"), "force": ("k_force_tile", "ff")}
# FP32 instructions of one double-float multiply-add (ff_madd, counted from
# fire2_table.cuh): the emulation's own ceiling is the FP32 FMA rate / 15 in
# FP64-equivalent FLOP/s (reported as emulation_efficiency, not as the
# roofline)
FF_FP32_PER_FMA = 15
# Algorithmic HBM bytes per atom and iteration (x, v read+write, F'(rho)
# write+read): 112 for RGL, 96 for LJ.
ALG_BYTES_PER_ATOM_ITER = {"rgl": 112, "lj": 96}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="rgl1m", choices=sorted(CONFIGS))
    ap.add_argument("--form", default="fp64", choices=["fp64", "fp32pair"])
    ap.add_argument("--pair", default=None, choices=["table", "analytic"],
                    help="RGL pair functions: quintic tables or exponentials (default: "
                         "tables for fp64, exponentials for fp32pair, the faster of each)")
    ap.add_argument("--newton", default="auto", choices=["auto", "on", "off"],
                    help="FP64 tabulated form: half list + atomics (on) or full list (off)")
    ap.add_argument("--tiles", default="auto", choices=["auto", "on", "off"],
                    help="FP64 half-list passes on shared-memory tiles (auto: the "
                         "library's choice, untiled)")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the batched block (512 systems), one timed batch (profiling aid)")
    ap.add_argument("--batch-tuning", default=None,
                    help="threads,ctas_per_sm,cluster_size for the batched block (default: autotune)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the second form (FP32-pair next to FP64 and vice versa)")
    ap.add_argument("--no-neb", action="store_true",
                    help="skip the nudged-elastic-band line (vacancy hop, 6 images)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--exec", default="graph", choices=["graph", "chunked"],
                    help="graph: one CUDA graph with a WHILE node per relaxation (default); "
                         "chunked: plain graphs of 32 iterations (lets ncu list the kernels)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--study", action="store_true",
                    help="instead of the throughput line: force evaluations to ftol per "
                         "integrator and FIRE variant, and the alpha0 / tmax / dt sweeps "
                         "(the paper's comparisons, on synthetic stand-ins)")
    ap.add_argument("--eval-only", action="store_true",
                    help="one energy/force evaluation of the config (profiling aid)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--cpu-full", action="store_true",
                    help="time the oracle's one-thread runs of the small configurations in "
                         "full instead of as bounded samples (several minutes)")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the LJ and 32k-atom configuration blocks")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def potential_for(cfg_name, form="fp64"):
    import paper_1908_02038_gb300 as fg
    if cfg_name.startswith("lj"):
        return (fg.Potential(fg.FIRE_POT_LJ, eps=1.0, sigma=1.0, rc_lj=2.5, skin=0.3),
                fi.LJ_MASS, fi.LJ_DT, 1e-8)
    prec = fg.FIRE_PREC_FP32_PAIR if form == "fp32pair" else fg.FIRE_PREC_FP64
    # the FP32-pair form stops at ftol on FP64 forces: by default the library
    # evaluates in FP64 from 3 ftol on (fire_params_t.confirm64), so its structure meets
    # ftol in FP64 (which the line checks again)
    ftol = FTOL
    return (fg.Potential(fg.FIRE_POT_RGL, precision=prec, skin=0.3, **fi.RGL_CU), fi.CU_MASS,
            fi.CU_DT, ftol)


def count_pairs(x, box, rc):
    """Unordered pairs closer than rc (periodic), for the algorithmic op count."""
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(x, box), boxsize=box)
    return int((t.count_neighbors(t, rc) - len(x)) // 2)


def gpu_smi_id(dev_index):
    """An id nvidia-smi resolves to the same physical GPU as torch's device
    dev_index: nvidia-smi ignores CUDA_VISIBLE_DEVICES, so a logical index
    could name another GPU of a shared machine.  The UUID, else the PCI bus
    id, else the index."""
    try:
        import torch
        props = torch.cuda.get_device_properties(dev_index)
        u = str(getattr(props, "uuid", "") or "")
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
        if hasattr(props, "pci_bus_id"):
            return "%08X:%02X:%02X.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id,
                                         getattr(props, "pci_device_id", 0))
    except Exception:
        pass
    return str(dev_index)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.smi_id = gpu_smi_id(index)
        self.proc = None
        self.lines = []
        # raw nvidia-smi samples go to a temporary file that is removed once
        # read, unless FIRE2_CLOCKS_DIR names a folder to keep them in (the
        # JSON line carries their summary)
        self.keep_dir = os.environ.get("FIRE2_CLOCKS_DIR")
        self.path = None

    def __enter__(self):
        try:
            if self.keep_dir:
                os.makedirs(self.keep_dir, exist_ok=True)
                self.path = os.path.join(self.keep_dir, f"clocks_bench_{os.getpid()}.csv")
                self.fh = open(self.path, "w")
            else:
                fd, self.path = tempfile.mkstemp(prefix="clocks_bench_", suffix=".csv")
                self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.smi_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.path:
            try:
                self.fh.close()
                with open(self.path) as fh:
                    self.lines = fh.readlines()
                if not self.keep_dir:
                    os.remove(self.path)
            except Exception:
                pass

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "sampled_gpu": self.smi_id}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "sampled_gpu": self.smi_id}


def _strip_comments(src):
    """C/CUDA source without comments and with whitespace collapsed, so that
    an edit to a comment or to the layout leaves the hash unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":   # string or character literal, copied whole
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def _device_src_hash():
    """Hash of the code of every kernel source (csrc/*.cu, *.cuh; comments
    and whitespace left out): ncu figures recorded under another hash
    describe other code."""
    import glob
    import hashlib
    h = hashlib.sha256()
    paths = glob.glob(os.path.join(ROOT, "paper_1908_02038_gb300", "csrc", "*.cu*"))
    for path in sorted(paths, key=os.path.basename):
        h.update(os.path.basename(path).encode())
        h.update(_strip_comments(open(path, encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def read_ncu(kernel, workload="rgl1m"):
    """ncu figures of `kernel` on `workload` from the committed summary
    profiles/ncu_counters.txt (one line per kernel: name, source hash,
    workload, then key=value pairs), if its recorded source hash matches the
    current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_counters.txt")
    if not os.path.exists(path):
        return None
    h = _device_src_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == h and parts[2] == workload:
            out = {}
            for kv in parts[3:]:
                if kv.startswith("#"):   # the command the line came from
                    break
                k, _, v = kv.partition("=")
                try:
                    out[k] = float(v)
                except ValueError:
                    out[k] = v
            return out
    return None


def host_cpu():
    """CPU model and core counts of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() == "Model name" and val.strip():
                model = val.strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"model": model or platform.processor() or "unknown", "arch": platform.machine(),
            "nproc": os.cpu_count(), "affinity": len(os.sched_getaffinity(0))}


TILE_MODES = {"auto": 0, "on": 1, "off": 2}   # FIRE_TILES_AUTO / ON / OFF


def tiles_active(args, form, pair, n):
    """Whether the library runs the FP64 half-list passes on tiles."""
    if form != "fp64" or pair != "table" or args.newton == "off":
        return False
    return args.tiles == "on"


def default_pair(form):
    return "analytic" if form == "fp32pair" else "table"


def relax_form(fg, torch, cfg, form, pair, args, dev, stream, clocks=True, confirm64=None):
    """Times args.steps relaxations of cfg (after args.warmup untimed ones) in
    one form; returns the measurement, the handle (still open) and the
    relaxed positions of the last step.  confirm64: the FP32-pair form's FP64
    check (fire_fp64_check; None = the library default, FP64 from 3 ftol on)."""
    pot, mass, dt, ftol = potential_for(args.config, form)
    pot.pair_eval = fg.FIRE_PAIR_ANALYTIC if pair == "analytic" else fg.FIRE_PAIR_TABLE
    pot.newton = {"auto": fg.FIRE_NEWTON_AUTO, "on": fg.FIRE_NEWTON_ON,
                  "off": fg.FIRE_NEWTON_OFF}[args.newton]
    x0 = torch.tensor(cfg.x, dtype=torch.float64, device=dev)
    work = torch.empty_like(x0)
    extra = {} if confirm64 is None else {"confirm64": confirm64}
    h = fg.FireHandle(cfg.n, mass, pot, dt_start=dt, **extra)
    h.set_pair_tiles(TILE_MODES[args.tiles])
    if args.exec == "chunked":
        h.set_exec_mode(fg.FIRE_EXEC_CHUNKED, 32)

    def step():
        work.copy_(x0)
        return h.minimize_dev(work, cfg.box, ftol, MAXITER, stream)

    for _ in range(args.warmup):
        step()
    results = []
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with (ClockSampler(dev.index) if clocks else _NoClock()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            results.append(step().as_dict())
        ev1.record(stream)
        torch.cuda.synchronize()
    return {"ms": ev0.elapsed_time(ev1), "results": results, "clocks": clk.summary(),
            "pot": pot, "ftol": ftol}, h, work


class _NoClock:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        pass

    def summary(self):
        return None


def launches_of(results, is_rgl, fp32, cell_mode, chunked=False, tiled=False, body=8, chunk=32):
    """Kernels one relaxation launches: prepare, list build, forces, the
    reductions with the control step (one launch), finalize once; then the
    loop passes, launched a whole WHILE body (`body` iterations, graph mode)
    or a whole chunk (`chunk`, chunked mode) at a time, the passes after the
    stop returning at once: per pass update, forces, reductions + control.
    The build chain (binning + list) runs under an IF node once per rebuild
    in graph mode with cell lists, and is launched with every pass (returning
    at once unless due) in the chunked mode and for all-pairs lists.  The
    FP32-pair form also has the two FP64 confirming passes: launched once in
    the set-up, then in the graph loop only in the passes that confirm a
    stop (an IF node), in the chunked loop with every pass.  Each
    confirmation is one more loop pass (force evaluations - iterations - 1)."""
    build_k = (6 + (1 if tiled else 0)) if cell_mode else 1
    force_k = (2 if fp32 else 3) if is_rgl else 1
    per = chunk if chunked else body
    total = 0
    for rr in results:
        conf = max(0, rr["force_evals"] - rr["iterations"] - 1) if fp32 else 0
        passes = rr["iterations"] + conf
        launched = -(-passes // per) * per
        total += (1 + build_k + force_k + 1 + 1) + (2 if fp32 else 0)
        total += (1 + force_k + 1) * launched
        if chunked or not cell_mode:
            total += build_k * launched
        else:
            total += build_k * max(0, rr["nbr_builds"] - 1)
        if fp32:
            total += 2 * (launched if chunked else conf)
    return total


def neb_block(fg, torch, form, dev):
    """Nudged elastic band of a vacancy hop in a 12^3-cell Cu box (6,911
    atoms, the size of the paper's NEB case 7) with 6 movable images and a
    climbing image, relaxed to 1e-4 eV/A on the NEB forces; end states
    relaxed first (FP64).  Reports atom-iterations over all images per
    second and the barrier; the climbing image is checked in FP64."""
    c = fi.neb_vacancy_hop(ncell=12, seed=6, n_img=6)
    n, m = c.x.shape[1], 6
    pot, mass, dt, _ = potential_for("rgl1m", form)
    pot.pair_eval = fg.FIRE_PAIR_ANALYTIC if default_pair(form) == "analytic" else fg.FIRE_PAIR_TABLE
    pot64, _, _, _ = potential_for("rgl1m", "fp64")
    path = c.x.copy()
    with fg.FireHandle(n, mass, pot64, dt_start=dt) as h:
        for e in (0, -1):
            x = np.ascontiguousarray(path[e])
            r = h.minimize(x, c.box, 1e-8, 100000)
            path[e] = x
    t = np.linspace(0.0, 1.0, m + 2)[:, None, None]
    path = np.ascontiguousarray(path[0][None] + t * (path[-1] - path[0])[None])
    d0 = torch.tensor(path, dtype=torch.float64, device=dev)
    d = torch.empty_like(d0)
    with fg.FireNEB(m, n, mass, pot, 1.0, True, dt_start=dt) as h:
        for _ in range(2):
            d.copy_(d0)
            h.minimize_dev(d, c.box, 1e-4, 100000)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d.copy_(d0)
        ev0.record()
        r, E, cl = h.minimize_dev(d, c.box, 1e-4, 100000)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    with fg.FireHandle(n, mass, pot64, dt_start=dt) as h:
        e_cl, f_cl = h.energy_forces(d[cl].cpu().numpy(), c.box)
        e_0, _ = h.energy_forces(path[0], c.box)
    return {"workload": f"vacancy hop in Cu 12^3 cells ({n} atoms), {m} images + climbing "
                        "image, NEB forces < 1e-4 eV/A", "form": form,
            "value": n * m * r.iterations / (ms * 1e-3), "unit": UNIT, "ms": ms,
            "iterations": r.iterations, "climbing_image": cl,
            "barrier_eV": float(E[cl] - E[0]),
            "barrier_fp64_check_eV": float(e_cl - e_0),
            "climbing_image_fp64_max_force": float(np.linalg.norm(f_cl, axis=1).max())}


def sw_block(fg, torch, dev, steps=3):
    """Stillinger-Weber silicon (the paper's three-body family): a 16^3-cell
    diamond box with one vacancy (32,767 atoms), FP64, relaxed to 1e-6 eV/A;
    atom-iterations per second over `steps` timed relaxations after one
    untimed."""
    c = fi.sw_si_vacancy_box(ncell=16, seed=7, n_vac=1, sigma=0.05)
    pot = fg.Potential(fg.FIRE_POT_SW, skin=0.3, **fi.SW_SI)
    x0 = torch.tensor(c.x, dtype=torch.float64, device=dev)
    w = torch.empty_like(x0)
    with fg.FireHandle(c.n, fi.SI_MASS, pot, dt_start=fi.SI_DT) as h:
        w.copy_(x0)
        h.minimize_dev(w, c.box, 1e-6, 100000)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = 0
        ev0.record()
        for _ in range(steps):
            w.copy_(x0)
            r = h.minimize_dev(w, c.box, 1e-6, 100000)
            its += r.iterations
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    return {"workload": f"SW Si diamond 16^3 cells, 1 vacancy ({c.n} atoms), FP64, "
                        "max|F_i| < 1e-6 eV/A",
            "value": c.n * its / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "iterations": r.iterations, "energy_per_atom": r.energy / c.n,
            "final_fmax_atom": r.fmax_atom}


def batch_block(fg, torch, dev, steps=3, tuning=None, compare=True):
    """The batched form: 512 independent Cu boxes of 3^3..12^3 cells (1-3
    vacancies each, ~1.24 M atoms) relaxed in one persistent launch,
    FP32-pair with FP64 reductions, each to max|F_i| < 1e-6 eV/A (every
    system finishing in FP64 from 3 ftol on, the library's default); launch shape from the library's
    autotuner; atom-iterations over all systems per second over `steps`
    timed batches after one untimed."""
    cfgs = fi.rgl_batch(n_sys=512, seed=4)
    x = np.ascontiguousarray(np.concatenate([c.x for c in cfgs]))
    boxes = np.array([c.box for c in cfgs])
    counts = np.array([c.n for c in cfgs])
    pot = fg.Potential(fg.FIRE_POT_RGL, precision=fg.FIRE_PREC_FP32_PAIR,
                       pair_eval=fg.FIRE_PAIR_ANALYTIC, skin=0.3, **fi.RGL_CU)
    x0 = torch.tensor(x, dtype=torch.float64, device=dev)
    w = torch.empty_like(x0)
    with fg.FireBatch(counts, fi.CU_MASS, pot, dt_start=fi.CU_DT) as b:
        if tuning:
            th, c, cl = (int(v) for v in tuning.split(","))
            b.set_tuning(th, c, cl)
            tune = {"threads_per_block": th, "ctas_per_sm": c, "cluster_size": cl}
        else:
            tune = b.autotune(x, boxes)
        w.copy_(x0)
        b.minimize_dev(w, boxes, FTOL, MAXITER)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = 0
        ev0.record()
        for _ in range(steps):
            w.copy_(x0)
            res = b.minimize_dev(w, boxes, FTOL, MAXITER)
            its += sum(int(r.iterations) * int(n) for r, n in zip(res, counts))
        ev1.record()
        torch.cuda.synchronize()
        x_fin = w.cpu().numpy()
    ms = ev0.elapsed_time(ev1)
    out = {"workload": f"512 Cu boxes 3^3..12^3 cells ({int(counts.sum())} atoms), FP32-pair, "
                       "one persistent launch", "value": its / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms / steps, "tuning": tune,
           "converged": int(sum(r.stop == fg.FIRE_STOP_FTOL for r in res)),
           "max_iterations": int(max(r.iterations for r in res))}
    if compare:
        # the same batch with one FP64 confirmation of each system's stop on
        # ftol (the default finishes in FP64 below 3 ftol), same launch shape
        with fg.FireBatch(counts, fi.CU_MASS, pot, dt_start=fi.CU_DT,
                          confirm64=fg.FIRE_FP64_CHECK_CONFIRM) as bf:
            bf.set_tuning(tune["threads_per_block"], tune["ctas_per_sm"],
                          tune.get("cluster_size", 1) or 1)
            w.copy_(x0)
            bf.minimize_dev(w, boxes, FTOL, MAXITER)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w.copy_(x0)
            e0.record()
            rf = bf.minimize_dev(w, boxes, FTOL, MAXITER)
            e1.record()
            torch.cuda.synchronize()
        msf = e0.elapsed_time(e1)
        out["confirm64"] = {"ms_per_step": msf,
                           "value": sum(int(r.iterations) * int(n) for r, n in zip(rf, counts))
                           / (msf * 1e-3), "unit": UNIT,
                           "converged": int(sum(r.stop == fg.FIRE_STOP_FTOL for r in rf)),
                           "max_iterations": int(max(r.iterations for r in rf))}
        out.update(batch_compare(fg, torch, dev, cfgs, x, x_fin, boxes, counts))
    return out


def batch_compare(fg, torch, dev, cfgs, x, x_fin, boxes, counts):
    """The batched FP32-pair result next to FP64 GPU paths on the same
    systems, all to the same converged max|F_i| < 1e-6 eV/A checked in FP64:
    every FP32-pair structure re-evaluated in FP64; the whole batch relaxed
    in the batched FP64 form (double-float table terms, the default FP64
    pair evaluation); and a sample of 32 systems (every 16th by
    size) relaxed one at a time through the single-system FP64 path (default
    form, whole loop in one CUDA graph), as a caller without the batched
    entry point would."""
    pot64 = fg.Potential(fg.FIRE_POT_RGL, precision=fg.FIRE_PREC_FP64, skin=0.3, **fi.RGL_CU)
    with fg.FireBatch(counts, fi.CU_MASS, pot64, dt_start=fi.CU_DT) as b:
        tune64 = b.autotune(x, boxes)
        chk, _ = b.minimize(x_fin.copy(), boxes, FTOL, 0)
        fmax64 = max(r.fmax_atom for r in chk)
        x0 = torch.tensor(x, dtype=torch.float64, device=dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        r64 = b.minimize_dev(x0, boxes, FTOL, MAXITER)
        ev1.record()
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1)
        its64 = sum(int(r.iterations) * int(n) for r, n in zip(r64, counts))
    order = np.argsort(counts, kind="stable")[::16]
    its1 = 0
    ms1 = 0.0
    conv1 = 0
    for s in order:
        c = cfgs[s]
        xs = torch.tensor(c.x, dtype=torch.float64, device=dev)
        ws = torch.empty_like(xs)
        with fg.FireHandle(c.n, fi.CU_MASS, pot64, dt_start=fi.CU_DT) as h:
            ws.copy_(xs)
            h.minimize_dev(ws, c.box, FTOL, MAXITER)
            ws.copy_(xs)
            torch.cuda.synchronize()
            ev0.record()
            r = h.minimize_dev(ws, c.box, FTOL, MAXITER)
            ev1.record()
            torch.cuda.synchronize()
        ms1 += ev0.elapsed_time(ev1)
        its1 += int(r.iterations) * c.n
        conv1 += int(r.stop == fg.FIRE_STOP_FTOL)
    return {"fp64_max_force_of_fp32pair_structures": fmax64,
            "fp64_batched": {"value": its64 / (ms64 * 1e-3), "unit": UNIT, "ms": ms64,
                             "tuning": tune64,
                             "converged": int(sum(r.stop == fg.FIRE_STOP_FTOL for r in r64))},
            "fp64_single_system_path": {"value": its1 / (ms1 * 1e-3), "unit": UNIT,
                                        "sample": f"{len(order)} of 512 systems, every 16th by size, "
                                                  "one fire_minimize each", "converged": conv1}}


def grad_block(fg, torch, dev):
    """The differentiable form on its workload, the 20^3-cell Cu box with one
    vacancy (31,999 atoms): the structure relaxed to max|F_i| < 1e-10 eV/A,
    then the hand-written backward (E, F and dE/dtheta in one call), the
    Hessian-vector product, and the implicit gradient dL/dtheta of the
    vacancy loss (sum over the atoms whose lattice site lies within 6 A of
    the vacancy of |x - x_lattice|^2) by CG to a relative residual 1e-10;
    milliseconds per call (the calls synchronise their stream; CUDA events
    around them)."""
    c = fi.rgl_vacancy_box(ncell=20, seed=5, n_vac=1)
    theta = [fi.RGL_CU[k] for k in ("A", "xi", "p", "q")]
    pot = fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **fi.RGL_CU)
    x = torch.tensor(c.x, dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            out = fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps, out

    with fg.FireHandle(c.n, fi.CU_MASS, pot, dt_start=fi.CU_DT) as h:
        r = h.minimize_dev(x, c.box, 1e-10, 400000)
        f = torch.empty_like(x)
        ms_eg, (e, de) = timed(lambda: fg.fire_rgl_energy_grad_dev(h.h, x, c.box, theta, f), 10)
        u = torch.randn(x.shape, dtype=torch.float64, device=dev,
                        generator=torch.Generator(device=dev).manual_seed(7))
        hu = torch.empty_like(x)
        ms_hvp, _ = timed(lambda: fg.fire_rgl_hvp_dev(h.h, x, c.box, theta, u, hu), 20)
        site = c.meta["vacancy_sites"][0]
        d = c.meta["lattice"] - site
        d -= c.box * np.rint(d / c.box)
        sel = np.flatnonzero(np.sum(d * d, 1) < 36.0)
        dd = x.cpu().numpy()[sel] - c.meta["lattice"][sel]
        dd -= c.box * np.rint(dd / c.box)
        g = np.zeros((c.n, 3))
        g[sel] = 2.0 * dd
        gd = torch.tensor(g, dtype=torch.float64, device=dev)
        ms_ig, (dl, cg_it) = timed(
            lambda: fg.fire_rgl_implicit_grad_dev(h.h, x, c.box, theta, gd, 1e-10), 3)
    return {"workload": f"Cu 20^3 cells, 1 vacancy ({c.n} atoms), FP64, relaxed to "
                        f"max|F_i| < 1e-10 eV/A ({r.iterations} iterations)",
            "energy_grad_ms": ms_eg, "hvp_ms": ms_hvp,
            "hvp_atoms_per_s": c.n / (ms_hvp * 1e-3),
            "implicit_grad_ms": ms_ig, "cg_iterations": cg_it,
            "dL_dtheta": {k: float(v) for k, v in zip(("A", "xi", "p", "q"), dl)},
            "dE_dtheta": {k: float(v) for k, v in zip(("A", "xi", "p", "q"), de)}}


def relax_timed(fg, torch, dev, stream, cfg, pot, mass, dt, ftol, steps=5, warmup=3, **hkw):
    """Median time-to-ftol of `steps` relaxations of cfg from its initial
    configuration (after `warmup` untimed ones): CUDA events on the launching
    stream around each fire_minimize_dev call (which synchronises its stream),
    and the host wall time of the same calls.  Returns (result dict, the
    relaxed positions of the last step)."""
    x0 = torch.tensor(cfg.x, dtype=torch.float64, device=dev)
    work = torch.empty_like(x0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev_ms, host_ms, res = [], [], None
    with fg.FireHandle(cfg.n, mass, pot, dt_start=dt, **hkw) as h:
        for k in range(warmup + steps):
            work.copy_(x0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev0.record(stream)
            r = h.minimize_dev(work, cfg.box, ftol, MAXITER, stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if k >= warmup:
                dev_ms.append(ev0.elapsed_time(ev1))
                host_ms.append(1e3 * (t1 - t0))
                res = r
    med = statistics.median(dev_ms)
    return ({"value": cfg.n * res.iterations / (med * 1e-3), "unit": UNIT,
             "time_to_ftol_ms": med, "time_to_ftol_host_ms": statistics.median(host_ms),
             "times_ms": [round(t, 4) for t in dev_ms], "iterations": int(res.iterations),
             "force_evals": int(res.force_evals), "stop": int(res.stop),
             "final_fmax_atom": res.fmax_atom, "energy_per_atom": res.energy / cfg.n},
            work)


def ieee_check(fg, torch, dev, cfg, x):
    """max_i |F_i| and E/N of positions x (CUDA) with the IEEE-FP64 kernels."""
    pot = fg.Potential(fg.FIRE_POT_RGL, skin=0.3, pair_eval=fg.FIRE_PAIR_ANALYTIC, **fi.RGL_CU)
    with fg.FireHandle(cfg.n, fi.CU_MASS, pot, dt_start=fi.CU_DT) as hv:
        fv = torch.empty_like(x)
        ev = torch.zeros(1, dtype=torch.float64, device=dev)
        fg.fire_energy_forces_dev(hv.h, x, cfg.box, fv, ev)
        torch.cuda.synchronize()
    return float(torch.linalg.norm(fv, dim=1).max().item()), float(ev.item()) / cfg.n


def lj_block(fg, torch, dev, stream):
    """Config 1: the LJ FCC 4^3-cell box with one vacancy (255 atoms, uniform
    +-0.1 sigma noise, seed 1), FP64, Table 1 parameters with dt_start =
    0.005 tau, relaxed to max_i |F_i| < 1e-8: time-to-ftol (median of 5 after
    3 warm-up relaxations), iterations and atom-iterations per second."""
    cfg = CONFIGS["lj256"]()
    pot, mass, dt, ftol = potential_for("lj256")
    r, _ = relax_timed(fg, torch, dev, stream, cfg, pot, mass, dt, ftol)
    r.update({"workload": f"{cfg.name} ({cfg.n} atoms), LJ shifted rc = 2.5 sigma, FP64, "
                          f"max|F_i| < {ftol:g}", "atoms": cfg.n, "ftol": ftol})
    return r


def rgl32k_block(fg, torch, dev, stream):
    """Config 2: the RGL-Cu FCC 20^3-cell box with 1 % vacancies (31,680
    atoms, Gaussian 0.05 A noise, seed 2) relaxed to max_i |F_i| < 1e-6 eV/A
    in the FP64 form (double-float table terms, the library default) and the
    FP32-pair form (finishing in FP64 from 3 ftol on, the library default); each relaxed
    structure re-evaluated with the IEEE-FP64 kernels."""
    cfg = CONFIGS["rgl32k"]()
    out = {"workload": f"{cfg.name} ({cfg.n} atoms), RGL Cu, max|F_i| < {FTOL:g} eV/A",
           "atoms": cfg.n, "ftol": FTOL}
    for form, pair in (("fp64", "table"), ("fp32pair", "analytic")):
        pot, mass, dt, ftol = potential_for("rgl32k", form)
        pot.pair_eval = fg.FIRE_PAIR_ANALYTIC if pair == "analytic" else fg.FIRE_PAIR_TABLE
        r, x = relax_timed(fg, torch, dev, stream, cfg, pot, mass, dt, ftol)
        r["pair_eval"] = pair
        r["final_fmax_atom_ieee_fp64_check"], r["energy_per_atom_ieee_fp64_check"] = \
            ieee_check(fg, torch, dev, cfg, x)
        out[form] = r
    return out


def _timed_oracle(fn, threads):
    import oracle
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    out = fn()
    return out, time.perf_counter() - t0


def cpu_oracle_block(gpu, full_single=False):
    """The FP64 CPU oracle as it stands, timed on this host's cores for the
    small configurations: on all cores and on one thread.  `gpu` carries the
    GPU iteration counts used where a single-thread run is a bounded sample
    (per-iteration time x iterations, marked "estimate").  The oracle runs
    all-pairs forces for boxes under 3 cells per axis, else its cell grid
    (bit-identical to all-pairs, tested)."""
    import oracle
    oracle.build()
    allc = oracle.max_threads()
    out = {"host": host_cpu(), "threads_all": allc}
    lj = oracle.Potential("lj", eps=1.0, sigma=1.0, rc_lj=2.5)
    cu = oracle.Potential("rgl", **fi.RGL_CU)
    plj, pcu = oracle.Params(dt_start=fi.LJ_DT), oracle.Params(dt_start=fi.CU_DT)

    def mode(c, rc):
        return (oracle.FORCE_CELLS if np.all(np.floor(np.asarray(c.box) / rc) >= 3)
                else oracle.FORCE_BRUTE)

    def entry(n, iters, secs, kind, note):
        return {"seconds": round(secs, 3), "iterations": int(iters), "kind": kind,
                "value": n * iters / secs, "unit": UNIT, "note": note}

    try:
        # config 1: both in full
        c = CONFIGS["lj256"]()
        blk = {"atoms": c.n}
        for th, key in ((allc, "all_cores"), (1, "one_thread")):
            (x, r, _), t = _timed_oracle(lambda: oracle.fire2(
                c.x, c.box, lj, plj, fi.LJ_MASS, 1e-8, MAXITER, mode=oracle.FORCE_BRUTE), th)
            blk[key] = entry(c.n, r.iterations, t, "full",
                             f"whole relaxation to max|F_i| < 1e-8, {th} thread(s)")
            blk["energy_per_atom"] = r.energy / c.n
        out["lj256"] = blk

        # config 2: all cores in full; one thread in full or as a sample
        c = CONFIGS["rgl32k"]()
        blk = {"atoms": c.n}
        (x, r, _), t = _timed_oracle(lambda: oracle.fire2(
            c.x, c.box, cu, pcu, fi.CU_MASS, FTOL, MAXITER, mode=oracle.FORCE_CELLS), allc)
        blk["all_cores"] = entry(c.n, r.iterations, t, "full",
                                 f"whole relaxation to max|F_i| < {FTOL:g} eV/A, {allc} threads")
        blk["energy_per_atom"] = r.energy / c.n
        its_full = r.iterations
        if full_single:
            (x, r1, _), t = _timed_oracle(lambda: oracle.fire2(
                c.x, c.box, cu, pcu, fi.CU_MASS, FTOL, MAXITER, mode=oracle.FORCE_CELLS), 1)
            blk["one_thread"] = entry(c.n, r1.iterations, t, "full",
                                      "whole relaxation, 1 thread")
        else:
            k = 8
            (_, r1, _), t = _timed_oracle(lambda: oracle.fire2(
                c.x, c.box, cu, pcu, fi.CU_MASS, 0.0, k, mode=oracle.FORCE_CELLS), 1)
            per_eval = t / (k + 1)
            blk["one_thread"] = entry(c.n, its_full, per_eval * (its_full + 1), "estimate",
                                      f"{k} FIRE iterations (+1 initial evaluation) timed on 1 "
                                      f"thread ({t:.1f} s); the remaining "
                                      f"{its_full - k} of the oracle's {its_full} iterations "
                                      "extrapolated at the same time per evaluation")
        out["rgl32k"] = blk

        # config 5: relaxation to 1e-10 eV/A + implicit gradient (CG to 1e-10)
        c = fi.rgl_vacancy_box(ncell=20, seed=5, n_vac=1)
        blk = {"atoms": c.n}
        site = c.meta["vacancy_sites"][0]
        d = c.meta["lattice"] - site
        d -= c.box * np.rint(d / c.box)
        sel = np.flatnonzero(np.sum(d * d, 1) < 36.0)

        def grad_pipeline(ftol_relax, maxiter, cg_maxit):
            xr, rr, _ = oracle.fire2(c.x, c.box, cu, pcu, fi.CU_MASS, ftol_relax, maxiter,
                                     mode=oracle.FORCE_CELLS)
            t_relax = time.perf_counter()
            dd = xr[sel] - c.meta["lattice"][sel]
            dd -= c.box * np.rint(dd / c.box)
            g = np.zeros_like(xr)
            g[sel] = 2.0 * dd
            try:
                lam, it = oracle.rgl_cg(xr, c.box, cu, g, 1e-10, cg_maxit, mode=oracle.FORCE_CELLS)
            except RuntimeError:
                it = cg_maxit
            _ = oracle.rgl_param_derivs(xr, c.box, cu, mode=oracle.FORCE_CELLS)
            return rr, it, t_relax

        t0 = time.perf_counter()
        oracle.set_threads(allc)
        rr, cg_it, t_mid = grad_pipeline(1e-10, MAXITER, 20000)
        t1 = time.perf_counter()
        blk["all_cores"] = {"seconds": round(t1 - t0, 3), "relax_seconds": round(t_mid - t0, 3),
                            "fire_iterations": int(rr.iterations), "cg_iterations": int(cg_it),
                            "kind": "full", "note": f"relaxation to max|F_i| < 1e-10 eV/A, CG "
                                                    f"to 1e-10, dF/dtheta; {allc} threads"}
        if full_single:
            oracle.set_threads(1)
            t0 = time.perf_counter()
            rr1, cg1, t_mid = grad_pipeline(1e-10, MAXITER, 20000)
            blk["one_thread"] = {"seconds": round(time.perf_counter() - t0, 3), "kind": "full",
                                 "fire_iterations": int(rr1.iterations),
                                 "cg_iterations": int(cg1)}
        else:
            oracle.set_threads(1)
            k, kc = 4, 4
            t0 = time.perf_counter()
            rr1, _, t_mid = grad_pipeline(0.0, k, kc)
            t1 = time.perf_counter()
            per_eval = (t_mid - t0) / (k + 1)
            per_cg = (t1 - t_mid) / kc      # includes dF/dtheta once (small)
            est = per_eval * (rr.iterations + 1) + per_cg * cg_it
            blk["one_thread"] = {"seconds": round(est, 3), "kind": "estimate",
                                 "note": f"{k} FIRE iterations ({t_mid - t0:.1f} s) and {kc} CG "
                                         f"iterations ({t1 - t_mid:.1f} s) timed on 1 thread, "
                                         f"extrapolated to the all-core run's "
                                         f"{rr.iterations} FIRE and {cg_it} CG iterations"}
        out["grad32k"] = blk

        # config 4: 16 of the 512 boxes (every 32nd by size) relaxed in full
        cfgs = fi.rgl_batch(n_sys=512, seed=4)
        sizes = np.array([cc.n for cc in cfgs])
        pick = np.argsort(sizes, kind="stable")[16::32]
        oracle.set_threads(allc)
        t0 = time.perf_counter()
        ai = 0
        for sidx in pick:
            cc = cfgs[sidx]
            _, rb, _ = oracle.fire2(cc.x, cc.box, cu, pcu, fi.CU_MASS, FTOL, MAXITER,
                                    mode=mode(cc, fi.RGL_CU["rc"] + 0.3))
            ai += cc.n * rb.iterations
        t = time.perf_counter() - t0
        rate = ai / t
        blk = {"systems_sampled": len(pick), "atoms_sampled": int(sizes[pick].sum()),
               "all_cores": {"value": rate, "unit": UNIT, "seconds": round(t, 3),
                             "kind": "sample",
                             "note": f"16 of the 512 boxes (every 32nd by size) relaxed in full "
                                     f"on {allc} threads"}}
        if gpu.get("batch_atom_iters"):
            blk["all_cores"]["estimate_512_seconds"] = gpu["batch_atom_iters"] / rate
        med = cfgs[pick[len(pick) // 2]]
        oracle.set_threads(1)
        t0 = time.perf_counter()
        _, rb, _ = oracle.fire2(med.x, med.box, cu, pcu, fi.CU_MASS, FTOL, MAXITER,
                                mode=mode(med, fi.RGL_CU["rc"] + 0.3))
        t = time.perf_counter() - t0
        blk["one_thread"] = {"value": med.n * rb.iterations / t, "unit": UNIT,
                             "seconds": round(t, 3), "kind": "sample",
                             "note": f"the median-size sampled box ({med.n} atoms) relaxed in "
                                     "full on 1 thread"}
        if gpu.get("batch_atom_iters"):
            blk["one_thread"]["estimate_512_seconds"] = \
                gpu["batch_atom_iters"] / blk["one_thread"]["value"]
        out["batch512"] = blk
    finally:
        oracle.set_threads(allc)
    return out


INTEGRATORS = {"semi_implicit_euler": 0, "explicit_euler": 1, "velocity_verlet": 2, "leapfrog": 3}


def study_block(fg, torch, dev):
    """The paper's comparisons (Sec. 5), repeated through the GPU path on
    synthetic stand-ins: force evaluations to the stopping force for FIRE 2.0
    (Algorithm 2) and the original FIRE (Algorithm 1) with each integrator
    (Algorithms 3-6) on the LJ vacancy box, the 32k Cu vacancy box and a Si
    slab with five vacancies (Stillinger-Weber, periodic in x and y -- the
    structure of the paper's silicon vacancy case); then on that slab the
    sweeps of alpha0 x tmax at dt = 1 fs and of tmax x dt at alpha0 = 0.15."""
    work = [
        ("lj_fcc4_vac1", fi.lj_fcc_vacancy(),
         fg.Potential(fg.FIRE_POT_LJ, eps=1.0, sigma=1.0, rc_lj=2.5, skin=0.3),
         fi.LJ_MASS, fi.LJ_DT, 1e-8),
        ("rgl_cu20_vac320", fi.rgl_vacancy_box(),
         fg.Potential(fg.FIRE_POT_RGL, skin=0.3, **fi.RGL_CU), fi.CU_MASS, fi.CU_DT, FTOL),
        ("sw_si_slab16_vac5", fi.sw_si_slab(),
         fg.Potential(fg.FIRE_POT_SW, skin=0.3, **fi.SW_SI), fi.SI_MASS, fi.SI_DT, FTOL),
    ]
    cap = 20000

    def run(c, pot, mass, ftol, **prm):
        x0 = torch.tensor(c.x, dtype=torch.float64, device=dev)
        with fg.FireHandle(c.n, mass, pot, periodic=c.periodic, **prm) as h:
            r = h.minimize_dev(x0, c.box, ftol, cap)
        return {"force_evals": int(r.force_evals),
                "stop": {fg.FIRE_STOP_FTOL: "ftol", fg.FIRE_STOP_MAXITER: "maxiter",
                         fg.FIRE_STOP_MAXVDOTF: "maxvdotf"}.get(r.stop, str(r.stop)),
                "fmax_atom": r.fmax_atom, "energy_per_atom": r.energy / c.n}

    out = {"maxiter": cap, "integrators": {}, "sweeps": {}}
    for name, c, pot, mass, dt, ftol in work:
        rows = {}
        for var_name, var in (("fire2", fg.FIRE_VARIANT_FIRE2), ("fire1", fg.FIRE_VARIANT_FIRE1)):
            for iname, integ in INTEGRATORS.items():
                rows[f"{var_name}/{iname}"] = run(c, pot, mass, ftol, dt_start=dt,
                                                  integrator=integ, variant=var)
        out["integrators"][name] = {"atoms": c.n, "ftol": ftol, "runs": rows}
    _, c, pot, mass, dt, ftol = work[2]
    tmaxs = [2, 4, 6, 8, 10, 12, 15, 20]
    out["sweeps"]["alpha0_x_tmax_dt1fs"] = {
        f"{a0:g}/{tm:g}": run(c, pot, mass, ftol, dt_start=dt, alpha0=a0, tmax=tm)["force_evals"]
        for a0 in (0.05, 0.10, 0.15, 0.20, 0.25, 0.30, 0.40) for tm in tmaxs}
    out["sweeps"]["tmax_x_dt_alpha0_0.15"] = {
        f"{d * 1e3:g}fs/{tm:g}": run(c, pot, mass, ftol, dt_start=d, alpha0=0.15,
                                     tmax=tm)["force_evals"]
        for d in (0.0005, 0.001, 0.002, 0.004) for tm in tmaxs}
    return out


def roofline_block(fg, args, is_rgl, pair, stages, pairs, workload="rgl1m", n=0):
    """Roofline of the dominant pair kernel against a measured hardware peak.
    No pass is HBM-bound (DRAM 5-15 % in every ncu capture), so the bound is
    the arithmetic unit the kernel issues on: the measured FP32 FMA rate for
    the double-float and FP32-pair kernels, the measured FP64 FMA rate for
    the IEEE-FP64 ones.  achieved = the method's FLOPs per pair (exponentials,
    taper, sums; METHOD_FLOP_PER_PAIR) x pairs within rc / the kernel's mean
    CUDA-event time."""
    if is_rgl:
        dom = "density" if stages["density"] >= stages["force"] else "force"
        kernels = (TILED_KERNELS if tiles_active(args, args.form, pair, n)
                   else STAGE_KERNELS[(args.form, pair)])
        kname, unit = kernels[dom]
        key = dom
    else:
        dom, kname, unit, key = "force", "k_force_lj", "fp64", "force_lj"
    flop = METHOD_FLOP_PER_PAIR[key] * pairs
    achieved = flop / (stages[dom] * 1e-3)
    fp32 = fg.fire_diag_fma_peak(1)
    fp64 = fg.fire_diag_fma_peak(0)
    peak = fp64 if unit == "fp64" else fp32
    src = ("measured %s FMA issue rate on this GPU (fire_diag_fma_peak, FMA = 2 FLOP)"
           % ("FP64" if unit == "fp64" else "FP32"))
    out = {"bound": "alu", "kernel": kname, "achieved": achieved / 1e12, "peak": peak / 1e12,
           "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": src,
           "pipe": {"ff": "FP32 (double-float arithmetic)", "fp32": "FP32",
                    "fp64": "FP64"}[unit],
           "flop_per_pair": METHOD_FLOP_PER_PAIR[key], "flop_count": "method (per pass)",
           "transcendentals_per_pair": TRANSCENDENTALS_PER_PAIR[key],
           "pairs_within_rc": pairs, "stage_ms": stages,
           "fp64_peak": fp64 / 1e12, "fp32_peak": fp32 / 1e12,
           "vs_fp64_peak": achieved / fp64}
    if unit == "ff":
        # the emulation's own ceiling: one double-float multiply-add is 15 FP32
        # instructions; not a hardware roof
        out["emulation_efficiency"] = achieved / (fp32 / FF_FP32_PER_FMA)
    ncu = read_ncu(kname, workload)
    out["traffic"] = (ncu or {}).get("dram_bytes")
    out["ncu"] = ncu
    if ncu and ncu.get("dram_bytes") and ncu.get("time_ms"):
        # DRAM bytes the kernel moved (ncu) over its ncu duration
        out["dram_gbs_ncu"] = ncu["dram_bytes"] / (ncu["time_ms"] * 1e-3) / 1e9
    return out


def run_gpu(args):
    import torch

    import paper_1908_02038_gb300 as fg

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    fg.build()
    fg.load_library()

    cfg = CONFIGS[args.config]()
    n = cfg.n
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    pair = args.pair or default_pair(args.form)
    fp32 = args.form == "fp32pair"
    is_rgl = not args.config.startswith("lj")
    if args.study:
        print(json.dumps(study_block(fg, torch, dev)))
        return
    if args.batch_only:
        print(json.dumps(batch_block(fg, torch, dev, steps=1, tuning=args.batch_tuning,
                                     compare=False)))
        return
    if args.eval_only:
        pot, mass, dt, _ = potential_for(args.config, args.form)
        pot.pair_eval = fg.FIRE_PAIR_ANALYTIC if pair == "analytic" else fg.FIRE_PAIR_TABLE
        h = fg.FireHandle(n, mass, pot, dt_start=dt)
        h.set_pair_tiles(TILE_MODES[args.tiles])
        t0 = time.perf_counter()
        e, _ = h.energy_forces(cfg.x, cfg.box)
        print(json.dumps({"eval_only": cfg.name, "atoms": n, "energy": e,
                          "seconds": time.perf_counter() - t0}))
        h.close()
        return

    barrier = (lambda: __import__("torch.distributed").distributed.barrier()) if world > 1 else (lambda: None)
    barrier()
    m, h, x_relaxed = relax_form(fg, torch, cfg, args.form, pair, args, dev, stream)
    barrier()
    pot, ftol, results = m["pot"], m["ftol"], m["results"]
    ms = m["ms"]
    iters_total = sum(rr["iterations"] for rr in results)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        it = torch.tensor([iters_total], device=dev, dtype=torch.float64)
        dist.all_reduce(it)
        iters_total_all = float(it.item())
    else:
        iters_total_all = float(iters_total)
    value = n * iters_total_all / (ms * 1e-3)
    rc = pot.rc if is_rgl else pot.rc_lj
    cell_mode = bool(np.all(np.floor(np.asarray(cfg.box) / (rc + pot.skin)) >= 3))

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": ("f32-pair/f64" if fp32 else
                     ("f64 (pair terms: int64 fixed point + double-float)" if is_rgl and pair == "table"
                      else "f64")),
           "data": "synthetic",
           "config": {"workload": f"{cfg.name} ({n} atoms), FIRE2 + semi-implicit Euler to "
                                  f"max|F_i| < {ftol:g}",
                      "atoms": n, "ftol": ftol, "form": args.form, "skin": pot.skin,
                      "exec": args.exec, "pair_eval": pair, "newton": args.newton,
                      "tiles": tiles_active(args, args.form, pair, n),
                      "iterations_per_step": [rr["iterations"] for rr in results],
                      "final_fmax_atom": [rr["fmax_atom"] for rr in results],
                      "final_energy_per_atom": [rr["energy"] / n for rr in results],
                      "nbr_builds": [rr["nbr_builds"] for rr in results],
                      "l2": "inputs larger than L2 (working set > 1 GB at 1M atoms)"},
           "gpu_launches": launches_of(results, is_rgl, fp32, cell_mode, args.exec == "chunked",
                                       tiles_active(args, args.form, pair, n)),
           "clocks": m["clocks"]}

    # per-stage device times (CUDA events) for the roofline of the dominant kernel
    stages = h.profile_stages(cfg.x, cfg.box, reps=5)
    pairs = count_pairs(cfg.x, cfg.box, rc)
    out["roofline"] = roofline_block(fg, args, is_rgl, pair, stages, pairs, n=n)
    # HBM roofline of the whole iteration, as the metric asks
    alg_b = ALG_BYTES_PER_ATOM_ITER["rgl" if is_rgl else "lj"]
    try:
        hbm, hsrc = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"], "measured"
    except Exception:
        hbm, hsrc = 6800.0, "fallback"
    out["hbm_roofline"] = {"alg_bytes_per_atom_iter": alg_b,
                           "achieved_gbs": value * alg_b / 1e9, "peak_gbs": hbm,
                           "peak_source": hsrc, "frac": value * alg_b / 1e9 / hbm}

    # end to end through the host-pointer API (H2D of positions, D2H of
    # result), the positions in pinned host memory
    if not args.no_e2e:
        xh = torch.empty(cfg.x.shape, dtype=torch.float64, pin_memory=True).numpy()
        t_e2e, it_e2e = 0.0, 0
        for k in range(max(1, args.steps)):
            xh[...] = cfg.x
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = h.minimize(xh, cfg.box, ftol, MAXITER)
            t_e2e += time.perf_counter() - t0
            it_e2e += r.iterations
        out["e2e"] = {"value": n * it_e2e / t_e2e, "unit": UNIT,
                      "h2d_bytes_per_step": int(cfg.x.nbytes) + 1024,
                      "d2h_bytes_per_step": int(cfg.x.nbytes) + 1024}
    h.close()

    # the other forms on the same workload, each relaxed state re-evaluated
    # with the IEEE FP64 exponential pair terms (k_density / k_force_rgl)
    if is_rgl and not args.no_forms and world == 1:
        # (form, pair evaluation, FP32-pair FP64 check): the FP32-pair form
        # with the library's default (FP64 from 3 ftol on) and with one FP64
        # confirmation of each stop on ftol
        others = [f for f in (("fp32pair", "analytic", None), ("fp64", "analytic", None),
                              ("fp64", "table", None))
                  if f[:2] != (args.form, pair)][:2]
        if args.form != "fp32pair":
            others.append(("fp32pair", "analytic", fg.FIRE_FP64_CHECK_CONFIRM))
        pot64, mass, dt, _ = potential_for(args.config, "fp64")
        pot64.pair_eval = fg.FIRE_PAIR_ANALYTIC
        out["forms"] = {}
        with fg.FireHandle(n, mass, pot64, dt_start=dt) as hv:
            def check(x):
                fv = torch.empty_like(x)
                ev = torch.zeros(1, dtype=torch.float64, device=dev)
                fg.fire_energy_forces_dev(hv.h, x, cfg.box, fv, ev)
                return float(torch.linalg.norm(fv, dim=1).max().item()), float(ev.item())
            fmax_head, e_head = check(x_relaxed)
            out["config"]["final_fmax_atom_ieee_fp64_check"] = fmax_head
            for oform, opair, ocheck in others:
                m2, h2, x2 = relax_form(fg, torch, cfg, oform, opair, args, dev, stream,
                                        clocks=False, confirm64=ocheck)
                h2.close()
                ms2 = m2["ms"]
                it2 = sum(rr["iterations"] for rr in m2["results"])
                f64_fmax, e64 = check(x2)
                key = f"{oform}_{opair}" + ("_confirm64" if ocheck == fg.FIRE_FP64_CHECK_CONFIRM
                                            else "")
                out["forms"][key] = {
                    "value": n * it2 / (ms2 * 1e-3), "unit": UNIT,
                    "ms_per_step": ms2 / args.steps, "ftol": m2["ftol"],
                    "iterations_per_step": [rr["iterations"] for rr in m2["results"]],
                    "force_evals_per_step": [rr["force_evals"] for rr in m2["results"]],
                    "final_fmax_atom_own": [rr["fmax_atom"] for rr in m2["results"]],
                    "final_fmax_atom_ieee_fp64_check": f64_fmax,
                    "energy_per_atom_ieee_fp64_check": e64 / n,
                    "energy_per_atom_diff_vs_headline": (e64 - e_head) / n}
    if is_rgl and not args.no_small and world == 1:
        out["lj"] = lj_block(fg, torch, dev, stream)
        out["rgl32k"] = rgl32k_block(fg, torch, dev, stream)
    if is_rgl and not args.no_neb and world == 1:
        out["neb"] = neb_block(fg, torch, args.form, dev)
        out["sw"] = sw_block(fg, torch, dev)
        out["batched"] = batch_block(fg, torch, dev)
        out["grad"] = grad_block(fg, torch, dev)
    if rank == 0:
        if world == 1 and not args.no_cpu:
            cb = cpu_baseline(cfg, args)
            if is_rgl and not args.no_small:
                gpu = {}
                if "batched" in out:
                    gpu["batch_atom_iters"] = (out["batched"]["value"] *
                                               out["batched"]["ms_per_step"] * 1e-3)
                cb["configs"] = cpu_oracle_block(gpu, args.cpu_full)
                co = cb["configs"]
                # energy of each GPU relaxation against the oracle's own
                # relaxation of the same box (same ftol)
                out["lj"]["energy_err_vs_oracle_per_atom"] = \
                    out["lj"]["energy_per_atom"] - co["lj256"]["energy_per_atom"]
                out["lj"]["oracle_iterations"] = co["lj256"]["all_cores"]["iterations"]
                for form in ("fp64", "fp32pair"):
                    out["rgl32k"][form]["energy_err_vs_oracle_per_atom"] = \
                        out["rgl32k"][form]["energy_per_atom"] - co["rgl32k"]["energy_per_atom"]
                out["rgl32k"]["oracle_iterations"] = co["rgl32k"]["all_cores"]["iterations"]
            out["cpu_baseline"] = cb
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _oracle_setup(cfg):
    import oracle
    oracle.build()
    lj = cfg.name.startswith("lj")
    opot = (oracle.Potential("lj", eps=1.0, sigma=1.0, rc_lj=2.5) if lj
            else oracle.Potential("rgl", **fi.RGL_CU))
    mass = fi.LJ_MASS if lj else fi.CU_MASS
    params = oracle.Params(dt_start=fi.LJ_DT if lj else fi.CU_DT)
    return oracle, opot, mass, params


def _oracle_iterations_for(cfg, target_s):
    """Number of oracle FIRE iterations that take about target_s seconds."""
    oracle, opot, mass, params = _oracle_setup(cfg)
    t0 = time.perf_counter()
    oracle.fire2(cfg.x, cfg.box, opot, params, mass, 0.0, 1, mode=oracle.FORCE_CELLS)
    per_eval = (time.perf_counter() - t0) / 2.0     # initial evaluation + one iteration
    return max(1, int(target_s / max(per_eval, 1e-4)) - 1)


def cpu_sample(cfg, k):
    """The FP64 oracle as it stands, on the host cores: k FIRE iterations of the
    same configuration with the oracle's cell-grid forces."""
    oracle, opot, mass, params = _oracle_setup(cfg)
    t0 = time.perf_counter()
    _, r, _ = oracle.fire2(cfg.x, cfg.box, opot, params, mass, 0.0, k, mode=oracle.FORCE_CELLS)
    t = time.perf_counter() - t0
    return {"value": cfg.n * r.iterations / t, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle", "seconds": t,
            "sample": f"{r.iterations} FIRE iterations (+1 initial force evaluation) of the same "
                      f"{cfg.n}-atom box timed ({t:.1f} s), oracle cell-grid forces; the "
                      "metric divides the atom-iterations of that sample by its time, so no "
                      "whole relaxation is extrapolated"}


def cpu_baseline(cfg, args):
    return cpu_sample(cfg, _oracle_iterations_for(cfg, args.cpu_seconds))


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    cfg = CONFIGS[args.config]()
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    k = _oracle_iterations_for(cfg, per_step)
    for _ in range(args.warmup):
        cpu_sample(cfg, 1)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        cb = cpu_sample(cfg, k)
        secs += cb["seconds"]
        vals.append(cb["value"])
    v = statistics.median(vals)
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": f"{cfg.name} ({cfg.n} atoms), FP64 CPU oracle sample"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                            "sample": cb["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
