#!/usr/bin/env python
"""Throughput of the three-phase EHD lattice Boltzmann step on one B300.

Workload: compound drop deforming under a uniform field on a 4096 x 4096
lattice (outer radius 600, inner 300, electric capillary number 0.5,
permittivity 1:2:4, conductivity 1:0.5:0.25, surface-charge convection on), the
potential solved every step until the relative increments of psi and J of the
pseudo-time LB iteration (Eq. 42-45) are <= 1e-8.  By default the LB iteration
runs on an FP64 anchor with a multigrid coarse correction (the same discrete
fixed point as the plain iteration, reached in a few hundred iterations instead of
~1e5; `--potential lb` runs the plain iteration, which stalls on its FP32 rounding
floor at this size).  The line reports, over the timed steps, how many solves
reached the tolerance and the largest final residual.  A "step" is one full time
step: moments, stencils and charge closure, the potential solve, and the fused
chemical-potential/force/collide/stream pass.  Metric: MLUPS = cells x steps /
second (all population sets updated per cell per step).  Inputs are synthetic (the
stated initial condition, no dataset).

Other workloads (`--workload`): sweep (the batched parameter sweep), regimes (drop
pairs and confined shear as one batch), adjoint (tangent-mode derivatives), eof (the
electro-osmotic channel with Nernst-Planck ions), deformation3d (the D3Q15 step on a
256^3 compound drop).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lb3e|reference]
Under torchrun (N > 1) every rank steps its own replica (no data exchange: a
single lattice does not shard without a halo exchange); value = all ranks' cell
updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "MLUPS"
SOLVER_NAMES = {
    0: "LB pseudo-time iterations of Eq. 42-45, h in the build's precision",
    1: "multigrid V-cycles on the finite-difference form of Eq. 27d",
    2: "LB pseudo-time iterations of Eq. 42-45 on an FP64 anchor, multigrid coarse correction every check "
       "(fixed point of Eq. 43; stop on its increments)",
    3: "LB pseudo-time iterations of Eq. 42-45 on an FP64 anchor",
}
# algorithmic bytes per cell: the compulsory traffic of each kernel (every array it must
# read or write once per cell), not counting halo re-reads
FUSED_BYTES = {0: 8 * 112, 1: 4 * 112, 2: 2 * 90 + 4 * 22, 5: 2 * 90 + 4 * 22}  # k_fused: 45 pops r+w, phi, q, E, d/dt state
POISSON_BYTES = {0: 8 * 20, 1: 4 * 20, 2: 4 * 20, 5: 4 * 20}  # one pseudo-iteration: h 9 r + 9 w, eps, q
# one pseudo-iteration on the correction to the FP64 anchor: delta 9 r + 9 w, eps,
# and the anchor's increment (9 planes) instead of q
POISSON_RS_BYTES = {0: 8 * 28, 1: 4 * 28, 2: 4 * 28, 5: 4 * 28}
# one anchor refresh.  FP64 build (two launches): fold and FP64 collision (anchor 9 r +
# 9 w, delta 9 r + 9 w, eps, q, 9 FP64 staging planes written) and increment (anchor
# and staging read, 9 increment planes written).  FP32 builds (one launch, the
# double-float anchor in 8-byte words): anchor 9 r + 9 w, delta 9 r, eps, q, 9
# increment planes and the anchor's flux (2) written; delta is left for the coarse
# correction to overwrite
ANCHOR_BYTES = {0: 72 * 4 + 8 * 20 + 72 + 8 * 9, 1: 72 * 2 + 4 * (9 + 2 + 9 + 2)}
ANCHOR_LAUNCHES = {0: 2, 1: 1}
for _p in (2, 5):  # 16-bit population storage: FP32 arithmetic, FP32 potential
    ANCHOR_BYTES[_p], ANCHOR_LAUNCHES[_p] = ANCHOR_BYTES[1], ANCHOR_LAUNCHES[1]
STEP_BYTES = {0: 960, 1: 480, 2: 300, 5: 300}               # whole step without the potential loop
DTYPE_NAMES = {0: "f64", 1: "f32", 2: "f32 (f16-stored populations)", 5: "f32 (bf16-stored populations)"}
# multigrid cycle per fine cell (defect correction): the FP64 fine residual (psi,
# rhs, 3 coefficients read, residual written: 48 B), then the FP32 V-cycle on the
# error equation -- defect load (16 B), 4 red-black sweeps (e r/w, rhs, 3
# coefficients: 4 x 24 B), residual (24 B), restriction (5 B), prolongation (9 B),
# FP64 correction (20 B) -- times 4/3 for the coarser levels
MG_VCYCLE_BYTES = 48 + round(170 * 4 / 3)
# Nernst-Planck ions per cell and step, in units of the compute type: k_ion_moments
# reads 18 populations and writes n_1, n_2, q (21); k_ions reads 18 populations,
# n_i, u, E and (n_i v_i)^{n-1} (28) and writes 18 populations and (n_i v_i)^n (22)
ION_WORDS = {"k_ion_moments": 21, "k_ions": 50}
# with ions on, k_fused also writes u, p and mu (6 planes) every step
FUSED_DIAG_WORDS = 6
# three-dimensional (D3Q15) kernels per cell, in words of the compute type:
# k3_collide reads 75 populations, phi (3), q, E (3), mu (3), rho, sigma, eps and the
# d/dt history (12) and writes 75 populations and the history (100 + 87); one
# potential iteration reads 15 h, eps, q and writes 15 h (32); k3_moments reads 60
# populations and writes phi (3), q~, rho, sigma, eps (67)
WORDS_3D = {"fused": 187, "poisson": 32, "moments": 67}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lb3e", choices=["lb3e", "reference"])
    ap.add_argument("--workload", default="deformation",
                    choices=["deformation", "sweep", "adjoint", "regimes", "eof", "deformation3d"],
                    help="deformation: the 4096^2 lattice (default); sweep: 256 lattices in one batch; "
                         "adjoint: cost of the three parameter derivatives relative to a forward step")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2, 5],
                    help="0 fp64, 1 fp32, 2 fp32 + fp16-stored populations, 5 fp32 + bf16-stored populations")
    ap.add_argument("--n", type=int, default=4096, help="lattice side (the stated workload is 4096)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline (profiling runs)")
    ap.add_argument("--potential", default="lbmg", choices=["lb", "mg", "lbmg", "lba"],
                    help="lb: the paper's pseudo-time LB solve, h in the build's precision; mg: multigrid on its "
                         "FD form; lbmg: the LB solve on an FP64 anchor with a multigrid coarse correction; "
                         "lba: the LB solve on an FP64 anchor")
    ap.add_argument("--max-iter", type=int, default=0,
                    help="cap on LB potential iterations per step (default: the workload's 20000); profiling "
                         "runs use a small cap to keep ncu captures short, and config records it")
    ap.add_argument("--fused-tile", type=int, default=0,
                    help="rows of the fused pass's 32-wide tiles, 4, 8 or 16 (default: the library's, 4 in FP32)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="LB potential iterations per launch, 1..8 (default: the library's)")
    ap.add_argument("--check-every", type=int, default=0,
                    help="potential residual cadence (default: the workload's; 1 runs one iteration per launch)")
    return ap.parse_args()


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# the files the profiled kernels' device code is compiled from (host sequencing and
# the ABI layer do not enter it), hashed with the build's flags
KERNEL_SOURCES = ("lb3e_kernels.cuh", "lb3e_anchor.cuh", "lb3e_mg.cuh", "lb3e_params.cuh", "lb3e_dual.cuh",
                  "lb3e_f32.cu", "lb3e_f64.cu")


def check_interval(params: dict) -> int:
    """Iterations between increment checks (each reads 3 FP64 sums back): with the
    coarse correction (solver 2) the cycle of poisson_check_every iterations holds
    max(2, cycle / 16) checks."""
    c = max(1, int(params["poisson_check_every"]))
    if params.get("potential_solver") == 2 and c >= 16:
        return c // max(2, c // 16)
    return c


def kernel_source_hash() -> str:
    from paper_2608_05787_b300 import build as B
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update((ROOT / "paper_2608_05787_b300" / "csrc" / name).read_bytes())
    common = [a for i, a in enumerate(B.COMMON) if a != "-I" and (i == 0 or B.COMMON[i - 1] != "-I")]
    units = [(u, B.UNITS[u]) for u in KERNEL_SOURCES if u in B.UNITS]
    h.update(repr((B.ARCH, common, units)).encode())
    return h.hexdigest()[:16]


def profiled_record(key: str):
    """The committed ncu record of a kernel (profiles/traffic.json, keyed
    "<kernel>:<precision>[:<iterations per launch>]"), if it was taken on the current
    kernel sources (else None)."""
    f = ROOT / "profiles" / "traffic.json"
    if not f.exists():
        return None
    e = json.loads(f.read_text()).get(key)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e


def profiled_traffic(key: str):
    """DRAM bytes per cell and launch from the committed ncu record, or None."""
    e = profiled_record(key)
    return float(e["bytes_per_cell"]) if e else None


def issue_bound(key: str, cells: int, ms_per_launch: float, sm_mhz):
    """The on-chip figure of merit of an issue-bound kernel: its warp instructions per
    launch (the ncu record's per-cell count x cells) over the launch time, against
    the schedulers' ceiling of one warp instruction a cycle on each of the 148 SMs'
    four sub-partitions at the sampled SM clock."""
    e = profiled_record(key)
    if not e or "warp_instructions_per_cell" not in e or not sm_mhz:
        return None
    inst = float(e["warp_instructions_per_cell"]) * cells
    peak = 148 * 4 * float(sm_mhz) * 1e6
    rate = inst / (ms_per_launch / 1e3)
    return {"warp_instructions_per_launch": inst, "achieved_warp_inst_per_s": rate,
            "peak_warp_inst_per_s": peak, "frac": rate / peak, "sm_mhz": sm_mhz}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        rows = [r.split(",") for r in Path(self.f.name).read_text().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if len(r) > 5 + k and r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _oracle_sample(n: int, iters: int = 0, solver: int = 0, tol: float = 1e-8):
    """The oracle on an n^2 lattice of the deformation workload (radii scaled), with
    the LB potential iterated to `tol` each step (or a fixed count when iters > 0),
    or with its FD solve (solver 1)."""
    import oracle
    import workloads as W
    scale = n / 4096.0
    cfg = W.config_deformation(n=n, r_out=600.0 * scale, r_in=300.0 * scale)
    p = dict(cfg["params"], poisson_fixed_iter=iters, potential_solver=solver, poisson_tol=tol,
             poisson_max_iter=10 ** 7)
    return oracle.Oracle(p, cfg["phi"])


# side of the oracle's sample lattice: the plain LB iteration needs O(n^2) iterations
# a step, so the sample stays small enough for a bounded run
CPU_SAMPLE_LB = 128
CPU_SAMPLE_MG = 256
# the workload's potential tolerance (relative increment, every step)
WORKLOAD_TOL = 1e-8


def _time_oracle_steps(o, warmup: int, steps: int):
    o.step(warmup)
    iters, t = [], 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        o.step(1)
        t += time.perf_counter() - t0
        iters.append(o.last_poisson()[0])
    return t / steps, iters


def cpu_baseline(args, iters_per_step: float):
    """The oracle, as it stands, on the host cores, on a bounded sample of the
    workload: a small lattice with the geometry scaled and the same potential
    tolerance.  Measured step times (no projection), init untimed."""
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if getattr(args, "potential", "lbmg") == "mg":
        n = CPU_SAMPLE_MG
        o = _oracle_sample(n, solver=1)
        per_step, _ = _time_oracle_steps(o, 0, 1)
        sample = (f"one step of a {n}x{n} lattice of the same workload (radii scaled) with the oracle's FD "
                  "potential solve (conjugate gradients to 1e-13); init untimed")
        iters = None
    else:
        n = CPU_SAMPLE_LB
        o = _oracle_sample(n, tol=WORKLOAD_TOL)
        per_step, iters = _time_oracle_steps(o, 1, 2)
        sample = (f"2 steps (after 1 untimed) of a {n}x{n} lattice of the same workload (radii scaled), the "
                  f"oracle's plain LB potential iteration to the same relative increment {WORKLOAD_TOL:g} "
                  "every step (the same discrete fixed point as the GPU's solve); init untimed")
    return {"value": n * n / per_step / 1e6, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample,
            "projected": False, "seconds_per_step": per_step, "sample_potential_iters": iters}


def run_reference(args):
    """The oracle timed on the host cores for the same metric as the lb3e arm; rank 0
    only.  Each timed step is a measured step of a bounded sample of the workload: a
    small lattice with the geometry scaled, the potential solved to the same
    tolerance by the oracle's plain LB iteration (or, with --potential mg, its FD
    solve by conjugate gradients)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    mg = getattr(args, "potential", "lbmg") == "mg"
    if mg:
        n = min(CPU_SAMPLE_MG, args.n)
        o = _oracle_sample(n, solver=1)
        cfg = {"potential_solver": "FD form, conjugate gradients (oracle)"}
        sample = (f"{args.steps} timed steps of a {n}x{n} lattice of the same workload (radii scaled), the "
                  "oracle's FD potential solve (conjugate gradients to 1e-13)")
    else:
        n = min(CPU_SAMPLE_LB, args.n)
        o = _oracle_sample(n, tol=WORKLOAD_TOL)
        cfg = {"potential_solver": "LB pseudo-time iterations of Eq. 42-45, plain (oracle)",
               "poisson_tol": WORKLOAD_TOL}
        sample = (f"{args.steps} timed steps of a {n}x{n} lattice of the same workload (radii scaled), the "
                  f"potential iterated to the relative increment {WORKLOAD_TOL:g} every step")
    per_step, iters = _time_oracle_steps(o, args.warmup, args.steps)
    value = n * n / per_step / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (stated initial condition of the workload)",
            "config": dict({"workload": f"compound drop deformation under field, {args.n}x{args.n}",
                            "sample_side": n, "potential_iters_per_step": iters}, **cfg),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample,
                             "projected": False},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_sample(args):
    """The reference arm for the eof and deformation3d workloads: the oracle, as it
    stands, stepping a bounded sample of that workload on the host cores (rank 0)."""
    import oracle
    import workloads as W
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if args.workload == "eof":
        nx, ny = 1280, 256
        c = W.config_eof_channel(nx=nx, ny=ny, precision=0)
        o = oracle.Oracle(c["params"], c["phi"], ions=c["ions"])
        cells, name = nx * ny, f"electro-osmotic channel with Nernst-Planck ions, {nx}x{ny} sample of 10240x2048"
    else:
        m = 48
        c = W.config_deformation_3d(n=m, r_out=40.0 * m / 256, r_in=20.0 * m / 256, precision=0)
        o = oracle.Oracle3D(c["params"], c["phi"])
        cells, name = m ** 3, f"compound drop deformation under field, D3Q15, {m}^3 sample of 256^3"
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    per_step = (time.perf_counter() - t0) / max(1, args.steps)
    value = cells / per_step / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (as the lb3e arm)",
            "config": {"workload": name},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed steps of the {name} (radii scaled alike)"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_lb3e(args):
    import torch
    import paper_2608_05787_b300 as L
    import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    prec = args.precision
    cfg = W.config_deformation(n=args.n, r_out=600.0 * args.n / 4096, r_in=300.0 * args.n / 4096, precision=prec)
    params = cfg["params"]
    if args.check_every:
        params = dict(params, poisson_check_every=args.check_every)
    if args.max_iter:
        params = dict(params, poisson_max_iter=args.max_iter)
    if args.potential == "mg":
        params = dict(params, potential_solver=1, poisson_max_iter=50)
    elif args.potential in ("lbmg", "lba"):
        # a coarse correction (lbmg) every 48 iterations, with the increment checked
        # every 16; the plain anchored iteration (lba) checks every 16
        params = dict(params, potential_solver=2 if args.potential == "lbmg" else 3,
                      poisson_check_every=args.check_every or (48 if args.potential == "lbmg" else 16))
    N = args.n * args.n
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        phi_dev = torch.from_numpy(cfg["phi"]).cuda()
        t_init0 = time.perf_counter()
        sim = L.Sim(params, phi_dev, stream=stream)
        if args.chunk:
            sim.set_chunk(args.chunk)
        if args.fused_tile:
            sim.set_tile(args.fused_tile)
        t_init = time.perf_counter() - t_init0
        init_obs = sim.observables()
        sim.step(args.warmup)
        torch.cuda.synchronize()
        sim.potential_stats()
        sim.set_timing(True)
        l0 = sim.launches
        it0 = sim.potential_iterations
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            ev0.record(stream)
            sim.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        barrier()
        ms = ev0.elapsed_time(ev1)
        launches = sim.launches - l0
        pot_iters = sim.potential_iterations - it0
        kt = sim.kernel_times()
        sim.set_timing(False)
        pstats = sim.potential_stats()
        obs = sim.observables()
        fd_res = sim.fd_residual() if params["electric"] else None

    t = ms / 1e3
    if dist:
        tt = torch.tensor([t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    total_cells = N * args.steps * ws
    value = total_cells / t / 1e6

    hbm, peak_kind = peaks()
    fused_ms, fused_n = kt["fused"]
    iters_per_step = pot_iters / args.steps
    kernels = {}
    for name, (kms, kn) in kt.items():
        if kn:
            kernels[name] = {"launches": kn, "ms_total": kms, "share": kms / max(1e-12, sum(v[0] for v in kt.values()))}
    solver = int(params.get("potential_solver", 0))
    mg = solver == 1
    anchored = solver in (2, 3)
    chunk = args.chunk or 4
    # per kernel class: algorithmic bytes per launch (units x bytes per unit), the
    # mean launch time, the kernel that carries the class, and its unit
    classes = {}
    if fused_n:
        classes["fused"] = (FUSED_BYTES[prec] * N, fused_ms / fused_n, "k_fused", f"{N} cells")
    poisson_ms, poisson_n = kt["poisson"]
    if poisson_n and not mg:
        per_it = POISSON_RS_BYTES[prec] if anchored else POISSON_BYTES[prec]
        ipl = pot_iters / poisson_n
        kname = ("k_poisson_tb_rs" if chunk > 1 else "k_poisson_rs") if anchored else \
            ("k_poisson_tb" if chunk > 1 else "k_poisson")
        classes["poisson"] = (per_it * N * ipl, poisson_ms / poisson_n, kname,
                              f"{N} cells x {ipl:.2f} pseudo-iterations ({per_it} B per cell-iteration)")
    elif poisson_n:
        classes["poisson"] = (MG_VCYCLE_BYTES * N * pot_iters / poisson_n, poisson_ms / poisson_n,
                              "multigrid V-cycle kernels", f"{N} cells x V-cycles")
    anchor_ms, anchor_n = kt.get("anchor", (0.0, 0))
    refreshes = anchor_n / ANCHOR_LAUNCHES[prec]
    if anchor_n:
        classes["anchor"] = (ANCHOR_BYTES[prec] * N, anchor_ms / refreshes,
                             "k_anchor_refresh + k_anchor_residual" if ANCHOR_LAUNCHES[prec] == 2
                             else "k_anchor_refresh_pull_df", f"{N} cells, one refresh")
    k_gbs = {k: b / (t / 1e3) / 1e9 for k, (b, t, _, _) in classes.items()}
    dominant = max(classes, key=lambda k: kt[k][0])
    dbytes, dms, kname, units = classes[dominant]
    key = f"{kname}:{prec}" + (f":{chunk}" if kname in ("k_poisson_tb", "k_poisson_tb_rs") else "")
    traffic = None if kname.startswith("multigrid") else profiled_traffic(key)
    roofline = {"bound": "hbm", "achieved": k_gbs[dominant], "peak": hbm, "unit": "GB/s",
                "frac": k_gbs[dominant] / hbm, "traffic": traffic * N if traffic else None,
                "dram_frac": (traffic * N / (dms / 1e3) / 1e9 / hbm) if traffic else None,
                "kernel": kname, "peak_kind": f"{peak_kind} copy bandwidth",
                "algorithmic_bytes_per_launch": dbytes, "units_per_launch": units, "ms_per_launch": dms,
                "other_kernel_gbs": {k: v for k, v in k_gbs.items() if k != dominant}}
    # the whole step: fused step bytes (Section 8 figure) + potential iterations +
    # anchor refreshes, over the measured step time
    step_bytes = STEP_BYTES[prec] * N + (classes["poisson"][0] * poisson_n if "poisson" in classes else 0) / \
        args.steps + ANCHOR_BYTES[prec] * N * refreshes / args.steps
    step_roofline = {"bytes_per_step": step_bytes, "achieved": step_bytes / (ms / args.steps / 1e3) / 1e9,
                     "frac": step_bytes / (ms / args.steps / 1e3) / 1e9 / hbm}

    # end to end through the public API: pinned host initial fields, init (with its
    # potential solve), K steps each followed by an observables read-back.  The
    # workspace is the caller's, allocated before (the device-timed run's, reused).
    e2e = None
    if not args.no_e2e:
        work = sim.workspace
        del sim
        host_phi = torch.from_numpy(cfg["phi"]).pin_memory()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            s2 = L.Sim(params, host_phi, stream=stream, workspace=work)
            if args.chunk:
                s2.set_chunk(args.chunk)
            if args.fused_tile:
                s2.set_tile(args.fused_tile)
            for _ in range(args.steps):
                s2.step(1)
                s2.observables()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        barrier()
        if dist:
            tt = torch.tensor([t_e2e], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t_e2e = float(tt.item())
        e2e = {"value": total_cells / t_e2e / 1e6, "unit": METRIC,
               "h2d_bytes_per_step": int(3 * N * 8 / args.steps),
               "d2h_bytes_per_step": int(20 * 8 + 32 * math.ceil(iters_per_step / check_interval(params))),
               "includes": "init from pinned host fields (with its potential solve; workspace allocated before) + "
                           "per-step observables read-back",
               "seconds": t_e2e}
        del s2, work

    cpu = None
    if rank == 0 and not args.no_cpu:
        try:
            cpu = cpu_baseline(args, iters_per_step)
        except Exception as exc:  # a failed baseline must not hide the GPU line
            cpu = {"value": None, "error": repr(exc)}

    if rank == 0:
        dtype = DTYPE_NAMES[prec]
        clocks = clk.summary()
        roofline["issue"] = None if kname.startswith("multigrid") else issue_bound(key, N, dms, clocks.get("sm_mhz"))
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (stated initial condition of the workload)",
            "config": {"workload": f"compound drop deformation under field, {args.n}x{args.n}",
                       "poisson_tol": params["poisson_tol"], "poisson_max_iter": params["poisson_max_iter"],
                       "poisson_check_every": params["poisson_check_every"], "potential_chunk": chunk,
                       "potential_iters_per_step": iters_per_step,
                       "anchor_refreshes_per_step": refreshes / args.steps,
                       "potential_solver": SOLVER_NAMES[solver],
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single lattice",
                       "l2": "working set (%.1f GB) exceeds the 126 MB L2; no flush needed" % (L.workspace_bytes(params) / 1e9),
                       "init_seconds": t_init, "init_potential_iters": init_obs["poisson_iters"]},
            "roofline": roofline,
            "step_roofline": step_roofline,
            "kernels": kernels,
            "fused_mlups": N / (fused_ms / fused_n / 1e3) / 1e6 if fused_n else None,
            "step_bytes_per_cell_no_potential": STEP_BYTES[prec],
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "observables": {k: obs[k] for k in ("D_inner", "D_outer", "max_sum_dev", "poisson_residual",
                                                 "poisson_iters", "nonfinite")},
            "potential_timed_steps": dict(pstats, fd_residual_after=fd_res),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_sweep(args):
    """The batched parameter sweep: 256 compound drops of sides 128..512 stepped as
    one batch (one launch per kernel over all tiles, pairs of steps as a CUDA
    graph), 16 warm-started potential iterations per step.  Under torchrun the
    instances are sharded by cell count and only D is gathered."""
    import torch
    import paper_2608_05787_b300 as L
    import workloads as W
    from paper_2608_05787_b300.sweep import shard

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    insts = W.config_batched_sweep(precision=args.precision)
    cells = [i["shape"][0] * i["shape"][1] for i in insts]
    mine = shard(cells, ws)[rank]
    from paper_2608_05787_b300.autotune import tune_batch
    tuned = tune_batch([insts[i]["params"] for i in mine])
    chunk = tuned["chunk"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = L.Batch([insts[i]["params"] for i in mine], [W.sweep_phi(insts[i]) for i in mine], stream=stream)
        b.set_chunk(chunk).set_tile(tuned["tile"])
        b.run(args.warmup)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = b.launches
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            ev0.record(stream)
            b.run(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        obs = b.observables()
    t = ms / 1e3
    if dist:
        tt = torch.tensor([t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    total = sum(cells) * args.steps
    if rank == 0:
        hbm, peak_kind = peaks()
        per_cell = FUSED_BYTES[args.precision] + 16 * POISSON_BYTES[args.precision]
        line = {"metric": METRIC, "value": total / t / 1e6, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None,
                "dtype": DTYPE_NAMES[args.precision],
                "data": "synthetic (seeded sweep of the stated parameter ranges)",
                "config": {"workload": "batched sweep: 256 compound drops, sides {128,192,256,384,512}",
                           "cells": sum(cells), "potential_iters_per_step": 16, "autotuned_chunk": chunk,
                           "autotuned_fused_tile": f"32x{tuned['tile']}",
                           "parallelism": f"instances sharded over {ws} ranks" if ws > 1 else "one batch"},
                "roofline": {"bound": "hbm", "achieved": per_cell * total / t / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": per_cell * total / t / 1e9 / hbm, "traffic": None,
                             "kernel": "whole step (batched fused + 16 potential iterations)",
                             "peak_kind": f"{peak_kind} copy bandwidth"},
                "gpu_launches": b.launches - l0, "clocks": clk.summary(),
                "D_outer": {"min": min(o["D_outer"] for o in obs), "max": max(o["D_outer"] for o in obs)}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_regimes(args):
    """The second workload as one batch: the confined-shear grid (20 compound drops
    in channels of heights 80..200, Ca_E 0.2..1 x W_c 0.3..0.75, sliding electrode
    walls) and the two drop pairs (coalescence and separation, 256^2), 16
    warm-started potential iterations per step.  Reports MLUPS over the timed steps
    and the outcome measures at their end (a short horizon: the steady states take
    tens of capillary times, see the GPU tests)."""
    import torch
    import paper_2608_05787_b300 as L
    import workloads as W
    from paper_2608_05787_b300 import regimes as G

    torch.cuda.set_device(0)
    shear = W.config_shear_regimes(precision=args.precision)
    pairs = [W.config_two_drops(r, precision=args.precision) for r in ("coalescence", "separation")]
    insts = [(c["params"], c["phi"]) for c in shear] + [(c["params"], c["phi"]) for c in pairs]
    cells = sum(p["nx"] * p["ny"] for p, _ in insts)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = L.Batch([p for p, _ in insts], [phi for _, phi in insts], stream=stream).set_chunk(4)
        b.run(args.warmup)
        torch.cuda.synchronize()
        l0 = b.launches
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(0) as clk:
            ev0.record(stream)
            b.run(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        outcome = {"shear": [dict(wc=c["wc"], ca_e=c["ca_e"], drops=G.count_drops(b.field(i, "phinow1")),
                                  **{k: round(v, 4) for k, v in G.shape_measures(b.field(i, "phinow1")).items()})
                             for i, c in enumerate(shear)],
                   "pairs": [dict(regime=c["regime"], **{k: round(v, 3) for k, v in
                                                         G.pair_measures(b.field(len(shear) + k, "phinow1")).items()})
                             for k, c in enumerate(pairs)]}
    t = ms / 1e3
    total = cells * args.steps
    hbm, peak_kind = peaks()
    per_cell = FUSED_BYTES[args.precision] + 16 * POISSON_BYTES[args.precision]
    line = {"metric": METRIC, "value": total / t / 1e6, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_NAMES[args.precision],
            "data": "synthetic (the paper's drop-pair and confined-shear set-ups)",
            "config": {"workload": "second workload: 20 confined-shear channels + 2 drop pairs, one batch",
                       "cells": cells, "potential_iters_per_step": 16, "chunk": 4,
                       "steps_before_outcome": args.warmup + args.steps},
            "roofline": {"bound": "hbm", "achieved": per_cell * total / t / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": per_cell * total / t / 1e9 / hbm, "traffic": None,
                         "kernel": "whole step (batched fused + 16 potential iterations)",
                         "peak_kind": f"{peak_kind} copy bandwidth"},
            "gpu_launches": b.launches - l0, "clocks": clk.summary(), "outcome": outcome}
    print(json.dumps(line), flush=True)


def run_eof(args):
    """The electro-osmotic channel with Nernst-Planck ions (Eq. 52-53; 10240 x 2048,
    5:1 like the paper's channel): one phase, two ion species started in their
    double layers, the multigrid potential with the ions' charge every step, the
    fused flow/phase/charge pass and the ion pass.  MLUPS over the timed steps, the
    roofline of the dominant kernel class, the ion pass's own bandwidth, an end-to-end
    run from pinned host fields, and the oracle on a bounded sample."""
    import torch
    import paper_2608_05787_b300 as L
    import workloads as W

    torch.cuda.set_device(0)
    prec = args.precision
    cfg = W.config_eof_channel(precision=prec)
    params = cfg["params"]
    N = params["nx"] * params["ny"]
    word = 8 if prec == 0 else 4
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = L.Sim(params, torch.from_numpy(cfg["phi"]).cuda(), ions=torch.from_numpy(cfg["ions"]).cuda(),
                    stream=stream)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        sim.set_timing(True)
        l0 = sim.launches
        it0 = sim.potential_iterations
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(0) as clk:
            ev0.record(stream)
            sim.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = sim.launches - l0
        cycles = sim.potential_iterations - it0
        kt = sim.kernel_times()
        sim.set_timing(False)
        obs = sim.observables()
        mass = [float(sim.field(k).sum()) for k in ("n1", "n2")]
    t = ms / 1e3
    total = N * args.steps
    hbm, peak_kind = peaks()
    per_cell = {"fused": FUSED_BYTES[prec] + FUSED_DIAG_WORDS * word, "ions": sum(ION_WORDS.values()) * word,
                "poisson": MG_VCYCLE_BYTES}
    gbs = {}
    for k in ("fused", "ions"):
        kms, kn = kt[k]
        if kn:
            gbs[k] = per_cell[k] * N * args.steps / (kms / 1e3) / 1e9
    pms, pn = kt["poisson"]
    if pn and cycles:
        # per V-cycle and fine cell (the unit of the multigrid figure), over the V-cycle kernels' time
        gbs["poisson"] = MG_VCYCLE_BYTES * N * cycles / (pms / 1e3) / 1e9
    dominant = max(("fused", "ions", "poisson"), key=lambda k: kt[k][0])
    kname = {"fused": "k_fused", "ions": "k_ion_moments + k_ions", "poisson": "multigrid V-cycle kernels"}[dominant]
    achieved = gbs.get(dominant)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved or 0) / hbm if achieved else None, "traffic": None, "kernel": kname,
                "peak_kind": f"{peak_kind} copy bandwidth",
                "algorithmic_bytes_per_cell": per_cell[dominant],
                "units": ("fine cells x V-cycles" if dominant == "poisson" else "cells x steps"),
                "other_kernel_gbs": {k: v for k, v in gbs.items() if k != dominant}}
    kernels = {k: {"launches": kn, "ms_total": kms, "share": kms / max(1e-12, sum(v[0] for v in kt.values()))}
               for k, (kms, kn) in kt.items() if kn}

    e2e = None
    if not args.no_e2e:
        work = sim.workspace  # the caller's workspace, allocated before the timed region
        del sim
        host_phi = torch.from_numpy(cfg["phi"]).pin_memory()
        host_ions = torch.from_numpy(cfg["ions"]).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            s2 = L.Sim(params, host_phi, ions=host_ions, stream=stream, workspace=work)
            for _ in range(args.steps):
                s2.step(1)
                s2.observables()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": total / t_e2e / 1e6, "unit": METRIC,
               "h2d_bytes_per_step": int(5 * N * 8 / args.steps), "d2h_bytes_per_step": 20 * 8,
               "includes": "init from pinned host phase and ion fields (with its potential solves; workspace "
                           "allocated before) + per-step observables read-back", "seconds": t_e2e}
        del s2, work

    cpu = None
    if not args.no_cpu:
        try:
            import oracle
            cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
            nx, ny, k = 1280, 256, 4
            c = W.config_eof_channel(nx=nx, ny=ny, precision=0)
            o = oracle.Oracle(c["params"], c["phi"], ions=c["ions"])
            t0 = time.perf_counter()
            o.step(k)
            dt = (time.perf_counter() - t0) / k
            cpu = {"value": nx * ny / dt / 1e6, "unit": METRIC, "cores": cores, "kind": "oracle",
                   "sample": f"{k} steps of the same channel at {nx}x{ny} (kappa h scaled alike) with the oracle's FD "
                             "potential solve (conjugate gradients); init untimed", "seconds_per_step": dt}
        except Exception as exc:
            cpu = {"value": None, "error": repr(exc)}

    line = {"metric": METRIC, "value": total / t / 1e6, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_NAMES[prec],
            "data": "synthetic (the paper's electro-osmotic channel in lattice units, ions in their double layers)",
            "config": {"workload": f"electro-osmotic channel with Nernst-Planck ions, {params['nx']}x{params['ny']}",
                       "kappa_h": 20.0, "potential_solver": "multigrid V-cycles on the FD form",
                       "poisson_tol": params["poisson_tol"],
                       "l2": "working set (%.1f GB) exceeds the 126 MB L2; no flush needed" % (
                           L.workspace_bytes(params) / 1e9), "v_cycles_per_step": cycles / args.steps},
            "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "observables": {"nonfinite": obs["nonfinite"], "poisson_iters": obs["poisson_iters"],
                            "poisson_residual": obs["poisson_residual"], "ion_totals": mass}}
    print(json.dumps(line), flush=True)


def run_deformation3d(args):
    """The compound drop under field on a 256^3 D3Q15 lattice (the paper's deformation
    runs are three-dimensional): MLUPS over the timed steps, 16 warm-started potential
    iterations a step, the roofline of the dominant kernel class, an end-to-end run
    from pinned host fields, and the oracle on a bounded sample."""
    import torch
    import paper_2608_05787_b300 as L
    import workloads as W

    torch.cuda.set_device(0)
    prec = min(args.precision, 1)
    # --n other than the 2-D default scales the 256^3 drop (profiling runs)
    n3 = 256 if args.n == 4096 else args.n
    cfg = W.config_deformation_3d(n=n3, r_out=40.0 * n3 / 256, r_in=20.0 * n3 / 256, precision=prec)
    params = cfg["params"]
    n = params["nx"]
    N = n ** 3
    word = 8 if prec == 0 else 4
    iters = params["poisson_fixed_iter"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = L.Sim(params, torch.from_numpy(cfg["phi"]).cuda(), stream=stream)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        sim.set_timing(True)
        l0 = sim.launches
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(0) as clk:
            ev0.record(stream)
            sim.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = sim.launches - l0
        kt = sim.kernel_times()
        sim.set_timing(False)
        obs = sim.observables()
    t = ms / 1e3
    total = N * args.steps
    hbm, peak_kind = peaks()
    units = {"fused": args.steps, "poisson": args.steps * iters, "moments": args.steps}
    gbs = {k: WORDS_3D[k] * word * N * units[k] / (kt[k][0] / 1e3) / 1e9 for k in WORDS_3D if kt[k][1]}
    dominant = max(WORDS_3D, key=lambda k: kt[k][0])
    # FP32 with nx a multiple of 4: the potential iteration's inputs staged by TMA
    pot3 = "k3_poisson_tma" if prec == 1 and n % 4 == 0 else "k3_poisson"
    kname = {"fused": "k3_collide", "poisson": pot3, "moments": "k3_moments"}[dominant]
    roofline = {"bound": "hbm", "achieved": gbs.get(dominant), "peak": hbm, "unit": "GB/s",
                "frac": gbs.get(dominant, 0) / hbm, "traffic": None, "kernel": kname,
                "peak_kind": f"{peak_kind} copy bandwidth",
                "algorithmic_bytes_per_cell": WORDS_3D[dominant] * word,
                "units": "cells x pseudo-iterations" if dominant == "poisson" else "cells x steps",
                "other_kernel_gbs": {k: v for k, v in gbs.items() if k != dominant}}
    kernels = {k: {"launches": kn, "ms_total": kms, "share": kms / max(1e-12, sum(v[0] for v in kt.values()))}
               for k, (kms, kn) in kt.items() if kn}
    e2e = None
    if not args.no_e2e:
        work = sim.workspace  # the caller's workspace, allocated before the timed region
        del sim
        host_phi = torch.from_numpy(cfg["phi"]).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            s2 = L.Sim(params, host_phi, stream=stream, workspace=work)
            for _ in range(args.steps):
                s2.step(1)
                s2.observables()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": total / t_e2e / 1e6, "unit": METRIC, "h2d_bytes_per_step": int(3 * N * 8 / args.steps),
               "d2h_bytes_per_step": 16 * 8, "includes": "init from pinned host phases (with its potential solve; "
               "workspace allocated before) + per-step observables read-back", "seconds": t_e2e}
        del s2, work
    cpu = None
    if not args.no_cpu:
        try:
            import oracle
            cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
            m = 48
            c = W.config_deformation_3d(n=m, r_out=40.0 * m / 256, r_in=20.0 * m / 256, precision=0)
            o = oracle.Oracle3D(c["params"], c["phi"])
            t0 = time.perf_counter()
            o.step(3)
            dt = (time.perf_counter() - t0) / 3
            cpu = {"value": m ** 3 / dt / 1e6, "unit": METRIC, "cores": cores, "kind": "oracle",
                   "sample": f"3 steps of the same drop at {m}^3 (radii scaled), 16 potential iterations a step; "
                             "init untimed", "seconds_per_step": dt}
        except Exception as exc:
            cpu = {"value": None, "error": repr(exc)}
    line = {"metric": METRIC, "value": total / t / 1e6, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {0: "f64", 1: "f32"}[prec],
            "data": "synthetic (a compound sphere between electrodes)",
            "config": {"workload": f"compound drop deformation under field, D3Q15, {n}^3",
                       "potential_iters_per_step": iters,
                       "l2": "working set (%.1f GB) exceeds the 126 MB L2; no flush needed" % (
                           L.workspace_bytes(params) / 1e9)},
            "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "observables": {k: obs[k] for k in ("D_inner", "D_outer", "max_sum_dev", "nonfinite")}}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Derivative cost on the 256^2 drop under field plus shear: time per step of
    the FP32 tangent build (three parameter directions: E0, eps3, gamma23) over the
    time per step of the plain FP32 build, potential iterated 16 times per step."""
    import torch
    import paper_2608_05787_b300 as L
    import workloads as W

    torch.cuda.set_device(0)
    cfg = W.config_adjoint()
    p = dict(cfg["params"], poisson_fixed_iter=16)
    res = {}
    for name, prec, extra in (("forward", 1, {}), ("tangent3", 3, {"tangent_param": (0, 3, 6)})):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            sim = L.Sim(dict(p, precision=prec, **extra), cfg["phi"], stream=stream)
            sim.step(args.warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / args.steps
            # per-kernel-class breakdown from a separate event-timed pass
            sim.set_timing(True)
            sim.step(args.steps)
            kt = sim.kernel_times()
            sim.set_timing(False)
            res[name + "_kernels"] = {k: {"launches": n, "ms_per_step": ms / args.steps}
                                      for k, (ms, n) in kt.items() if n}
            sim.close()
    # reverse mode: one sweep (forward run with a snapshot every 200 steps, the
    # segment re-run keeping each step's snapshot, lb3e_adjoint_step back through it,
    # the creation's adjoint) over S steps, all eleven parameter slots at once
    from paper_2608_05787_b300.gradients import reverse_gradient
    S = max(args.steps, 200)
    for prec in (1, 0):
        pr = dict(p, precision=prec)
        reverse_gradient(pr, cfg["phi"], 8, checkpoint_every=200)  # warm-up (workspace, module load)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D, g, _ = reverse_gradient(pr, cfg["phi"], S, checkpoint_every=200)
        torch.cuda.synchronize()
        res[f"reverse{prec}"] = (time.perf_counter() - t0) * 1e3 / S
        res[f"reverse{prec}_grad"] = {k: g[k] for k in ("V_top", "eps3", "gamma23")}
        if prec == 0:
            # the FP64 forward step for the FP64 sweep's ratio
            sim = L.Sim(pr, cfg["phi"])
            sim.step(args.warmup)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.step(S)
            torch.cuda.synchronize()
            res["forward0"] = (time.perf_counter() - t0) * 1e3 / S
            sim.close()
    N = p["nx"] * p["ny"]
    line = {"metric": "derivative/forward time per step", "value": res["tangent3"] / res["forward"],
            "unit": "ratio", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["tangent3"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (dual numbers, 3 directions)", "data": "synthetic (stated initial condition)",
            "config": {"workload": "compound drop under field + shear, 256x256", "potential_iters_per_step": 16,
                       "forward_ms_per_step": res["forward"], "forward_mlups": N / res["forward"] / 1e3,
                       "forward_kernels": res["forward_kernels"], "tangent_kernels": res["tangent3_kernels"],
                       "derivatives": ["dD/dE0", "dD/d(eps3/eps1)", "dD/dgamma23"], "mode": "tangent (forward)"},
            "reverse": {"steps": S, "checkpoint_every": 200, "slots": 11,
                        "fp32_ms_per_step": res["reverse1"], "fp32_over_forward": res["reverse1"] / res["forward"],
                        "fp64_ms_per_step": res["reverse0"], "fp64_forward_ms_per_step": res["forward0"],
                        "fp64_over_forward": res["reverse0"] / res["forward0"],
                        "timing": "host clock around the whole sweep (forward run, re-runs, adjoint steps, the "
                                  "creation's adjoint), divided by the steps",
                        "fp32_gradient": res["reverse1_grad"], "fp64_gradient": res["reverse0_grad"]}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference" and args.workload in ("eof", "deformation3d"):
        run_reference_sample(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "regimes":
        run_regimes(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "eof":
        run_eof(args)
    elif args.workload == "deformation3d":
        run_deformation3d(args)
    else:
        run_lb3e(args)


if __name__ == "__main__":
    main()
