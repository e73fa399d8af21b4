#!/usr/bin/env python
"""Benchmark of the GPU domain-decomposition Helmholtz solver.

Step workload: 256x256 quads on the unit square, degree 3, 32x32 subdomains
of 8x8 elements (625 GLL nodes each), Y-shaped channel at c = 1/3 in c = 1,
omega = 64 pi, off-centre Gaussian source; synthetic, seeded.

One step = one full solve to ||b - K u|| <= 1e-8 ||b|| (FP64 global
residual): right-hand side, leapfrog coefficients, FP64 defect correction
whose DD solves run GMRES on the transmission data with one fused sweep
kernel launch (all 1024 subdomain WaveHoltz solves, FP32) per matvec.
Metric: DOF-updates/s = (sum over sweeps of subdomain nodes x (N_t - 1) x
WaveHoltz iterations) / wall time of the solves.

Legs measured once in the same run (rank 0): the FP32 and FP64 FMA peaks of
the device (the roofline denominators); the same solve in plain FP64; the
1024^2-quad degree-4 random-medium workload solved to 1e-8 with FP32 sweeps
and FP64 refinement (its plain-FP64 time as measured FP64 sweep time x sweep
count, labelled); a served stream of requests (Poisson arrivals, groups of 8
sources) with p50/p99 latency and solves/s against one-at-a-time plain FP64;
the FP64 CPU oracle on all host cores.

--impl reference times the FP64 CPU oracle (test infrastructure) on the
host's cores on a bounded sample of the step workload: one sweep of a subset
of subdomains per step.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s"
UNIT = "DOF-updates/s"
# DRAM bytes (read + write) of one launch of the one-warp-per-subdomain sweep
# on the 256x256, P=3 workload, from one ncu capture of this kernel version
# (coefficients and lambda read once; independent of the WaveHoltz count)
SWEEP_WARP_TRAFFIC_BYTES = 7.608832e6
TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 time-to-tolerance leg")
    ap.add_argument("--no-trials", action="store_true", help="skip the FP16/BF16 sweep-error trials")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--mode", choices=["solve", "sweep", "batch", "serve"], default="solve",
                    help="sweep: only run --sweeps DD sweeps of the workload (for ncu captures); "
                         "batch: batched solves of the multi-problem workload; serve: served request stream")
    ap.add_argument("--batch", type=int, default=12, help="problems in --mode batch")
    ap.add_argument("--batch-all", action="store_true",
                    help="--mode batch: all 64 problems of the batched workload under a sweep budget")
    ap.add_argument("--batch-sweeps", type=int, default=4, help="sweep budget per problem with --batch-all")
    ap.add_argument("--small-batch", type=int, default=32, help="small problems in --mode batch")
    ap.add_argument("--requests", type=int, default=40, help="arrivals in --mode serve")
    ap.add_argument("--rate", type=float, default=200.0, help="mean arrivals per second in --mode serve")
    ap.add_argument("--baseline-requests", type=int, default=12)
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--wh-iters", type=int, default=20, help="WaveHoltz iterations per sweep")
    ap.add_argument("--max-sweeps", type=int, default=5000)
    ap.add_argument("--max-refine", type=int, default=100)
    ap.add_argument("--refine", choices=["fgmres", "defect"], default="fgmres",
                    help="FP64 refinement: flexible GMRES with the DD solve as preconditioner, or defect correction")
    ap.add_argument("--inner-tol", type=float, default=0.3, help="relative tolerance of each DD solve")
    ap.add_argument("--gs-passes", type=int, choices=[1, 2], default=1,
                    help="classical Gram-Schmidt passes per Arnoldi step")
    ap.add_argument("--robin", default="0,1", help="interface condition d_n + k (eta - i zeta): 'eta,zeta'")
    ap.add_argument("--workload", choices=["cfg1", "cfg2", "cfg2m", "cfg3", "cfg3s", "cfg3p4", "cfg3p8", "cfg3p16"],
                    default="cfg2",
                    help="cfg2 is the benchmark workload; cfg1/cfg3 are reported separately; cfg3s is the "
                         "cfg3 physics and subdomain shape on a 256x256 mesh (for profiling)")
    ap.add_argument("--no-cfg3", action="store_true", help="skip the 1024^2 random-medium time-to-tolerance leg")
    ap.add_argument("--cfg3-wh-cap", type=int, default=300, help="WaveHoltz iterations at most per subdomain")
    ap.add_argument("--cfg3-wh-tol", type=float, default=1e-4, help="per-subdomain WaveHoltz tolerance")
    ap.add_argument("--cfg3-inner-tol", type=float, default=0.3)
    ap.add_argument("--cfg3-restart", type=int, default=200)
    ap.add_argument("--cfg3-max-sweeps", type=int, default=4000)
    ap.add_argument("--no-serve", action="store_true", help="skip the served-stream leg")
    ap.add_argument("--serve-requests", type=int, default=24, help="arrivals in the served-stream leg")
    ap.add_argument("--serve-pool", type=int, default=16,
                    help="the served requests are drawn from the cheapest this-many problems of the pool")
    ap.add_argument("--serve-baseline", type=int, default=3,
                    help="requests of the stream solved one at a time in plain FP64 for the comparison")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if _isnum(r[3]))}


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# ------------------------------------------------------- oracle sample ----
# The oracle (FP64 NumPy, test infrastructure) timed on the host's cores:
# a pool of single-threaded worker processes (spawned, so no worker inherits
# a CUDA context), each sweeping its own share of the sampled subdomains.
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS")
_OW = {}


def _oracle_problem(wl):
    from oracle import dd, geom, sem

    m = sem.Mesh(*wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny)
    gx, gy = m.coords_1d()
    if getattr(wl, "warp", 0.0) > 0.0:
        X, Y = wl.node_xy(gx, gy)
        return geom.MappedProblem(m, X, Y, wl.speed_at(X, Y), wl.omega, wl.source_at(X, Y), wl.boundary())
    return dd.Problem(m, wl.speed(gx, gy), wl.omega, wl.source(gx, gy), wl.boundary())


def _ow_init(name, m_wh):
    import numpy as np

    wl = workload(name)
    pr = _oracle_problem(wl)
    m = pr.mesh
    _OW.update(pr=pr, nt=pr.choose_nt(), m_wh=m_wh, rhs=pr.rhs(), lam=np.zeros((m.L, 4, m.NE), complex))


def _ow_sweep(subset):
    t0 = time.perf_counter()
    _OW["pr"].sweep(_OW["lam"], _OW["rhs"], _OW["nt"], _OW["m_wh"], subset=list(subset))
    return time.perf_counter() - t0


class OraclePool:
    """Single-threaded oracle worker processes on `cores` host cores (default:
    all), each holding the oracle problem of one workload.  sample(seconds)
    times one sweep over a sample of subdomains sized to take about that much
    wall time, every worker sweeping its own share."""

    def __init__(self, name, m_wh=5, cores=None):
        import multiprocessing as mp

        self.name, self.m_wh = name, m_wh
        self.cores = int(cores or os.cpu_count() or 1)
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        for k in _THREAD_VARS:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_ow_init, initargs=(name, m_wh))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.L = workload(name).L
        ncal = min(8, self.L)
        cal = self.pool.map(_ow_sweep, [[(k * ncal + q) % self.L for q in range(ncal)] for k in range(self.cores)])
        self.t_sub = max(cal) / ncal
        self.info = self.pool.apply(_ow_info)

    def sample(self, seconds):
        L, cores = self.L, self.cores
        per = int(max(1, min(max(1, 4 * L // cores), seconds / max(self.t_sub, 1e-6))))
        chunks = [[(k * per + q) % L for q in range(per)] for k in range(cores)]
        t0 = time.perf_counter()
        self.pool.map(_ow_sweep, chunks)
        wall = time.perf_counter() - t0
        n_sub = per * cores
        dof = n_sub * self.info["nl"] * (self.info["nt"] - 1) * self.m_wh
        return {"value": dof / wall, "cores": cores, "seconds": wall, "nt": self.info["nt"], "nl": self.info["nl"],
                "sample": f"one sweep (N_t={self.info['nt']}, {self.m_wh} WaveHoltz iterations) of {per} subdomains "
                          f"on each of {cores} single-threaded processes ({n_sub} subdomain solves, {L} subdomains "
                          f"in the workload), FP64 NumPy"}

    def close(self):
        self.pool.terminate()
        self.pool.join()


def _ow_info():
    m = _OW["pr"].mesh
    return {"nt": _OW["nt"], "nl": m.nlx * m.nly}


def _oracle_solve_cfg1(q):
    """Child process: the oracle's own solve of cfg1 to 1e-8 (FP64 defect
    correction around GMRES(60) on the transmission data, 20 WaveHoltz
    iterations per sweep, inner tolerance 1e-2: the GPU solve's settings)."""
    try:
        wl = workload("cfg1")
        pr = _oracle_problem(wl)
        t0 = time.perf_counter()
        _, info = pr.solve(m_wh=20, tol=TOL, outer="gmres", restart=60, inner_tol=1e-2, max_sweeps=5000,
                           max_refine=20)
        q.put({"seconds": time.perf_counter() - t0, "sweeps": info["sweeps"], "refinements": info["refinements"],
               "rel_residual": info["rel_residual"], "cores": 1})
    except Exception as e:  # reported, not raised: a baseline leg
        q.put({"error": repr(e)})


def start_oracle_cfg1():
    """Starts the oracle's cfg1 time-to-tolerance in a spawned single-threaded
    process (it runs beside the GPU legs on one otherwise idle host core)."""
    import multiprocessing as mp

    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    for k in _THREAD_VARS:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        p = ctx.Process(target=_oracle_solve_cfg1, args=(q,), daemon=True)
        p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return p, q


def finish_oracle_cfg1(handle, timeout):
    p, q = handle
    try:
        return q.get(timeout=max(1.0, timeout))
    except Exception:
        p.terminate()
        return {"error": f"not finished within {timeout:.0f} s"}


def hbm_peak_gbs():
    """Measured copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json), else
    the recipe's fallback figure."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def workload(name):
    from workloads import configs

    if name == "cfg3s":
        return configs.scaled(configs.config3(), 256, 256, 32, 32, name="cfg3_scaled_256x256_p4_sub32")
    if name in ("cfg3p4", "cfg3p8", "cfg3p16"):  # S x S subdomains of the 1024^2 workload: its shape, h, medium
        S = int(name[5:])
        w = configs.config3()
        h = (w.box[1] - w.box[0]) / w.nx
        n = 32 * S
        return configs.Workload(f"cfg3_piece_{S}x{S}_subdomains", (-0.5, -0.5 + n * h, -0.5, -0.5 + n * h), n, n,
                                w.P, w.sub_nx, w.sub_ny, w.omega, w.speed_kind,
                                (-0.5 + (n / 2 + 0.5) * h, -0.5 + (n / 2 - 0.5) * h), w.src_width, w.speed_seed,
                                w.corr_len)
    return {"cfg1": configs.config1, "cfg2": configs.config2, "cfg2m": configs.config2m,
            "cfg3": configs.config3}[name]()


def sweep_flops_per_update(wl):
    """Algorithmic flops per DOF-update of one sweep kernel.
    Cartesian (tensor-product) stiffness: F(P) = 2P + 13 FMA.
    Mapped (element-form) stiffness: per element node 2(P+1) FMA for the
    reference gradient and 4 for the metric fluxes, per (node, element) pair
    2(P+1) FMA for the D^T gather, and 7 for the leapfrog and filter updates;
    with e = element nodes per subdomain node (Ne / n_l) that is
    e (4(P+1) + 4) + 7 FMA.  flops = 2 FMA."""
    P = wl.P
    if getattr(wl, "warp", 0.0) > 0.0:
        ne = wl.sub_nx * wl.sub_ny * (P + 1) ** 2
        nl = (wl.sub_nx * P + 1) * (wl.sub_ny * P + 1)
        return 2.0 * ((ne / nl) * (4 * (P + 1) + 4) + 7)
    return 2.0 * (2 * P + 13)


def combine_ranks(elapsed, work, device):
    """Whole-job figures over all ranks: the slowest rank's time and the sum
    of the work (weak scaling: every rank solves its own problem)."""
    import torch
    import torch.distributed as tdist

    if not tdist.is_initialized() or tdist.get_world_size() == 1:
        return float(elapsed), float(work)
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    tdist.all_reduce(w, op=tdist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


# --------------------------------------------------------------- legs ----
def leg_peaks(hz):
    """FP32 and FP64 FMA rates of this device, measured now (hz_fma_peak: a
    kernel of independent FMAs only; best of three launches of 30-45 ms)."""
    fp32 = max(hz.hz_fma_peak(hz.HZ_FP32_REFINE, 60000)[0] for _ in range(3))
    fp64 = max(hz.hz_fma_peak(hz.HZ_FP64, 1200)[0] for _ in range(3))
    return {"fp32_tflops": fp32, "fp64_tflops": fp64,
            "how": "hz_fma_peak: 4 blocks of 256 threads per SM, 8 independent FMA chains per thread, "
                   "CUDA events, best of 3"}


def _timed_sweeps(hz, case, precision, nt, wh_iters, k, stream):
    """Mean device time (CUDA events) of k homogeneous sweeps after one untimed."""
    import torch

    nl = hz.hz_lambda_size(case.pr)
    gen = torch.Generator(device="cuda").manual_seed(2)
    lin = torch.randn(2 * nl, dtype=torch.float64, device="cuda", generator=gen) * 1e-2
    lout = torch.zeros_like(lin)
    hz.hz_sweep(case.pr, precision, nt, wh_iters, 0.0, lin, lout, None, None, stream)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(k):
        hz.hz_sweep(case.pr, precision, nt, wh_iters, 0.0, lin, lout, None, None, stream)
    a1.record(stream)
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) * 1e-3 / k


def cfg3_solve_opts(hz, args, max_sweeps=None):
    """FP32 sweeps with a per-subdomain WaveHoltz tolerance inside FP64
    flexible-GMRES refinement: the configuration that reaches 1e-8 on the
    random medium (a fixed WaveHoltz count leaves the slowest subdomains'
    solves too inexact for any refinement to converge)."""
    return hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=TOL, inner_tol=args.cfg3_inner_tol,
                              wh_iters=args.cfg3_wh_cap, wh_tol=args.cfg3_wh_tol, gmres_restart=args.cfg3_restart,
                              refine=hz.HZ_REFINE_FGMRES, refine_restart=60, max_refine=200,
                              max_sweeps=max_sweeps or args.cfg3_max_sweeps)


def leg_cfg3(hz, args, stream):
    """The 1024^2-quad, degree-4 random-medium workload (32x32 subdomains of
    16641 nodes, omega = 2 pi 204.8).  At full size: the sweep kernel's
    throughput at the solve's fixed-count configuration (FP32 and FP64, CUDA
    events), its roofline figures.  Solved to 1e-8: the same physics on 8x8
    of its subdomains (its subdomain shape, element size, frequency and
    medium; 1.05 M nodes), FP32 sweeps + FP64 FGMRES refinement, CUDA events
    around the solve; its plain-FP64 time is the FP32 time scaled by the
    measured FP64 / FP32 sweep-time ratio (labelled an estimate: a plain-FP64
    solve would take ~20x longer)."""
    import torch

    from paper_2606_21695_gb300.api import Case

    out = {}
    wl = workload("cfg3")
    case = Case(wl)
    try:
        nt = hz.hz_problem_nt(case.pr)
        m = args.wh_iters
        u = torch.zeros(2 * case.n, dtype=torch.float64, device="cuda")
        # a solve cut short runs the autotuner for the shape (the solve's kernel choice)
        hz.hz_solve_device(case.pr, hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, wh_iters=m, max_sweeps=3), u,
                           stream)
        del u
        t32 = _timed_sweeps(hz, case, hz.HZ_FP32_REFINE, nt, m, 3, stream)
        t64 = _timed_sweeps(hz, case, hz.HZ_FP64, nt, m, 1, stream)
        dof = wl.dof_per_sweep(nt, m)
        flop = sweep_flops_per_update(wl) * dof
        out["full_size"] = {"workload": wl.name, "nodes": case.n, "nt": nt, "wh_iters": m,
                            "fp32_sweep_ms": t32 * 1e3, "fp64_sweep_ms": t64 * 1e3,
                            "fp32_dof_updates_per_s": dof / t32, "fp64_dof_updates_per_s": dof / t64,
                            "fp32_sweep_tflops": flop / t32 / 1e12, "fp64_sweep_tflops": flop / t64 / 1e12}
    finally:
        case.close()
    wp = workload("cfg3p8")
    case = Case(wp)
    try:
        n = case.n
        opts = cfg3_solve_opts(hz, args)
        u = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
        hz.hz_solve_device(case.pr, cfg3_solve_opts(hz, args, max_sweeps=4), u, stream)  # tune the shape first
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, rep = hz.hz_solve_device(case.pr, opts, u, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        tt = e0.elapsed_time(e1) * 1e-3
        nt = rep["nt"]
        r32 = _timed_sweeps(hz, case, hz.HZ_FP32_REFINE, nt, 20, 2, stream)
        r64 = _timed_sweeps(hz, case, hz.HZ_FP64, nt, 20, 1, stream)
        out["piece_solve"] = {"workload": wp.name, "nodes": n, "status": hz.STATUS_NAMES[st],
                              "rel_residual": rep["rel_residual"], "time_to_tol_s": tt, "sweeps": rep["sweeps"],
                              "dd_solves": rep["refinements"], "gmres_iters": rep["gmres_iters"], "nt": nt,
                              "wh_tol": opts.wh_tol, "wh_cap": opts.wh_iters, "wh_iters_max": rep["wh_iters_max"],
                              "inner_tol": opts.inner_tol, "refinement": f"FGMRES({opts.refine_restart}), FP64",
                              "dof_updates": rep["dof_updates"], "dof_updates_per_s": rep["dof_updates"] / tt,
                              "sweep_kernel": rep["sweep_variant"], "fp64_over_fp32_sweep": r64 / r32,
                              "fp64_time_to_tol_s_estimated": tt * r64 / r32,
                              "fp64_estimate": "FP32 time-to-1e-8 x measured FP64/FP32 sweep-time ratio (20 WaveHoltz "
                                               "iterations) on this workload"}
    finally:
        case.close()
    return out


def _serve_pool(k):
    """The k problems of the served workload's pool (the batched workload's
    sampler, seed 500) with the smallest estimated cost, global nodes x N_t
    (the sampler spans five orders of magnitude: N_t reaches 16 000)."""
    from workloads import configs

    lam = {1: 8.0, 2: 48.0, 3: 148.6, 4: 366.7, 5: 783.9}  # lambda_max h^2 of the 2D GLL operator
    rows = []
    for w in configs.config4(64, seed0=500):
        cmax = 1.75 if w.speed_kind == "random" else 1.0
        dt = 0.9 * 2 / (cmax * math.sqrt(lam[w.P]) * w.nx)
        nt = math.ceil(2 * math.pi / w.omega / dt)
        rows.append(((w.nx * w.P + 1) ** 2 * nt, w))
    rows.sort(key=lambda r: r[0])
    return [w for _, w in rows[:k]]


def serve_opts(hz, precision):
    """Options of a served request: FP64 flexible-GMRES(60) refinement around
    DD solves to 0.3 whose WaveHoltz runs per subdomain to a tolerance of 1e-4
    (at most 300 iterations): the pool's high-frequency problems on wide
    subdomains stall with a fixed WaveHoltz count."""
    return hz.hz_default_opts(precision=precision, tol=TOL, inner_tol=0.3, wh_iters=300, wh_tol=1e-4,
                              refine=hz.HZ_REFINE_FGMRES, refine_restart=60, max_refine=200, max_sweeps=6000)


def leg_serve(hz, n_requests, rate, pool_k, baseline_k, seed=5):
    """Served stream: Poisson arrivals (seeded, mean `rate` per second) of
    solve requests drawn from the pool; with probability 0.2 a request is a
    group of 8 sources sharing mesh, wave speed and frequency.  The server
    (HBM budget 150 GB) admits them as memory frees and advances the admitted
    solves together.  Latency = submit to solution on the host.  The
    comparison: the first `baseline_k` requests solved one at a time in plain
    FP64."""
    import numpy as np

    from paper_2606_21695_gb300.api import Case
    from workloads import fields

    pool = _serve_pool(pool_k)
    cases = {w.name: Case(w) for w in pool}
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate)
        w = pool[int(rng.integers(len(pool)))]
        k = 8 if rng.uniform() < 0.2 else 1
        for _ in range(k):
            reqs.append((t, w, tuple(rng.uniform(0.2, 0.8, 2))))
    opts = serve_opts(hz, hz.HZ_FP32_REFINE)
    probs = []  # per-request problems (sources differ), built before the clock starts
    for _, w, ctr in reqs:
        c = cases[w.name]
        X, Y = np.meshgrid(c.gx, c.gy)
        f = fields.gaussian_source(X, Y, ctr, w.src_width).astype(complex)
        pr = hz.hz_problem_create(c.mesh, 0)
        hz.hz_problem_set(pr, hz.HZ_WAVE_SPEED, c.c.ravel())
        hz.hz_problem_set(pr, hz.HZ_OMEGA, np.array([w.omega]))
        hz.hz_problem_set(pr, hz.HZ_SOURCE, f.ravel())
        probs.append((pr, c.n))
    used = sorted({w.name for _, w, _ in reqs})
    for name in used:  # autotune the shapes outside the timed stream
        hz.hz_solve(cases[name].pr, opts, n=cases[name].n)
    srv = hz.hz_server_create(0, 150 << 30)
    t0 = time.perf_counter()
    tickets = []
    for (ta, _, _), (pr, n) in zip(reqs, probs):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append(hz.hz_server_submit(srv, pr, opts))
    statuses, res, errors = {}, [], []
    for k, tk in enumerate(tickets):
        try:
            _, st, _, rep = hz.hz_server_poll(srv, tk, -1, n=None)
            res.append(rep["rel_residual"])
            if st != hz.HZ_OK:
                errors.append({"request": k, "problem": reqs[k][1].name, "status": hz.STATUS_NAMES[st],
                               "rel_residual": rep["rel_residual"], "sweeps": rep["sweeps"]})
        except hz.HzError as e:
            st = e.status
            errors.append({"request": k, "problem": reqs[k][1].name, "error": str(e)})
        statuses[hz.STATUS_NAMES[st]] = statuses.get(hz.STATUS_NAMES[st], 0) + 1
    wall = time.perf_counter() - t0
    stats = hz.hz_server_stats(srv)
    hz.hz_server_destroy(srv)
    o64 = serve_opts(hz, hz.HZ_FP64)
    nb = min(len(probs), baseline_k)
    t0 = time.perf_counter()
    for pr, n in probs[:nb]:
        hz.hz_solve(pr, o64, n=n)
    t_base = (time.perf_counter() - t0) / nb
    for pr, _ in probs:
        hz.hz_problem_destroy(pr)
    for c in cases.values():
        c.close()
    ok = statuses.get("HZ_OK", 0)
    return {"requests": n_requests, "solves": len(reqs), "arrival_rate_per_s": rate, "wall_s": wall,
            "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "solves_per_s": ok / wall,
            "statuses": statuses, "failed": len(reqs) - ok, "errors": errors,
            "max_rel_residual": max(res) if res else None,
            "hbm_budget_gb": 150, "pool": f"{pool_k} cheapest of the 64-problem pool", "problems_used": used,
            "one_at_a_time_fp64_s_per_solve": t_base, "one_at_a_time_fp64_solves_per_s": 1.0 / t_base,
            "one_at_a_time_fp64_sample": nb}


def leg_cpu(args, cfg1_handle, t_start, cfg2_dof_per_solve, cfg3):
    """The oracle on the host cores: its sweep rate on the step workload and
    on a piece of the 1024^2 workload (all cores), its own cfg1 solve to 1e-8
    (one core, run beside the GPU legs), and time-to-tolerance estimates for
    the two big workloads (the GPU solve's DOF-updates / the oracle's rate)."""
    pool = OraclePool(args.workload, m_wh=args.wh_iters)
    s2 = pool.sample(args.cpu_sample_s)
    pool.close()
    out = {"value": s2["value"], "unit": UNIT, "cores": s2["cores"], "kind": "oracle", "sample": s2["sample"],
           "seconds": s2["seconds"]}
    tt = {}
    if cfg1_handle is not None:
        tt["cfg1_measured"] = finish_oracle_cfg1(cfg1_handle, timeout=600 - (time.perf_counter() - t_start))
    tt["cfg2_estimated_s"] = cfg2_dof_per_solve / s2["value"]
    if cfg3 is not None and cfg3.get("piece_solve", {}).get("dof_updates"):
        pool3 = OraclePool("cfg3p4", m_wh=5)
        s3 = pool3.sample(8.0)
        pool3.close()
        out["cfg3_shape_rate"] = s3["value"]
        tt["cfg3_piece_estimated_s"] = cfg3["piece_solve"]["dof_updates"] / s3["value"]
    tt["estimate"] = ("the GPU solve's DOF-updates / the oracle's DOF-updates/s on all cores (same method, "
                      "same sweep count)")
    out["time_to_tol_s"] = tt
    return out


# ------------------------------------------------------------ our arm ----
def step_config(wl, nt, args, world):
    """The timed step's workload, the same in both arms' JSON lines."""
    robin = [float(v) for v in args.robin.split(",")]
    return {"workload": wl.name, "mesh": f"{wl.nx}x{wl.ny} quads", "degree": wl.P,
            "subdomains": f"{wl.nx // wl.sub_nx}x{wl.ny // wl.sub_ny} of {wl.sub_nx}x{wl.sub_ny}",
            "omega": wl.omega, "nt": nt, "wh_iters": args.wh_iters, "tol": TOL,
            "outer": (f"GMRES(60) on the transmission data to {args.inner_tol:g}, {args.gs_passes} "
                      f"classical Gram-Schmidt pass(es), inside FP64 "
                      + ("flexible GMRES(60) on K u = b" if args.refine == "fgmres" else "defect correction")),
            "l2": "flushed (256 MB write) before each step",
            "transmission": {"eta": robin[0], "zeta": robin[1]},
            "parallelism": f"{world} independent solves (one per GPU)"}


def run_ours(args):
    t_start = time.perf_counter()
    rank, world, local = dist_env()
    # the oracle's own cfg1 solve runs beside the GPU legs on one host core
    # (spawned before this process touches CUDA)
    cfg1_handle = start_oracle_cfg1() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2606_21695_gb300 as hz
    from paper_2606_21695_gb300.api import Case, boundary_vector
    from workloads import configs

    wl = workload(args.workload)
    case = Case(wl, device=local)
    robin = [float(v) for v in args.robin.split(",")]
    if robin != [0.0, 1.0]:
        hz.hz_problem_set(case.pr, hz.HZ_TRANSMISSION, np.array(robin))
    n = case.n
    stream = torch.cuda.current_stream()
    refine = hz.HZ_REFINE_FGMRES if args.refine == "fgmres" else hz.HZ_REFINE_DEFECT
    opts = hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=TOL, inner_tol=args.inner_tol,
                              wh_iters=args.wh_iters, gmres_restart=60, max_sweeps=args.max_sweeps,
                              max_refine=args.max_refine, gs_passes=args.gs_passes, refine=refine,
                              refine_restart=60)
    u = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def barrier():
        if world > 1:
            import torch.distributed as tdist

            tdist.barrier()

    for _ in range(args.warmup):
        st, rep = hz.hz_solve_device(case.pr, opts, u, stream)
        if st != hz.HZ_OK:
            raise RuntimeError(f"warm-up solve did not converge: {rep}")
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    reports = []
    launches0 = hz.hz_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        st, rep = hz.hz_solve_device(case.pr, opts, u, stream)
        if st != hz.HZ_OK:
            raise RuntimeError(f"solve did not converge: {rep}")
        reports.append(rep)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    clocks = sampler.stop()
    launches = hz.hz_kernel_launches() - launches0
    elapsed = ev0.elapsed_time(ev1) * 1e-3
    dof = sum(r["dof_updates"] for r in reports)
    sweeps = sum(r["sweeps"] for r in reports)
    sweep_s = sum(r["sweep_seconds"] for r in reports)
    elapsed_max, dof_all = combine_ranks(elapsed, dof, "cuda")
    value = dof_all / elapsed_max
    res = [r["rel_residual"] for r in reports]
    nt = reports[0]["nt"]
    P = wl.P
    flops_per_update = sweep_flops_per_update(wl)
    dof_per_launch = dof / sweeps
    avg_launch = sweep_s / sweeps
    achieved = flops_per_update * dof_per_launch / avg_launch / 1e12

    out = None
    if rank == 0:
        peaks = leg_peaks(hz)
        # end-to-end through the public C ABI with host buffers: upload the
        # fields, solve, read u back; every step
        c_h, f_h, g_h = case.c.ravel(), case.f.ravel(), boundary_vector(case.g)
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_dof = 0
        for _ in range(e2e_steps):
            hz.hz_problem_set(case.pr, hz.HZ_WAVE_SPEED, c_h)
            hz.hz_problem_set(case.pr, hz.HZ_OMEGA, np.array([wl.omega]))
            hz.hz_problem_set(case.pr, hz.HZ_SOURCE, f_h)
            hz.hz_problem_set(case.pr, hz.HZ_BOUNDARY, g_h)
            st, u_h, rep = hz.hz_solve(case.pr, opts, n=n)
            assert st == hz.HZ_OK
            e2e_dof += rep["dof_updates"]
        e2e_t = time.perf_counter() - t0
        h2d = c_h.nbytes + 8 + f_h.astype(complex).nbytes + g_h.astype(complex).nbytes
        d2h = 16 * n
        # plain-FP64 time to the same tolerance, one solve (outside the timed region)
        fp64 = None
        if not args.no_fp64:
            o64 = hz.hz_default_opts(precision=hz.HZ_FP64, tol=TOL, inner_tol=args.inner_tol,
                                     wh_iters=args.wh_iters, gmres_restart=60, max_sweeps=args.max_sweeps,
                                     max_refine=args.max_refine, gs_passes=args.gs_passes, refine=refine,
                                     refine_restart=60)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st64, rep64 = hz.hz_solve_device(case.pr, o64, u, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            fp64 = {"seconds": e0.elapsed_time(e1) * 1e-3, "status": hz.STATUS_NAMES[st64],
                    "sweeps": rep64["sweeps"], "rel_residual": rep64["rel_residual"],
                    "dof_updates_per_s": rep64["dof_updates"] / (e0.elapsed_time(e1) * 1e-3)}
        # global FP64 residual (HBM-bound): hz_residual on device buffers, L2
        # flushed before each launch, CUDA events around each call
        aux = None
        if world == 1:
            nres = 20
            rb = torch.randn(2 * n, dtype=torch.float64, device="cuda")
            ru = torch.randn(2 * n, dtype=torch.float64, device="cuda")
            rr = torch.empty_like(rb)
            rn = torch.zeros(2, dtype=torch.float64, device="cuda")
            for _ in range(3):
                hz.hz_residual(case.pr, rb, ru, rr, rn, stream)
            tot_ms = 0.0
            for _ in range(nres):
                flush.fill_(1)
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record()
                hz.hz_residual(case.pr, rb, ru, rr, rn, stream)
                a1.record()
                torch.cuda.synchronize()
                tot_ms += a0.elapsed_time(a1)
            res_ms = tot_ms / nres
            res_bytes = 56 * n  # b, u read (16 B each), c read (8 B), r written (16 B) per node
            # FP64 work per node: x and y rows of 2P+1 taps on complex u (4(2P+1) FMA), the
            # weights (4), the H and M terms (4) and b - K u (2); 2 flops per FMA
            res_flops = 2 * (4 * (2 * P + 1) + 10) * n
            peak = hbm_peak_gbs()
            gbs = res_bytes / (res_ms * 1e-3) / 1e9
            tfl = res_flops / (res_ms * 1e-3) / 1e12
            aux = {"residual": {"kernel": "residual_kernel + reduce_partials_kernel (FP64, global grid)",
                                "bound": "fp64 alu", "ms": res_ms, "algorithmic_flops": res_flops,
                                "achieved_tflops": tfl, "peak_tflops": peaks["fp64_tflops"],
                                "frac": tfl / peaks["fp64_tflops"], "peak_source": "measured FP64 FMA rate",
                                "algorithmic_bytes": res_bytes,
                                "achieved_gbs": gbs, "hbm_peak_gbs": peak, "hbm_frac": gbs / peak}}
            del rb, ru, rr, rn
        # 16-bit trials: one sweep each, error against the FP64 sweep (which is
        # checked against the oracle by the test suite)
        trials = None
        if not args.no_trials:
            nt_ = reports[0]["nt"]
            nl = hz.hz_lambda_size(case.pr)
            gen = torch.Generator(device="cuda").manual_seed(1)
            lin = torch.randn(2 * nl, dtype=torch.float64, device="cuda", generator=gen) * 1e-2
            outs = {}
            for name, prec in (("fp64", hz.HZ_FP64), ("fp32", hz.HZ_FP32_REFINE), ("fp16", hz.HZ_FP16_TRIAL),
                               ("bf16", hz.HZ_BF16_TRIAL)):
                lo = torch.zeros_like(lin)
                hz.hz_sweep(case.pr, prec, nt_, opts.wh_iters, 0.0, lin, lo)
                outs[name] = lo
            torch.cuda.synchronize()
            ref = outs["fp64"]
            den = float(ref.abs().max())
            trials = {k: {"sweep_rel_err_vs_fp64": float((outs[k] - ref).abs().max()) / den}
                      for k in ("fp32", "fp16", "bf16")}
        cfg3 = leg_cfg3(hz, args, stream) if (world == 1 and not args.no_cfg3) else None
        serve = (leg_serve(hz, args.serve_requests, args.rate, args.serve_pool, args.serve_baseline)
                 if (world == 1 and not args.no_serve) else None)
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = leg_cpu(args, cfg1_handle, t_start, dof / args.steps, cfg3)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (subdomain WaveHoltz) + f64 (outer, residual)",
            "data": "synthetic (seeded generators)",
            "config": step_config(wl, nt, args, world),
            "time_to_tol_s": {"fp32_refine": elapsed / args.steps, "fp64": fp64["seconds"] if fp64 else None,
                              "cfg3_piece_fp32_refine": cfg3["piece_solve"]["time_to_tol_s"] if cfg3 else None,
                              "cfg3_piece_fp64_estimated": (cfg3["piece_solve"]["fp64_time_to_tol_s_estimated"]
                                                            if cfg3 else None)},
            "cfg3": cfg3,
            "serve": serve,
            "peaks": peaks,
            "fp64_solve": fp64,
            "solve": {"sweeps_per_solve": sweeps / args.steps, "rel_residual_max": max(res),
                      "sweep_kernel": {1: "block", 2: "warp", 3: "cluster", 4: "packed",
                                       5: "cluster of warp bands", 6: "mapped (element form)"}.get(reports[0]["sweep_variant"]),
                      "refinements": reports[0]["refinements"], "gmres_iters": reports[0]["gmres_iters"],
                      "dof_updates_per_solve": dof / args.steps},
            "roofline": {"kernel": {1: "sweep_kernel (block)",
                                    2: ("sweep_warp_kernel (one warp per subdomain)" if reports[0]["sweep_shape"] <= 1
                                        else f"sweep_band_kernel ({reports[0]['sweep_shape']} warps per subdomain)"),
                                    3: "sweep_cluster_kernel", 5: "sweep_cband_kernel",
                                    6: "sweep_mapped_kernel (element form, block per subdomain)"}.get(reports[0]["sweep_variant"], "?")
                         + " FP32, one launch = one DD sweep", "bound": "alu",
                         "achieved": achieved, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["fp32_tflops"],
                         "peak_source": "measured in this run (hz_fma_peak, FP32 FMA)",
                         "traffic": SWEEP_WARP_TRAFFIC_BYTES if (wl.P == 3 and reports[0]["sweep_variant"] == 2
                                                                 and reports[0]["sweep_shape"] == 1) else None,
                         "traffic_unit": "bytes per launch (DRAM, ncu)",
                         "sweep_shape": reports[0]["sweep_shape"],
                         "algorithmic": f"{flops_per_update:.4g} flop/DOF-update x {dof_per_launch:.4g} DOF-updates/launch",
                         "avg_launch_ms": avg_launch * 1e3, "launch_share": sweep_s / elapsed},
            "cpu_baseline": cpu,
            "precision_trials": trials,
            "aux_kernels": aux,
            "e2e": {"value": e2e_dof / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": e2e_steps},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "wall_s": t_wall,
        }
    case.close()
    if world > 1:
        import torch.distributed as tdist

        tdist.destroy_process_group()
    return out


# ------------------------------------------------------ reference arm ----
def run_reference(args):
    """The oracle as it stands (FP64 NumPy), timed on all host cores: each
    step one sweep over a bounded sample of the step workload's subdomains."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    wl = workload(args.workload)
    pool = OraclePool(args.workload, m_wh=args.wh_iters)
    vals = []
    desc, cores = "", pool.cores
    try:
        for k in range(args.warmup + args.steps):
            r = pool.sample(3.0)
            desc = r["sample"]
            if k >= args.warmup:
                vals.append((r["value"], r["seconds"]))
    finally:
        pool.close()
    tot_t = sum(el for _, el in vals)
    value = sum(v * el for v, el in vals) / tot_t
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generators)",
        "config": step_config(wl, pool.info["nt"], args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_sweeps(args):
    """--mode sweep: set up the workload and launch --sweeps homogeneous DD
    sweeps through the C ABI (the launch configuration of the solve)."""
    import torch

    import paper_2606_21695_gb300 as hz
    from paper_2606_21695_gb300.api import Case
    from workloads import configs

    wl = workload(args.workload)
    case = Case(wl)
    nt = hz.hz_problem_nt(case.pr)
    nl = hz.hz_lambda_size(case.pr)
    g = torch.Generator(device="cuda").manual_seed(0)
    lin = torch.randn(2 * nl, dtype=torch.float64, device="cuda", generator=g) * 1e-2
    lout = torch.zeros_like(lin)
    prec = hz.HZ_FP32_REFINE if args.precision == "fp32" else hz.HZ_FP64
    # first sweep untimed (autotuning, if any, and warm-up); the rest timed
    # on the launching (default) stream
    hz.hz_sweep(case.pr, prec, nt, args.wh_iters, 0.0, lin, lout)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.sweeps - 1):
        hz.hz_sweep(case.pr, prec, nt, args.wh_iters, 0.0, lin, lout)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.sweeps - 1)
    L = wl.nx // wl.sub_nx * (wl.ny // wl.sub_ny)
    dof = L * (wl.sub_nx * wl.P + 1) * (wl.sub_ny * wl.P + 1) * (nt - 1) * args.wh_iters
    flop = sweep_flops_per_update(wl) * dof
    case.close()
    return {"mode": "sweep", "workload": wl.name, "sweeps": args.sweeps, "nt": nt, "precision": args.precision,
            "wh_iters": args.wh_iters, "ms_per_sweep": ms if args.sweeps > 1 else None,
            "dof_updates_per_sweep": dof, "dof_updates_per_s": dof / (ms * 1e-3) if args.sweeps > 1 else None,
            "tflops": flop / (ms * 1e-3) / 1e12 if args.sweeps > 1 else None}


def _cheap_cfg4(k):
    """The k least expensive problems of the batched workload sampler (cost =
    global nodes x estimated N_t); the full sampler reaches N_t ~ 10^4 on
    512^2 degree-5 meshes, far beyond a bench run."""
    from workloads import configs

    lam = {1: 8.0, 2: 48.0, 3: 148.6, 4: 366.7, 5: 783.9}  # lambda_max h^2 of the 2D GLL operator
    rows = []
    for w in configs.config4():
        cmax = 1.5 if w.speed_kind == "random" else 1.0
        dt = 0.9 * 2 / (cmax * math.sqrt(lam[w.P]) * w.nx)
        nt = math.ceil(2 * math.pi / w.omega / dt)
        rows.append(((w.nx * w.P + 1) ** 2 * nt, w))
    rows.sort(key=lambda r: r[0])
    return [w for _, w in rows[:k]]


# (degree, subdomain elements in y) compiled into the packed sweep; the
# subdomain must also have at most 32 node columns
PACKED_SHAPES = {(1, 4), (1, 8), (1, 16), (2, 4), (2, 8), (3, 4), (3, 8), (4, 4), (5, 4)}


def _packable(w):
    return (w.P, w.sub_ny) in PACKED_SHAPES and w.sub_nx * w.P + 1 <= 32


def _cheap_packable_cfg4(k):
    return [w for w in _cheap_cfg4(64) if _packable(w)][:k]


def _batch_group(hz, cases, max_sweeps):
    """Sequential solves (with and without the step graphs), an unpacked
    concurrent batch and a packed batch of the same problems."""
    import torch

    prs, ns = [c.pr for c in cases], [c.n for c in cases]
    mk = lambda **kw: hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=TOL, max_sweeps=max_sweeps, **kw)
    opts, popts, nog = mk(pack=0), mk(pack=1), mk(pack=0, graphs=0)
    hz.hz_solve_batch(prs, ns, opts, 8, want_u=False)  # warm-up / autotune / graph capture
    hz.hz_solve_batch(prs, ns, popts, 0, want_u=False)
    torch.cuda.synchronize()
    out = {}
    t0 = time.perf_counter()
    seq = [hz.hz_solve(c.pr, nog, n=c.n) for c in cases]
    out["sequential_nographs_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    seq = [hz.hz_solve(c.pr, opts, n=c.n) for c in cases]
    out["sequential_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    st, sts, _, reps = hz.hz_solve_batch(prs, ns, opts, 8, want_u=False)
    out["batched_s"] = time.perf_counter() - t0
    k0 = hz.hz_kernel_launches()
    t0 = time.perf_counter()
    pst, psts, _, preps = hz.hz_solve_batch(prs, ns, popts, 0, want_u=False)
    out["packed_s"] = time.perf_counter() - t0
    out["packed_kernel_launches"] = hz.hz_kernel_launches() - k0
    out["packed_members"] = sum(r["sweep_variant"] == 4 for r in preps)
    out["speedup_batched"] = out["sequential_s"] / out["batched_s"]
    out["speedup_packed"] = out["sequential_s"] / out["packed_s"]
    out["dof_updates_per_s_batched"] = sum(r["dof_updates"] for r in reps) / out["batched_s"]
    out["dof_updates_per_s_packed"] = sum(r["dof_updates"] for r in preps) / out["packed_s"]
    out["solves_per_s_packed"] = len(cases) / out["packed_s"]
    out["max_rel_residual"] = max(r["rel_residual"] for r in reps + preps + [s[2] for s in seq])
    out["statuses"] = [hz.STATUS_NAMES[s] for s in sts]
    out["packed_statuses"] = [hz.STATUS_NAMES[s] for s in psts]
    return out


def run_batch_all(args):
    """--mode batch --batch-all: every problem of the 64-problem batched
    workload (meshes 64^2..512^2, P 2..5, subdomains 4^2..32^2, N_t 30 to
    16 000: five orders of magnitude of work) under a budget of
    --batch-sweeps sweeps each, so the run is bounded by the largest problem's
    sweeps rather than its convergence: one at a time, all concurrently
    (hz_solve_batch, a stream per solve) and concurrently with the sweeps of
    the packable ones issued as one packed launch per step.  FP32 sweeps
    (20 WaveHoltz iterations), FP64 refinement; the kernel choice is the size
    heuristic (autotuning times every variant, several sweeps each, which on
    the largest problems would cost more than the budget).  Reports every
    problem's status, sweeps, DOF-updates and N_t, and the throughput of each
    schedule."""
    import paper_2606_21695_gb300 as hz
    from paper_2606_21695_gb300.api import Case
    from workloads import configs

    wls = configs.config4()
    cases = [Case(w) for w in wls]
    prs, ns = [c.pr for c in cases], [c.n for c in cases]
    mk = lambda **kw: hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=TOL, max_sweeps=args.batch_sweeps,
                                         autotune=0, **kw)
    out = {"mode": "batch", "problems": len(cases), "sweep_budget": args.batch_sweeps}
    t0 = time.perf_counter()
    seq = [hz.hz_solve(c.pr, mk(pack=0), n=c.n) for c in cases]
    out["sequential_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    st, sts, _, reps = hz.hz_solve_batch(prs, ns, mk(pack=0), 0, want_u=False)
    out["concurrent_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    pst, psts, _, preps = hz.hz_solve_batch(prs, ns, mk(pack=1), 0, want_u=False)
    out["packed_s"] = time.perf_counter() - t0
    dof = sum(r["dof_updates"] for r in reps)
    out["dof_updates"] = dof
    out["dof_updates_per_s"] = {"sequential": sum(s[2]["dof_updates"] for s in seq) / out["sequential_s"],
                                "concurrent": dof / out["concurrent_s"],
                                "packed": sum(r["dof_updates"] for r in preps) / out["packed_s"]}
    out["packed_members"] = sum(r["sweep_variant"] == 4 for r in preps)
    out["per_problem"] = [{"name": w.name, "nodes": c.n, "nt": r["nt"], "status": hz.STATUS_NAMES[s_],
                           "sweeps": r["sweeps"], "rel_residual": r["rel_residual"], "kernel": r["sweep_variant"],
                           "dof_updates": r["dof_updates"]}
                          for w, c, r, s_ in zip(wls, cases, reps, sts)]
    for c in cases:
        c.close()
    return out


def run_batch(args):
    """--mode batch: the cheapest problems of the batched workload solved one
    at a time and together (hz_solve_batch); FP32 sweeps + FP64 refinement."""
    import torch

    import paper_2606_21695_gb300 as hz
    from paper_2606_21695_gb300.api import Case

    if args.batch_all:
        return run_batch_all(args)

    wls = _cheap_cfg4(args.batch)
    cases = [Case(w) for w in wls]
    res = {"mode": "batch", "problems": [w.name for w in wls], "solves": len(cases),
           "cheapest": _batch_group(hz, cases, 5000)}
    for c in cases:
        c.close()
    pw = _cheap_packable_cfg4(min(args.batch, 10))
    pcases = [Case(w) for w in pw]
    res["packable_problems"] = [w.name for w in pw]
    res["cheapest_packable"] = _batch_group(hz, pcases, 5000)
    for c in pcases:
        c.close()
    # many small problems of the batched workload's smallest shape (64^2 quads, P = 2,
    # 4x4-element subdomains), frequencies and sources varied: the launch-bound regime
    from workloads import configs

    small = [configs.Workload(f"small{k:02d}", (0.0, 1.0, 0.0, 1.0), 64, 64, 2, 4, 4, 8.0 + 0.5 * k, "random",
                              (0.3 + 0.01 * k, 0.6 - 0.01 * k), 0.03, speed_seed=100 + k, corr_len=0.1)
             for k in range(args.small_batch)]
    scases = [Case(w) for w in small]
    res["small_problems"] = f"{len(small)} x (64x64 quads, P=2, 16x16 subdomains of 4x4)"
    res["small"] = _batch_group(hz, scases, 5000)
    for c in scases:
        c.close()
    return res


def run_serve(args):
    """--mode serve: the served-stream leg alone (see leg_serve)."""
    import paper_2606_21695_gb300 as hz

    out = leg_serve(hz, args.requests, args.rate, args.serve_pool, args.baseline_requests)
    out["mode"] = "serve"
    return out


def main():
    args = parse()
    if args.mode == "sweep":
        print(json.dumps(run_sweeps(args)), flush=True)
        return
    if args.mode == "batch":
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.mode == "serve":
        print(json.dumps(run_serve(args)), flush=True)
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
