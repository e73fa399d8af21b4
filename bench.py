#!/usr/bin/env python
"""Benchmark of the GPU domain-decomposition Helmholtz solver.

Workload: 256x256 quads on the unit square, degree 3, 32x32 subdomains of
8x8 elements (625 GLL nodes each), Y-shaped channel at c = 1/3 in c = 1,
omega = 64 pi, off-centre Gaussian source; synthetic, seeded.

One step = one full solve to ||b - K u|| <= 1e-8 ||b|| (FP64 global
residual): right-hand side, leapfrog coefficients, FP64 defect correction
whose DD solves run GMRES on the transmission data with one fused sweep
kernel launch (all 1024 subdomain WaveHoltz solves, FP32) per matvec.
Metric: DOF-updates/s = (sum over sweeps of subdomain nodes x (N_t - 1) x
WaveHoltz iterations) / wall time of the solves.

--impl reference times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload: one sweep of a subset of subdomains
per step.
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
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flops x max SM clock
TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 time-to-tolerance leg")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--mode", choices=["solve", "sweep"], default="solve",
                    help="sweep: only run --sweeps DD sweeps of the workload (for ncu captures)")
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--wh-iters", type=int, default=20)
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
def oracle_sample(wl, seconds, nsub_max=1024):
    """Times the FP64 oracle sweep on a bounded subset of subdomains of the
    workload (single-threaded NumPy).  Returns (DOF-updates/s, description)."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:  # pragma: no cover
        threadpool_limits = None
    import numpy as np

    from oracle import dd, sem

    m = sem.Mesh(*wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny)
    gx, gy = m.coords_1d()
    pr = dd.Problem(m, wl.speed(gx, gy), wl.omega, wl.source(gx, gy), wl.boundary())
    nt = pr.choose_nt()
    m_wh = 5
    rhs = pr.rhs()
    lam = np.zeros((m.L, 4, m.NE), complex)
    ctx = threadpool_limits(1) if threadpool_limits else None
    try:
        # calibrate on 2 subdomains, then size the sample to ~seconds
        t0 = time.perf_counter()
        pr.sweep(lam, rhs, nt, 1, subset=[0, 1])
        t_cal = (time.perf_counter() - t0) / (2 * 1)
        nsub = int(max(1, min(nsub_max, seconds / max(t_cal * m_wh, 1e-6))))
        subset = list(range(0, m.L, max(1, m.L // nsub)))[:nsub]
        t0 = time.perf_counter()
        pr.sweep(lam, rhs, nt, m_wh, subset=subset)
        el = time.perf_counter() - t0
    finally:
        if ctx is not None:
            ctx.__exit__(None, None, None)
    dof = len(subset) * m.nlx * m.nly * (nt - 1) * m_wh
    desc = f"one sweep (N_t={nt}, {m_wh} WaveHoltz iterations) over {len(subset)} of {m.L} subdomains, FP64 NumPy"
    return dof / el, desc, el


# ------------------------------------------------------------ our arm ----
def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2606_21695_gb300 as hz
    from paper_2606_21695_gb300.api import Case, boundary_vector
    from workloads import configs

    wl = configs.config2()
    case = Case(wl, device=local)
    n = case.n
    stream = torch.cuda.current_stream()
    opts = hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=TOL, inner_tol=1e-3, wh_iters=20,
                              gmres_restart=60, max_sweeps=5000)
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
    # max time over ranks, total work over ranks
    tot = torch.tensor([elapsed, float(dof)], dtype=torch.float64, device="cuda")
    if world > 1:
        import torch.distributed as tdist

        tmax = tot[:1].clone()
        tdist.all_reduce(tmax, op=tdist.ReduceOp.MAX)
        tsum = tot[1:].clone()
        tdist.all_reduce(tsum, op=tdist.ReduceOp.SUM)
        elapsed_max, dof_all = float(tmax.item()), float(tsum.item())
    else:
        elapsed_max, dof_all = elapsed, float(dof)
    value = dof_all / elapsed_max
    res = [r["rel_residual"] for r in reports]
    nt = reports[0]["nt"]
    P = wl.P
    flops_per_update = 2 * (2 * P + 13)
    dof_per_launch = dof / sweeps
    avg_launch = sweep_s / sweeps
    achieved = flops_per_update * dof_per_launch / avg_launch / 1e12

    out = None
    if rank == 0:
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
            o64 = hz.hz_default_opts(precision=hz.HZ_FP64, tol=TOL, inner_tol=1e-3, wh_iters=20, gmres_restart=60,
                                     max_sweeps=5000)
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
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            v, desc, el = oracle_sample(wl, args.cpu_sample_s)
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, "seconds": el}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (subdomain WaveHoltz) + f64 (outer, residual)",
            "data": "synthetic (seeded generators)",
            "config": {"workload": wl.name, "mesh": f"{wl.nx}x{wl.ny} quads", "degree": P,
                       "subdomains": f"{wl.nx // wl.sub_nx}x{wl.ny // wl.sub_ny} of {wl.sub_nx}x{wl.sub_ny}",
                       "omega": wl.omega, "nt": nt, "wh_iters": opts.wh_iters, "tol": TOL,
                       "outer": "GMRES(60) in FP64 defect correction", "l2": "flushed (256 MB write) before each step",
                       "parallelism": f"{world} independent solves (one per GPU)"},
            "time_to_tol_s": {"fp32_refine": elapsed / args.steps, "fp64": fp64["seconds"] if fp64 else None},
            "fp64_solve": fp64,
            "solve": {"sweeps_per_solve": sweeps / args.steps, "rel_residual_max": max(res),
                      "sweep_kernel": {1: "block", 2: "warp", 3: "cluster"}.get(reports[0]["sweep_variant"]),
                      "refinements": reports[0]["refinements"], "gmres_iters": reports[0]["gmres_iters"],
                      "dof_updates_per_solve": dof / args.steps},
            "roofline": {"kernel": "sweep_kernel<float,3,1> (one launch = one DD sweep)", "bound": "alu",
                         "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                         "algorithmic": f"{flops_per_update} flop/DOF-update x {dof_per_launch:.4g} DOF-updates/launch",
                         "avg_launch_ms": avg_launch * 1e3, "launch_share": sweep_s / elapsed},
            "cpu_baseline": cpu,
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
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from workloads import configs

    wl = configs.config2()
    vals = []
    desc = ""
    for k in range(args.warmup + args.steps):
        v, desc, el = oracle_sample(wl, seconds=3.0, nsub_max=16)
        if k >= args.warmup:
            vals.append((v, el))
    tot_t = sum(el for _, el in vals)
    value = sum(v * el for v, el in vals) / tot_t
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generators)",
        "config": {"workload": wl.name, "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_sweeps(args):
    """--mode sweep: set up the workload and launch --sweeps homogeneous DD
    sweeps through the C ABI (the launch configuration of the solve)."""
    import torch

    import paper_2606_21695_gb300 as hz
    from paper_2606_21695_gb300.api import Case
    from workloads import configs

    wl = configs.config2()
    case = Case(wl)
    nt = hz.hz_problem_nt(case.pr)
    nl = hz.hz_lambda_size(case.pr)
    g = torch.Generator(device="cuda").manual_seed(0)
    lin = torch.randn(2 * nl, dtype=torch.float64, device="cuda", generator=g) * 1e-2
    lout = torch.zeros_like(lin)
    prec = hz.HZ_FP32_REFINE if args.precision == "fp32" else hz.HZ_FP64
    for _ in range(args.sweeps):
        hz.hz_sweep(case.pr, prec, nt, args.wh_iters, 0.0, lin, lout)
    torch.cuda.synchronize()
    case.close()
    return {"mode": "sweep", "sweeps": args.sweeps, "nt": nt, "precision": args.precision, "wh_iters": args.wh_iters}


def main():
    args = parse()
    if args.mode == "sweep":
        print(json.dumps(run_sweeps(args)), flush=True)
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
