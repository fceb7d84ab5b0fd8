"""Benchmark: N1280-shaped Helmholtz solves/s to a true FP64 relative residual of 1e-8.

One step = one complete solve (hz_solve through the C ABI) of the synthetic
2560x1920x70 system (coefficient seed 21, right-hand side seed 22, Earth-radius
vertical unit), mixed precision (FP32 inner BiCGStab + T^-1, FP64 outer
residual and update), operator already set up on the GPU, b resident in HBM.
Every vector is 1.4-2.8 GB, far larger than the 129 MB L2, so no flush is
needed between steps.  The plain FP64 solver is timed on the same system in the
same run (fp64_* keys).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload n1280|mixed640|plain96] [--z-unit radius|m]

Under torchrun every rank solves its own copy (replicas: the path has no
data-parallel exchange) and rank 0 prints one JSON line.  --impl reference
times the CPU oracle (C, its OpenMP build on all host cores) instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "N1280-shape solves/s at 1e-8 FP64 residual, mixed vs FP64; % of HBM BW"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n1280", choices=["n1280", "mixed640", "plain96", "batched", "learned", "nnfwd", "fig1", "table1"])
    ap.add_argument("--train-systems", type=int, default=200)
    ap.add_argument("--test-systems", type=int, default=50)
    ap.add_argument("--train-steps", type=int, default=800)
    ap.add_argument("--z-unit", default="radius", choices=["radius", "m"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--eta", type=float, default=None,
                    help="inner relative tolerance of the mixed solver (default: the fastest of 1e-3, 3e-4, 1e-4 in an "
                         "untimed sweep before the timed region)")
    ap.add_argument("--restart", type=int, default=150, help="forced BiCGStab restart period")
    ap.add_argument("--precond", default="tri", choices=["tri", "trisor"],
                    help="preconditioner of the headline solves: T^-1 or tri-SOR (Sec. 2)")
    ap.add_argument("--no-trisor", action="store_true", help="skip the tri-SOR side measurement")
    ap.add_argument("--no-table1", action="store_true", help="skip the paper's Table 1 comparison")
    ap.add_argument("--no-bands16", action="store_true", help="skip the 16-bit horizontal-band solves")
    ap.add_argument("--no-batched", action="store_true", help="skip the small-system batches")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-stage line")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed solves with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--dims", type=int, nargs=3, metavar=("NX", "NY", "NZ"),
                    help="override the workload's grid (same recipe and seeds; for profiling smaller cases)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven inner loop (same kernels); ncu cannot profile kernels inside conditional graphs")
    ap.add_argument("--variants", type=int, nargs=2, metavar=("PRE32", "MV32"),
                    help="fix the FP32 Thomas and stencil variants instead of autotuning them (profiling a known launch "
                         "shape); FP64 and tri-SOR kernels are still tuned unless --no-fp64 / --no-trisor")
    ap.add_argument("--sor-variants", type=int, nargs=3, metavar=("PASS", "MATVEC", "FIRST"),
                    help="after tuning, fix the FP32 tri-SOR colour-pass, matvec and first-pass variants (profiling a "
                         "known launch shape)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def replica_max(value, device):
    """Largest value over the ranks of the process group (all-reduce MAX); the value itself
    without a group or with one rank.  The replicas' slowest time is the job's time."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput of `world` replicas that each processed `units_per_rank` units,
    the slowest taking `seconds`."""
    return world * units_per_rank / seconds


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_inputs(args, workload=None):
    import gen

    w = gen.WORKLOADS[workload or args.workload]
    nx, ny, nz = args.dims if args.dims else (w["nx"], w["ny"], w["nz"])
    A = gen.make_operator(nx, ny, nz, w["seed_coef"], z_unit=args.z_unit)
    b = gen.make_rhs(nx, ny, nz, w["seed_rhs"])
    return (nx, ny, nz), A, b


def _oracle_pieces(A, b, Ah32, bh32, threads, iters):
    """Wall time of one FP64 true residual and of `iters` (ascending) FP32 BiCGStab runs of
    the oracle on the full system with the given OpenMP threads."""
    import oracle

    used = oracle.use_openmp(True, threads)
    x = np.zeros_like(b)
    t0 = time.perf_counter()
    oracle.residual(A, b, x)
    t_res = time.perf_counter() - t0
    t_k = {}
    for k in iters:
        t0 = time.perf_counter()
        oracle.bicgstab(Ah32, bh32, eta=1e-30, maxit=k, fp32=True)
        t_k[k] = time.perf_counter() - t0
    return used, t_res, t_k


def cpu_baseline(A, b, dims, outer, inner, full_solve=True):
    """The oracle as it stands (plain C; its OpenMP build shares out the point and column loops
    and gives the same bits as the serial build) timed on this host's cores on a bounded sample
    of the same solve: one FP64 true residual, and the oracle's own FP32 BiCGStab (T^-1, every
    vector update and dot product included) run for 1 and 3 iterations, which separates the
    cost of an inner iteration from that of an inner solve's start.  The solve is composed from
    them with the GPU solve's refinement steps and inner iterations.  The same sample with one
    thread is reported too; and, where it takes seconds, a full oracle mixed solve of the
    640x480x70 system (seeds 11/12), not extrapolated."""
    import oracle

    nx, ny, nz = dims
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.use_openmp(True, cores)
    Ah32 = oracle.scale(A).astype(np.float32)
    bh32 = (b / A[0]).astype(np.float32)
    t_prep = time.perf_counter() - t0
    used, t_res, t_k = _oracle_pieces(A, b, Ah32, bh32, cores, (1, 3))
    t_it = max((t_k[3] - t_k[1]) / 2.0, 1e-9)
    t_start = max(t_k[1] - t_it, 0.0)
    t_solve = (outer + 1) * t_res + outer * t_start + inner * t_it
    used1, t_res1, t_k1 = _oracle_pieces(A, b, Ah32, bh32, 1, (1,))
    t_solve1 = (outer + 1) * t_res1 + inner * t_k1[1]
    out = {
        "value": 1.0 / t_solve,
        "unit": "solves/s",
        "cores": used,
        "kind": "oracle",
        "sample": (f"oracle (C, OpenMP build, {used} threads on {cores} host cores, FP32 inner / FP64 outer) timed on "
                   f"the full {nx}x{ny}x{nz} system: true residual {t_res:.2f} s, its FP32 BiCGStab for 1 and 3 "
                   f"iterations {t_k[1]:.2f} / {t_k[3]:.2f} s (an iteration {t_it:.2f} s, a start {t_start:.2f} s; "
                   f"scaling and FP32 casts {t_prep:.1f} s, not counted); composed as {outer + 1} residuals + "
                   f"{outer} starts + {inner} iterations, the counts of the GPU mixed solve of this system"),
        "single_thread": {"value": 1.0 / t_solve1, "unit": "solves/s", "cores": used1,
                          "sample": f"the same pieces with one thread: true residual {t_res1:.2f} s, one FP32 "
                                    f"iteration with its start {t_k1[1]:.2f} s; composed as {outer + 1} residuals + "
                                    f"{inner} iterations (each charged a start)"},
    }
    del Ah32, bh32
    if full_solve:
        import gen

        w = gen.WORKLOADS["mixed640"]
        A6 = gen.make_operator(w["nx"], w["ny"], w["nz"], w["seed_coef"], z_unit="radius")
        b6 = gen.make_rhs(w["nx"], w["ny"], w["nz"], w["seed_rhs"])
        oracle.use_openmp(True, cores)
        t0 = time.perf_counter()
        _, info = oracle.solve(A6, b6, mode=oracle.MODE_MIXED, tol=1e-8, max_outer=20, max_inner=4000)
        sec = time.perf_counter() - t0
        out["full_solve_640x480x70"] = {
            "value": 1.0 / sec, "unit": "solves/s", "cores": used, "seconds": round(sec, 2),
            "outer": info["outer"], "inner": info["inner"], "true_rel_residual": info["R"],
            "sample": "one complete oracle mixed solve (FP32 inner, FP64 outer, tol 1e-8, scaling included) of the "
                      "640x480x70 system, seeds 11/12, Earth-radius unit"}
    oracle.use_openmp(False)
    return out


# Refinement steps and inner iterations of the GPU mixed solve of the full-size
# workloads (same algorithm and seeds; the bench's own run on a GB300): the work
# the oracle's timed pieces are composed with where a full oracle solve would
# take hours.
GPU_COUNTS = {("n1280", "radius"): (3, 515)}


def run_reference(args):
    """The oracle as it stands, timed on all host cores (its OpenMP build; same bits as the
    serial one) for this arm's workload and metric: per step a full oracle mixed solve where
    that takes seconds, otherwise a bounded sample of the solve (one FP64 true residual and one
    FP32 inner iteration of the full system) composed with the solve's counts."""
    import oracle

    world, rank, local = dist_setup()
    if rank != 0:
        return
    dims, A, b = make_inputs(args)
    n = dims[0] * dims[1] * dims[2]
    key = (args.workload, args.z_unit)
    cores = os.cpu_count() or 1
    used = oracle.use_openmp(True, cores)
    vals = []
    cb = None
    if n > 2_000_000:
        if key not in GPU_COUNTS:
            print(json.dumps({"impl": "reference", "unavailable": f"no solve counts recorded for {key} and a full "
                                                                  f"oracle solve of {n} points takes hours"}))
            return
        outer, inner = GPU_COUNTS[key]
        Ah32 = oracle.scale(A).astype(np.float32)
        bh32 = (b / A[0]).astype(np.float32)
    for i in range(args.warmup + args.steps):
        if n <= 2_000_000:
            t0 = time.perf_counter()
            _, info = oracle.solve(A, b, mode=oracle.MODE_MIXED, tol=1e-8, max_outer=20, max_inner=4000)
            sec = time.perf_counter() - t0
            cb = {"value": 1.0 / sec, "unit": "solves/s", "cores": used, "kind": "oracle",
                  "sample": f"full oracle mixed solve (C, OpenMP build, {used} threads; FP32 inner, FP64 outer) of the "
                            f"{'x'.join(map(str, dims))} system: {info['outer']} refinement steps, {info['inner']} "
                            f"inner iterations, true R {info['R']:.2e}, {sec:.2f} s"}
        else:
            _, t_res, t_k = _oracle_pieces(A, b, Ah32, bh32, cores, (1,))
            t_solve = (outer + 1) * t_res + inner * t_k[1]
            cb = {"value": 1.0 / t_solve, "unit": "solves/s", "cores": used, "kind": "oracle",
                  "sample": f"oracle (C, OpenMP build, {used} threads) on the full {'x'.join(map(str, dims))} system: "
                            f"one FP64 true residual {t_res:.2f} s and one FP32 BiCGStab iteration with its start "
                            f"{t_k[1]:.2f} s per step, composed as {outer + 1} residuals + {inner} iterations (the "
                            f"GPU mixed solve's counts for this system; the full solve would take "
                            f"{t_solve / 60:.0f} min)"}
        if i >= args.warmup:
            vals.append(cb["value"])
    oracle.use_openmp(False)
    v = statistics.median(vals)
    cb["value"] = v
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
        "config": {"workload": f"{args.workload} {'x'.join(map(str, dims))} z_unit={args.z_unit}"},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def paper_table1(op, bd, x, stream, dims, restart=150, ablation=True):
    """The paper's Table 1 on this system: iterations and time of its mixed-precision solver (one
    BiCGStab solve, x in FP64, everything else FP32, Sec. 3) and of the 64-bit solver to the
    halting criteria R_c = 1e-3 and 1e-4 (the recursive residual of the scaled system), with the
    paper's tri-SOR preconditioner (3 sweeps, omega 1.5) and with T^-1; the mixed-precision solver
    also with FP32 global sums (Sec. 4's original sums) and, at 1e-4, without the restart at 150
    iterations.  Each entry is one solve after an untimed one, timed with CUDA events."""
    import torch

    import paper_1811_03852_gb300 as hz

    pres = [("trisor", hz.HZ_PRE_TRISOR), ("tri", hz.HZ_PRE_TRI)] if dims[0] % 2 == 0 else [("tri", hz.HZ_PRE_TRI)]
    rows = {}

    def one(**kw):
        kw.setdefault("restart", restart)
        p = hz.default_params(**kw)
        op.solve(bd, x, params=p, raise_on_error=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        info = op.solve(bd, x, params=p, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return {"iterations": info["inner_iters"], "ms": round(ms, 2),
                "ms_per_iteration": round(ms / max(1, info["inner_iters"]), 3),
                "R_recursive_scaled": info["scaled_rel_residual"], "R_true": info["true_rel_residual"],
                "status": info["status"]}

    for pname, pc in pres:
        for rc in (1e-3, 1e-4):
            key = f"{pname} R_c={rc:g}"
            mp = one(mode=hz.HZ_MODE_PAPER_MP, precond=pc, tol=rc)
            dp = one(mode=hz.HZ_MODE_PAPER_DP, precond=pc, tol=rc)
            row = {"mixed": mp, "double": dp, "time_ratio_double_over_mixed": round(dp["ms"] / mp["ms"], 3)}
            if pname == pres[0][0]:
                row["mixed_fp32_global_sums"] = one(mode=hz.HZ_MODE_PAPER_MP, precond=pc, tol=rc, dot_fp32=1)
                if ablation and rc == 1e-4:
                    row["mixed_no_restart"] = one(mode=hz.HZ_MODE_PAPER_MP, precond=pc, tol=rc, restart=10**9)
            rows[key] = row
    return rows


def table1_hard(restart=150):
    """paper_table1 on the 640x480x70 system of the metres family (seeds 11/12)."""
    import torch

    import gen
    import paper_1811_03852_gb300 as hz

    w = gen.WORKLOADS["mixed640"]
    dims = (w["nx"], w["ny"], w["nz"])
    A = gen.make_operator(*dims, w["seed_coef"], z_unit="m")
    b = gen.make_rhs(*dims, w["seed_rhs"])
    stream = torch.cuda.current_stream()
    op = hz.Operator(A, stream=stream)
    op.autotune(fp64=True, trisor=True)
    bd = torch.from_numpy(b.reshape(-1)).cuda()
    x = torch.empty_like(bd)
    rows = paper_table1(op, bd, x, stream, dims, restart=restart)
    op.close()
    return {f"mixed640 {'x'.join(map(str, dims))} z_unit=m": rows}


def run_table1(args):
    """The paper's Table 1 comparison alone (default: the N1280 system)."""
    import torch

    import paper_1811_03852_gb300 as hz

    torch.cuda.set_device(0)
    dims, A, b = make_inputs(args, "n1280")
    stream = torch.cuda.current_stream()
    op = hz.Operator(A, stream=stream)
    op.autotune(fp64=True, trisor=dims[0] % 2 == 0)
    bd = torch.from_numpy(b.reshape(-1)).cuda()
    x = torch.empty_like(bd)
    rows = {f"n1280 {'x'.join(map(str, dims))} z_unit={args.z_unit}":
            paper_table1(op, bd, x, stream, dims, restart=args.restart)}
    op.close()
    rows.update(table1_hard(args.restart))
    print(json.dumps({"workload": "paper Table 1 (synthetic)", "table1": rows}), flush=True)


def run_ours(args):
    import torch

    import paper_1811_03852_gb300 as hz

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    wall = {"start": time.perf_counter()}  # wall-clock marks of the bench's sections
    dims, A, b = make_inputs(args)
    nx, ny, nz = dims
    n = nx * ny * nz
    stream = torch.cuda.current_stream()
    op = hz.Operator(A, stream=stream)
    bd = torch.from_numpy(b.reshape(-1)).to(f"cuda:{dev}")
    x = torch.empty(n, dtype=torch.float64, device=f"cuda:{dev}")
    use_sor = (args.precond == "trisor" or not args.no_trisor) and nx % 2 == 0
    # launch-shape search, outside the timed region
    if args.variants:
        if not args.no_fp64 or use_sor:
            op.autotune(fp64=not args.no_fp64, trisor=use_sor)
        op.set_variants(pre32=args.variants[0], mv32=args.variants[1])
        variants = op.variants()
    else:
        variants = op.autotune(fp64=not args.no_fp64, trisor=use_sor)
    if use_sor and args.sor_variants:
        for kind, vid in enumerate(args.sor_variants):
            op.set_sor_variant(hz.HZ_PREC_FP32, kind, vid)
    if use_sor:
        variants["trisor"] = {f"{'fp64' if p == hz.HZ_PREC_FP64 else 'fp32'}/{('pass', 'matvec', 'first')[k]}": v
                              for (p, k), v in op.sor_variants().items()}
    ug = 0 if args.no_graph else 1
    pc = hz.HZ_PRE_TRISOR if args.precond == "trisor" else hz.HZ_PRE_TRI
    wall["inputs_autotune"] = time.perf_counter()
    # the inner tolerance eta of the refinement steps (a free parameter of the method): the fastest of
    # a few, each timed on one solve of this system after an untimed one, unless given
    eta_sweep = None
    if args.eta is None:
        eta_sweep = {}
        for eta in (1e-3, 3e-4, 1e-4):
            pe = hz.default_params(mode=hz.HZ_MODE_MIXED_IR, tol=1e-8, inner_tol=eta, restart=args.restart,
                                   use_graph=ug, precond=pc)
            op.solve(bd, x, params=pe)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ie = op.solve(bd, x, params=pe)
            e1.record(stream)
            torch.cuda.synchronize()
            eta_sweep[f"{eta:g}"] = {"ms": round(e0.elapsed_time(e1), 2), "outer": ie["outer_iters"],
                                     "inner": ie["inner_iters"]}
        args.eta = float(min(eta_sweep, key=lambda k: eta_sweep[k]["ms"]))
    pm = hz.default_params(mode=hz.HZ_MODE_MIXED_IR, tol=1e-8, inner_tol=args.eta, restart=args.restart, use_graph=ug,
                           precond=pc)
    p64 = hz.default_params(mode=hz.HZ_MODE_FP64, tol=1e-8, restart=args.restart, use_graph=ug, precond=pc)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(params, steps, warmup, region=False):
        infos = []
        for _ in range(warmup):
            op.solve(bd, x, params=params)
        barrier()
        if region:
            torch.cuda.cudart().cudaProfilerStart()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            infos.append(op.solve(bd, x, params=params))
        e1.record(stream)
        barrier()
        if region:
            torch.cuda.cudart().cudaProfilerStop()
        ms = replica_max(e0.elapsed_time(e1), f"cuda:{dev}")
        return ms, infos

    # setup (operator update: scaling + Thomas factors), timed separately
    Ad = torch.from_numpy(A).to(f"cuda:{dev}")
    su = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        op.update(Ad)  # device-resident coefficients: 7-band copy + scaling + Thomas factors
        e1.record(stream)
        torch.cuda.synchronize()
        su.append(e0.elapsed_time(e1))
    del Ad

    wall["eta_setup"] = time.perf_counter()
    with Clocks(dev) as clk:
        ms, infos = timed(pm, args.steps, args.warmup, region=args.profile_region)
    wall["timed"] = time.perf_counter()
    clocks = clk.summary()
    for i in infos:
        assert i["status"] == 0 and i["true_rel_residual"] <= 1e-8, i
    value = job_rate(world, args.steps, ms * 1e-3)
    launches = int(sum(i["kernel_launches"] for i in infos))

    fp64 = None
    if not args.no_fp64:
        ms64, inf64 = timed(p64, max(1, min(2, args.steps)), 1)
        for i in inf64:
            assert i["status"] == 0 and i["true_rel_residual"] <= 1e-8, i
        fp64 = {"value": world * len(inf64) / (ms64 * 1e-3), "ms_per_solve": ms64 / len(inf64),
                "outer": inf64[0]["outer_iters"], "inner": inf64[0]["inner_iters"]}
        # the FP64 iteration moves 38 FP64 values per point (304 B): its rate against the copy peak
        # (the FP64 residual passes, two per solve, are counted in the time, not in the bytes)
        ms_it = fp64["ms_per_solve"] / max(1, fp64["inner"])
        gbs64 = 304.0 * nx * ny * nz / (ms_it * 1e-3) / 1e9
        fp64.update({"ms_per_inner": round(ms_it, 3), "iteration_GBps": round(gbs64, 1),
                     "frac_of_hbm": round(gbs64 / measured_peaks()[0], 3)})

    # the paper's tri-SOR preconditioner (3 red-black sweeps, omega 1.5) on the same system, one solve each
    trisor = None
    if not args.no_trisor and args.precond == "tri" and nx % 2 == 0:
        ps = hz.default_params(mode=hz.HZ_MODE_MIXED_IR, tol=1e-8, inner_tol=args.eta, restart=args.restart,
                               use_graph=ug, precond=hz.HZ_PRE_TRISOR)
        mss, infs = timed(ps, 1, 1)
        for i in infs:
            assert i["status"] == 0 and i["true_rel_residual"] <= 1e-8, i
        trisor = {"mixed": {"value": round(world / (mss * 1e-3), 4), "ms_per_solve": round(mss, 3),
                            "outer": infs[0]["outer_iters"], "inner": infs[0]["inner_iters"]}}
        if not args.no_fp64:
            ps64 = hz.default_params(mode=hz.HZ_MODE_FP64, tol=1e-8, restart=args.restart, use_graph=ug,
                                     precond=hz.HZ_PRE_TRISOR)
            mss64, infs64 = timed(ps64, 1, 1)
            for i in infs64:
                assert i["status"] == 0 and i["true_rel_residual"] <= 1e-8, i
            trisor["fp64"] = {"value": round(world / (mss64 * 1e-3), 4), "ms_per_solve": round(mss64, 3),
                              "outer": infs64[0]["outer_iters"], "inner": infs64[0]["inner_iters"]}
        op.profile(True)
        op.solve(bd, x, params=ps)
        sp = {k: v for k, v in op.profile_read().items() if v[0] > 0}
        op.profile(False)
        st = sum(v[1] for v in sp.values())
        trisor["kernels"] = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / st, 4),
                                 "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1) if v[1] > 0 else None}
                             for k, v in sp.items()}

    wall["fp64_trisor"] = time.perf_counter()
    # 16-bit storage of the horizontal bands (BF16 and FP16) in the same mixed solve
    bands16 = None
    if not args.no_bands16:
        bands16 = {}
        p16 = hz.default_params(mode=hz.HZ_MODE_MIXED_IR, tol=1e-8, inner_tol=args.eta, restart=args.restart,
                                use_graph=ug, max_outer=30)
        keep = op.variants()
        for name, fmt in (("bf16", hz.HZ_BANDS_BF16), ("fp16", hz.HZ_BANDS_FP16)):
            op.set_band_format(fmt)
            v16 = op.autotune(fp64=False)  # the stencil variant that suits the narrower loads
            ms16, inf16 = timed(p16, max(1, min(2, args.steps)), 1)
            op.profile(True)
            op.solve(bd, x, params=p16)
            pr16 = {k: v for k, v in op.profile_read().items() if v[0] > 0 and k != "k_setup"}
            op.profile(False)
            bands16[name] = {
                "value": round(world * len(inf16) / (ms16 * 1e-3), 4), "ms_per_solve": round(ms16 / len(inf16), 3),
                "outer": inf16[0]["outer_iters"], "inner": inf16[0]["inner_iters"],
                "true_rel_residual": max(i["true_rel_residual"] for i in inf16),
                "status": [i["status"] for i in inf16],
                "ms_per_inner": round(ms16 / len(inf16) / max(1, inf16[0]["inner_iters"]), 3),
                "kernels_GBps": {k: round(v[2] / (v[1] * 1e-3) / 1e9, 1) for k, v in pr16.items() if v[1] > 0},
                "kernels_ms_per_launch": {k: round(v[1] / v[0], 4) for k, v in pr16.items()},
                "variants": {"pre32": v16["pre32"], "mv32": v16["mv32"]}}
        op.set_band_format(hz.HZ_BANDS_FP32)
        op.set_variants(pre32=keep["pre32"], mv32=keep["mv32"])

    wall["bands16"] = time.perf_counter()
    # batches of small systems and of many right-hand sides of one operator (one persistent launch each)
    batched = None
    if not args.no_batched:
        batched = batched_small(max(1, min(3, args.steps)), 1)

    wall["batched"] = time.perf_counter()
    # the learned stage, trained and evaluated at 640x480x70 on the hard (metres) family (a reduced
    # count of systems; --workload learned runs the full 200 / 50)
    learned = None
    if not args.no_learned:
        learned = learned_line((640, 480, 70), [(10000 + 2 * i, 10001 + 2 * i) for i in range(8)],
                               [(20000 + 2 * i, 20001 + 2 * i) for i in range(2)], 160, "m")

    wall["learned"] = time.perf_counter()
    # the paper's own mixed-precision solver against the 64-bit one (Table 1, Sec. 4): on this
    # system, and on the hard (metres) family at 640x480x70, where the solve from x0 = 0 takes
    # tens of iterations as the paper's did
    table1 = None
    if not args.no_table1 and not args.no_fp64:
        table1 = {f"{args.workload} {nx}x{ny}x{nz} z_unit={args.z_unit}":
                  paper_table1(op, bd, x, stream, dims, restart=args.restart, ablation=False)}
        table1.update(table1_hard(args.restart))

    wall["table1"] = time.perf_counter()
    # end to end through the public API with host buffers (pinned b, pinned x)
    bh = torch.from_numpy(b.reshape(-1)).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    op.solve(bh, xh, params=pm)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(3, args.steps))
    for _ in range(e2e_steps):
        op.solve(bh, xh, params=pm)
    barrier()
    e2e_s = replica_max(time.perf_counter() - t0, f"cuda:{dev}")
    e2e = {"value": job_rate(world, e2e_steps, e2e_s), "unit": "solves/s", "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n}

    # per-kernel profile of one more solve (CUDA events around every launch on the op's stream)
    op.profile(True)
    op.solve(bd, x, params=pm)
    prof = op.profile_read()
    op.profile(False)
    busy = {k: v for k, v in prof.items() if v[0] > 0 and k != "k_setup"}
    tot_ms = sum(v[1] for v in busy.values())
    dom = max(busy, key=lambda k: busy[k][1])
    la, kms, kby = busy[dom]
    peak, peak_kind = measured_peaks()
    achieved = kby / (kms * 1e-3) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tp):
        try:
            from paper_1811_03852_gb300 import _build

            # DRAM bytes per launch of the autotuned variant from an ncu capture (scaled to
            # this workload), valid only while that variant's source files are unchanged
            tj = json.load(open(tp))
            ent = tj.get(dom)
            kind = "mv32" if dom.startswith("k_mv") else "pre32"
            rec = (ent or {}).get("variants", {}).get(str(variants.get(kind)))
            if (rec and ent.get("workload") == args.workload and rec.get("src") == _build.src_hash(rec["files"])):
                traffic = rec["bytes_per_launch"]
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dom,
                "bytes_per_launch": kby / la, "launches": la, "avg_launch_ms": kms / la,
                "peak_source": f"{peak_kind} hbm_gbs"}
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / tot_ms, 4),
                   "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1) if v[1] > 0 else None} for k, v in busy.items()}

    wall["e2e_profile"] = time.perf_counter()
    if rank != 0:
        return
    cb = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cb = cpu_baseline(A, b, dims, infos[0]["outer_iters"], infos[0]["inner_iters"])
        except MemoryError:
            cb = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": "host memory exhausted"}
    wall["cpu_baseline"] = time.perf_counter()
    marks = list(wall.items())
    sections_s = {k: round(t - marks[i - 1][1], 1) for i, (k, t) in enumerate(marks) if i > 0}
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
        "config": {"workload": f"{args.workload} {nx}x{ny}x{nz} z_unit={args.z_unit} seeds "
                               f"{make_seed(args)} mixed IR tol 1e-8 eta {args.eta:g} precond {args.precond}",
                   "l2": "inputs larger than L2 (vectors 1.4-2.8 GB)", "parallelism": f"replicas x{world}"},
        "eta_sweep": eta_sweep,
        "solve": {"outer": infos[0]["outer_iters"], "inner": infos[0]["inner_iters"],
                  "true_rel_residual": infos[0]["true_rel_residual"],
                  "ms_per_inner": round(ms / args.steps / max(1, infos[0]["inner_iters"]), 3),
                  "inner_all_timed": sorted({i["inner_iters"] for i in infos})},
        "device": {"name": torch.cuda.get_device_name(dev),
                   "sms": torch.cuda.get_device_properties(dev).multi_processor_count},
        "fp64": fp64,
        "mixed_over_fp64": round(value / fp64["value"], 3) if fp64 else None,
        "trisor": trisor,
        "bands16": bands16,
        "batched": batched,
        "learned": learned,
        "paper_table1": table1,
        "setup_ms": round(min(su), 3),
        "variants": variants,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roofline,
        "kernels": kernels,
        "cpu_baseline": cb,
        "clocks": clocks,
        "bench_sections_s": sections_s,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def make_seed(args):
    import gen

    w = gen.WORKLOADS[args.workload]
    return f"{w['seed_coef']}/{w['seed_rhs']}"


def batched_measure(ops, bs, xs, dims_list, strategy, steps, warmup, use_graph=1):
    """Time solve_batched on a prepared batch: systems/s, ms per batch, iterations and the
    algorithmic traffic (152 B per point and inner iteration, 88 B per point and residual pass)."""
    import torch

    import paper_1811_03852_gb300 as hz

    for _ in range(max(1, warmup)):
        hz.solve_batched(ops, bs, xs, strategy=strategy, use_graph=use_graph)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    infos = None
    for _ in range(steps):
        infos = hz.solve_batched(ops, bs, xs, strategy=strategy, use_graph=use_graph)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    npts = [nx * ny * nz for nx, ny, nz in dims_list]
    inner = sum(i["inner_iters"] * n for i, n in zip(infos, npts))
    outer = sum((i["outer_iters"] + 1) * n for i, n in zip(infos, npts))
    gbs = (152.0 * inner + 88.0 * outer) / (ms * 1e-3) / 1e9
    peak, _ = measured_peaks()
    return {"systems_per_s": round(len(ops) / (ms * 1e-3), 3), "ms_per_batch": round(ms, 3),
            "max_true_rel_residual": max(i["true_rel_residual"] for i in infos),
            "status": sorted({i["status"] for i in infos}),
            "inner_iters": [i["inner_iters"] for i in infos],
            # the persistent strategy reports its one launch in every system's record
            "kernel_launches": (max if strategy == hz.HZ_BATCH_PERSISTENT else sum)(i["kernel_launches"] for i in infos),
            "effective_GBps": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 3)}


def batched_small(steps, warmup, z_unit="m"):
    """Batches of systems too small to fill the GPU alone, where the persistent launch is the
    automatic strategy: 64 distinct systems of 48x36x70, and 32 right-hand sides of one 192x144x70
    operator; persistent (graph-replayed) against sequential.  Metres family: hundreds of inner
    iterations per system, so the steady state of the inner phases dominates."""
    import torch

    import gen
    import paper_1811_03852_gb300 as hz

    out = {}
    dims = (48, 36, 70)
    ops = [hz.Operator(gen.make_operator(*dims, 3000 + 2 * i, z_unit=z_unit)) for i in range(64)]
    bs = [torch.from_numpy(gen.make_rhs(*dims, 3001 + 2 * i).reshape(-1)).cuda() for i in range(64)]
    xs = [torch.empty_like(b) for b in bs]
    out["64 systems 48x36x70"] = {
        "persistent_graph": batched_measure(ops, bs, xs, [dims] * 64, hz.HZ_BATCH_PERSISTENT, steps, warmup),
        "sequential": batched_measure(ops, bs, xs, [dims] * 64, hz.HZ_BATCH_SEQUENTIAL, steps, warmup)}
    del ops, bs, xs
    dims = (192, 144, 70)
    op = hz.Operator(gen.make_operator(*dims, 3200, z_unit=z_unit))
    bs = [torch.from_numpy(gen.make_rhs(*dims, 3201 + i).reshape(-1)).cuda() for i in range(32)]
    xs = [torch.empty_like(b) for b in bs]
    out["32 right-hand sides of one 192x144x70 operator"] = {
        "persistent_graph": batched_measure([op] * 32, bs, xs, [dims] * 32, hz.HZ_BATCH_PERSISTENT, steps, warmup),
        "sequential": batched_measure([op] * 32, bs, xs, [dims] * 32, hz.HZ_BATCH_SEQUENTIAL, steps, warmup)}
    return out


def run_batched(args):
    """32 uneven systems (192x144, 320x240, 640x480; 70 levels) solved together per step, and the
    small-system batches."""
    import torch

    import gen
    import paper_1811_03852_gb300 as hz

    torch.cuda.set_device(0)
    specs = [gen.batched_spec(i) for i in range(32)]
    ops, bs, xs, dims_list = [], [], [], []
    for s in specs:
        A = gen.make_operator(s["nx"], s["ny"], s["nz"], s["seed_coef"], z_unit=args.z_unit)
        b = gen.make_rhs(s["nx"], s["ny"], s["nz"], s["seed_rhs"])
        ops.append(hz.Operator(A))
        bs.append(torch.from_numpy(b.reshape(-1)).cuda())
        xs.append(torch.empty(b.size, dtype=torch.float64, device="cuda"))
        dims_list.append((s["nx"], s["ny"], s["nz"]))
    _, kind = measured_peaks()
    auto = batched_measure(ops, bs, xs, dims_list, hz.HZ_BATCH_AUTO, args.steps, args.warmup)
    persistent = batched_measure(ops, bs, xs, dims_list, hz.HZ_BATCH_PERSISTENT, args.steps, args.warmup)
    del ops, bs, xs
    small = batched_small(args.steps, args.warmup)
    print(json.dumps({"workload": "batched 32 systems (192x144, 320x240, 640x480) x 70, mixed IR tol 1e-8",
                      "points": int(sum(a * b * c for a, b, c in dims_list)),
                      "strategy": "auto (sequential: every system fills the GPU)", **auto,
                      "persistent_graph": persistent, "small_systems": small, "peak_source": f"{kind} hbm_gbs"}),
          flush=True)


def learned_line(dims, train_systems, test_systems, steps, z_unit, lr=1e-3):
    """The learned stage at one size: trained by hz_nn_train on fresh systems (operator-weighted
    loss), then on held-out systems its own gain (the residual it leaves, relative to its input) and
    the solves to 1e-8: plain and learned FGMRES(30), plain mixed BiCGStab."""
    import torch

    import gen
    import paper_1811_03852_gb300 as hz
    from paper_1811_03852_gb300 import learn

    nx, ny, nz = dims
    n = nx * ny * nz
    net = hz.Net(learn.init_params(1))
    t0 = time.perf_counter()
    losses = learn.train(net, train_systems, dims, steps=steps, batch=16, crop=min(64, nx - 8, ny - 1), lr=lr,
                         seed=7, z_unit=z_unit)
    t_train = time.perf_counter() - t0
    rows = []
    for sc, sr in test_systems:
        op = hz.Operator(gen.make_operator(*dims, sc, z_unit=z_unit))
        b = torch.from_numpy(gen.make_rhs(*dims, sr).reshape(-1)).cuda()
        x = torch.empty_like(b)
        # the stage's own gain on a pair of this held-out system
        xs = torch.empty_like(b)
        op.solve(b, xs, mode=hz.HZ_MODE_FP64, tol=1e-11, raise_on_error=False)
        xk = torch.empty_like(b)
        op.solve(b, xk, max_outer=1, max_inner=8, inner_tol=1e-12, raise_on_error=False)
        inp = torch.empty(n, dtype=torch.float32, device="cuda")
        tg = torch.empty_like(inp)
        op.make_pair(b, xk, xs, inp, tg)
        y = torch.empty_like(inp)
        net.forward(inp, y, dims, periodic=True)
        ay = torch.empty_like(inp)
        op.matvec(y, ay, hz.HZ_PREC_FP32)
        stage = float(torch.linalg.norm(inp - ay) / torch.linalg.norm(inp))
        plain = op.solve(b, x, krylov=hz.HZ_KRYLOV_FGMRES, raise_on_error=False)
        op.set_nn(net)
        learned = op.solve(b, x, krylov=hz.HZ_KRYLOV_FGMRES, precond=hz.HZ_PRE_TRI_NN, raise_on_error=False)
        bic = op.solve(b, x, raise_on_error=False)
        rows.append({"stage_residual_ratio": stage, "plain": plain, "learned": learned, "bicgstab": bic})
        op.close()

    def summary(key):
        r = [row[key] for row in rows]
        return {"solves_per_s": round(len(r) / sum(i["seconds"] for i in r), 4),
                "inner_iters": [i["inner_iters"] for i in r], "status": sorted({i["status"] for i in r}),
                "max_true_rel_residual": max(i["true_rel_residual"] for i in r),
                **({"fallbacks": [i["fallbacks"] for i in r]} if key == "learned" else {})}

    return {"dims": "x".join(map(str, dims)), "z_unit": z_unit, "train_systems": len(train_systems),
            "test_systems": len(test_systems), "train_steps": len(losses), "train_s": round(t_train, 1),
            "loss_first20_median": float(np.median(losses[:20])), "loss_last20_median": float(np.median(losses[-20:])),
            "stage_residual_ratio_held_out": [round(r["stage_residual_ratio"], 4) for r in rows],
            "fgmres_plain": summary("plain"), "fgmres_learned": summary("learned"), "bicgstab_plain": summary("bicgstab")}


def run_learned(args):
    """Learned stage on 640x480x70: train on fresh seeds, evaluate on held-out seeds."""
    import torch

    torch.cuda.set_device(0)
    train_sys = [(10000 + 2 * i, 10001 + 2 * i) for i in range(args.train_systems)]
    test_sys = [(20000 + 2 * i, 20001 + 2 * i) for i in range(args.test_systems)]
    out = learned_line((640, 480, 70), train_sys, test_sys, args.train_steps, args.z_unit)
    print(json.dumps({"workload": f"learned stage 640x480x70 z_unit={args.z_unit}", **out}), flush=True)


def run_nn_forward(args):
    """Inference of the learned stage's conv net alone on one 640x480x70 field (random-init weights)."""
    import torch

    import paper_1811_03852_gb300 as hz
    from paper_1811_03852_gb300 import learn

    torch.cuda.set_device(0)
    dims = tuple(args.dims) if args.dims else (640, 480, 70)
    n = dims[0] * dims[1] * dims[2]
    net = hz.Net(learn.init_params(1))
    x = torch.randn(n, device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    for _ in range(max(1, args.warmup)):
        net.forward(x, y, dims)
    ts = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.forward(x, y, dims)  # returns after its stream is idle
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.median(ts))
    flop = 2.0 * (432 + 6912 + 6912 + 432) * n  # multiply-adds of the four layers
    nbytes = 200.0 * n  # x 4 + h1 32 + (32 + 32) x 2 + h3 32 + y 4 bytes per point
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    print(json.dumps({"workload": f"conv-net forward {dims[0]}x{dims[1]}x{dims[2]} (4 layers, 16 channels, 3x3x3)",
                      "ms_per_forward": round(ms, 3), "TFLOPs": round(flop / (ms * 1e-3) / 1e12, 2),
                      "frac_of_bf16_peak": round(flop / (ms * 1e-3) / 1e12 / bf16, 4),
                      "GBps_algorithmic": round(nbytes / (ms * 1e-3) / 1e9, 1),
                      "frac_of_hbm": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 4),
                      "roofline_ms": round(max(flop / (bf16 * 1e12), nbytes / (hbm * 1e9)) * 1e3, 3),
                      "note": "wall clock per call (the call waits for its stream), median of steps"}), flush=True)


def run_fig1(args):
    """The paper's Sec. 4 / Fig. 1 comparison on a synthetic system: one FP32 and one FP64 BiCGStab
    (T^-1 preconditioner, restart 150, FP64 global sums, no refinement) run far past convergence,
    their recursive residuals per iteration and true FP64 residuals at checkpoints, next to the
    mixed solver's refinement loop."""
    import torch

    import gen
    import paper_1811_03852_gb300 as hz

    torch.cuda.set_device(0)
    dims = tuple(args.dims) if args.dims else (96, 72, 20)
    A, b = gen.make_system(*dims, 1, 2, z_unit=args.z_unit)
    op = hz.Operator(A)
    bd = torch.from_numpy(b.reshape(-1)).cuda()
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    nmax = 600
    curves, true_r = {}, {}
    for name, mode in (("fp32", hz.HZ_MODE_MIXED_IR), ("fp64", hz.HZ_MODE_FP64)):
        op.solve(bd, x, mode=mode, max_outer=1, inner_tol=1e-15, max_inner=nmax, record_history=1,
                 raise_on_error=False)
        curves[name] = [float(v) for v in op.history()]
        true_r[name] = {}
        for it in (10, 25, 50, 100, 150, 200, 300, 400, 600):
            info = op.solve(bd, x, mode=mode, max_outer=1, inner_tol=1e-15, max_inner=it, raise_on_error=False)
            true_r[name][it] = info["true_rel_residual"]

    def first_below(c, lvl):
        for i, v in enumerate(c):
            if v <= lvl:
                return i + 1
        return None

    levels = [1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8]
    gap = {f"{lvl:g}": {"fp32": first_below(curves["fp32"], lvl), "fp64": first_below(curves["fp64"], lvl)}
           for lvl in levels}
    ir = op.solve(bd, x, tol=1e-8)
    early = [abs(a - c) / c for a, c in zip(curves["fp32"][:5], curves["fp64"][:5])]
    print(json.dumps({
        "workload": f"paper Sec. 4 FP32 vs FP64 BiCGStab, {dims[0]}x{dims[1]}x{dims[2]} z_unit={args.z_unit} seeds 1/2",
        "iterations_to_reach_recursive_R": gap,
        "first5_rel_diff_fp32_vs_fp64": [round(v, 8) for v in early],
        "true_R_at_iteration": true_r,
        "min_true_R": {k: min(v.values()) for k, v in true_r.items()},
        "mixed_refinement": {"outer": ir["outer_iters"], "inner": ir["inner_iters"],
                             "true_R": ir["true_rel_residual"]},
        "recursive_R_every_10": {k: [c[i] for i in range(9, len(c), 10)] for k, c in curves.items()},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "nnfwd":
        run_nn_forward(args)
    elif args.workload == "fig1":
        run_fig1(args)
    elif args.workload == "table1":
        run_table1(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
