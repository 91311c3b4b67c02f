"""Benchmark: solved nodes/s to relative residual 1e-10 on the 3-D heterogeneous dielectric workload.

Workload (one "step" = one full solve from the lifted boundary values, inputs resident in HBM):
div(eps grad u) = f on the unit cube, 257^3 nodes, eps = 1 with 32 seeded spheres of eps = 80,
f = 8 seeded unit Gaussian charges (std 2h), u = 0 on the boundary, solved by the SGML cycle until
||r||_inf / ||f||_inf <= 1e-10.  The mixed form (FP32 cycle, FP64 outer step) gives `value`; the FP64
form is measured in the same run and reported beside it, with its roofline against both HBM and the
measured FP64 pipe.  Each form's error is reported against a tighter reference solution, the CPU
oracle is timed on full solves (one thread and all cores), the coefficient-pyramid setup is timed
on its own, and the other workloads of the benchmark set get secondary lines in `configs`:
2-D Poisson 129^2 to 1e-12, the 3 x 513^3 trefoil vector Poisson, the batch of 256 uneven 2-D
Helmholtz problems, and the 16 x 129^3 adjoint (forward + backward).  With --gpus N > 1 (torchrun,
one rank per GPU) every rank solves its own seeded instance: independent replicas, weak scaling.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead (host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solved nodes/s to rel. residual 1e-10 (mixed vs FP64 form), % of HBM roofline"
TOL = 1e-10
ACC_TOL = 5e-12  # residual tolerance at which the 257^3 solutions are within 1e-10 (relative L2) of the reference
# Algorithmic HBM bytes per fine node per cycle of the schedule (3-D, heterogeneous eps): one DRAM
# pass per phase, n_r = 2, zig-zag, 8 level-0 sweeps (outer step 24 + 2b + 8, level-0 sweeps
# 8 (3b + b), coarse levels (18b + 6b) / 7, b = bytes of the cycle precision).
BYTES_PER_NODE_CYCLE = {"mixed": 182.0, "fp64": 331.0}
# Algorithmic bytes per node per cycle of the other workloads (same count; 2-D / 3-D constant
# coefficients: no sigma arrays).
BYTES_2D_CONST = {"mixed": 152.0, "fp64": 280.0}
BYTES_3D_CONST = {"mixed": 138.0, "fp64": 253.0}
# FP64 instructions per node per cycle of the FP64 form on the 3-D heterogeneous workload at 257^3,
# counted from the kernels' arithmetic (n_r = 2, zig-zag; ncu's DADD + DFMA + DMUL counts of the
# two dominant kernels agree: 87.7 per node for the residual, 28.2 for a level-0 sweep at 129^3,
# where the sweep's short z-runs add plane sums of 2 halo planes per ~14 planes):
#   8 level-0 sweeps x 25.7 (sigma e once per halo cell 1.3, pair / face / corner sums 10, rolled z
#   terms 10, Jacobi update 4, halo planes of ~108-plane runs 0.4), the solution update 1, the FP64
#   residual 87.7 (27 sigma-weighted differences 78, sums, cast, norms), coarse-level sweeps 26.8
#   (6 per level and cycle, on short runs), restrictions 5.6, interpolations 11.
FP64_INSTR_PER_NODE_CYCLE = 338.0
KERNEL_SOURCES = ["paper_1703_07206_gb300/csrc/sgml_kernels.cu", "paper_1703_07206_gb300/csrc/sgml_internal.cuh"]


def workload_name(n):
    N = 2 ** n + 1
    return (f"3-D heterogeneous dielectric div(eps grad u)=f, {N}^3 nodes, eps 1 / 80 in 32 seeded spheres, "
            f"8 Gaussian charges (std 2h), Dirichlet 0, solve to rel. residual 1e-10")


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_traffic():
    """DRAM bytes per node per cycle of the cycle kernel from the committed ncu summary, if the
    kernel sources are unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return {}
    if d.get("kernel_hash") != kernel_hash():
        return {}
    return d.get("bytes_per_node_cycle", {})


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, device):
    """The largest value of x over the ranks of the initialised process group (x itself alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Seed of the workload replica a rank solves (replicas only: no data is exchanged)."""
    return 2000 + rank


def whole_job_rate(world, nodes_per_replica, ms_per_step):
    """Solved nodes per second of all replicas: every rank solves its own replica per step; the step
    time is the slowest rank's."""
    return world * nodes_per_replica / (ms_per_step / 1e3)


# ------------------------------------------------------------------------------------------------
# CPU oracle (the cpu_baseline leg and the reference arm): measured full solves, never tuned
# ------------------------------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_solve(n_sample, threads, tol=TOL, max_cycles=1000):
    """One full FP64 oracle solve of the n_sample instance of the workload recipe to `tol` on
    `threads` host threads.  Returns (seconds, cycles, solution, threads used)."""
    from oracle import oracle
    from oracle.oracle import Problem
    from paper_1703_07206_gb300 import inputs
    used = oracle.set_threads(threads)
    d = inputs.dielectric_spheres_3d(n=n_sample, seed=2000)
    p = Problem(3, n_sample, sigma=d["sigma"])
    t0 = time.perf_counter()
    u, cycles, _ = p.solve(d["f"], tol=tol, max_cycles=max_cycles)
    dt = time.perf_counter() - t0
    return dt, cycles, u, used


def run_reference(args):
    """The oracle as it stands, on the machine's host cores: every step one full solve of the 33^3
    instance of the workload recipe to the tolerance (a bounded sample of the 257^3 workload: same
    recipe, 1/512 of its nodes, ~3/5 of its cycles)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    n_s = args.ref_n
    M_s = (2 ** n_s + 1) ** 3
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_solve(n_s, cores)
    per, cycles, used = [], 0, cores
    for _ in range(args.steps):
        dt, cycles, _, used = oracle_solve(n_s, cores)
        per.append(dt)
    ms = float(np.mean(per)) * 1e3
    value = M_s / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args.n), "form": "fp64 CPU oracle"},
            "cpu_baseline": {"value": value, "unit": "nodes/s", "cores": used, "kind": "oracle",
                             "sample": f"each step one full solve of the {2 ** n_s + 1}^3 instance of the recipe "
                                       f"({M_s} nodes) to rel. residual {TOL:g}: {cycles} cycles, "
                                       f"{ms / 1e3:.1f} s on {used} threads"},
            "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(args):
    """The oracle timed on full solves to the tolerance: the 65^3 instance on every core of the
    affinity mask (the value) and the 33^3 instance on one thread.  Returns (cpu_baseline dict,
    the 65^3 oracle solution for the accuracy comparison)."""
    cores = host_cores()
    dt_all, cyc_all, u_all, used = oracle_solve(args.cpu_n, cores)
    M_all = (2 ** args.cpu_n + 1) ** 3
    dt_one, cyc_one, _, _ = oracle_solve(args.cpu_n - 1, 1)
    M_one = (2 ** (args.cpu_n - 1) + 1) ** 3
    from oracle import oracle
    oracle.set_threads(cores)
    cpu = {"value": M_all / dt_all, "unit": "nodes/s", "cores": used, "kind": "oracle",
           "sample": f"one full solve of the {2 ** args.cpu_n + 1}^3 instance of the recipe to rel. residual "
                     f"{TOL:g}: {cyc_all} cycles, {dt_all:.1f} s on {used} threads",
           "single_thread": {"value": M_one / dt_one, "unit": "nodes/s", "cores": 1,
                             "sample": f"one full solve of the {2 ** (args.cpu_n - 1) + 1}^3 instance to "
                                       f"{TOL:g}: {cyc_one} cycles, {dt_one:.1f} s"}}
    return cpu, u_all


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def make_grid(d, precision, stream):
    from paper_1703_07206_gb300 import sgml
    g = sgml.Grid(3, [d["n"]], precision=precision, stream=stream)
    g.set_params(max_cycles=args_global.max_cycles)
    g.set_launch(0, 1, 0, args_global.tile_x, args_global.slab_z)
    g.set_fusion(args_global.pair_levels)
    g.set_quad(args_global.quad_levels)
    return g


def time_solves(torch, g, stream, steps, warmup, tol=TOL):
    """Warm-up, then time `steps` solves with CUDA events on the grid's stream.  Returns (total ms,
    mean ms per solve, cycles (largest of the batch), relative residual (largest), launches)."""
    from paper_1703_07206_gb300 import sgml
    for _ in range(warmup):
        st, cyc, rel = g.solve_to_tol(tol)
        if st != sgml.OK:
            raise RuntimeError(f"solve failed: status {st}, cycles {cyc}, rel {rel}")
    launches0 = g.launch_count()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per = []
    e0.record(stream)
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, cyc, rel = g.solve_to_tol(tol)
        b.record(stream)
        per.append((a, b))
        if st != sgml.OK:
            raise RuntimeError(f"solve failed: status {st}")
    e1.record(stream)
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    kernel_ms = float(np.mean([a.elapsed_time(b) for a, b in per]))
    return total_ms, kernel_ms, int(np.max(cyc)), float(np.max(rel)), g.launch_count() - launches0


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def hbm_roofline(bytes_per_node_cycle, nodes, cycles, ms, peak, peak_kind, traffic=None):
    achieved = bytes_per_node_cycle * nodes * cycles / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": f"{peak_kind} HBM copy bandwidth",
            "algorithmic_bytes_per_node_cycle": bytes_per_node_cycle}


def run_gpu(args):
    import torch
    from paper_1703_07206_gb300 import build, inputs, sgml
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    stream = torch.cuda.Stream()
    dev = f"cuda:{local}"
    n = args.n
    N = 2 ** n + 1
    M = N ** 3
    d = inputs.dielectric_spheres_3d(n=n, seed=replica_seed(rank))
    f = np.ascontiguousarray(d["f"])
    sig = np.ascontiguousarray(d["sigma"])
    f_dev = torch.from_numpy(f).to(dev)
    s_dev = torch.from_numpy(sig).to(dev)
    results = {}
    forms = ["mixed", "fp64"] if args.form == "both" else [args.form]
    grids = {}
    setup_ms = {}
    for form in forms:
        prec = sgml.MIXED if form == "mixed" else sgml.FP64
        g = make_grid(d, prec, stream)
        g.set_bc(0, [sgml.DIRICHLET] * 6)
        g.set_source(0, f_dev)
        g.set_coeffs(0, s_dev)
        g.launch_info()  # work tables and the first pyramid (allocates the coefficient pools)
        # A0, the coefficient pyramid (restricted sigma, local steps per level), timed on its own
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_coeffs(0, s_dev)
        g.launch_info()  # rebuilds the pyramid and synchronises
        torch.cuda.synchronize()
        setup_ms[form] = (time.perf_counter() - t0) * 1e3
        grids[form] = g
    peak, peak_kind = load_peaks()
    traffic = load_traffic()
    fp64_rate, fp32_rate = sgml.measure_fma_rates(stream)
    for form in forms:
        g = grids[form]
        steps = args.steps if form == forms[0] else max(1, min(args.steps, args.fp64_steps))
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            total_ms, kernel_ms, cycles, rel, launches = time_solves(torch, g, stream, steps, args.warmup)
        total_ms = max_over_ranks(total_ms, dev)
        ms = total_ms / steps
        value = whole_job_rate(world, M, ms)
        tr = traffic.get(form)
        ctas, threads, smem = g.launch_info()
        results[form] = {"value": value, "ms_per_step": ms, "kernel_ms": kernel_ms, "cycles": cycles, "rel": rel,
                         "launches_per_step": launches / steps, "steps": steps, "clocks": clk.summary(),
                         "launch": {"ctas": ctas, "threads_per_cta": threads, "smem_bytes_per_cta": smem},
                         "roofline": hbm_roofline(BYTES_PER_NODE_CYCLE[form], M, cycles, kernel_ms, peak, peak_kind,
                                                  tr * M * cycles if tr is not None else None)}
        if form == "fp64":
            achieved = FP64_INSTR_PER_NODE_CYCLE * M * cycles / (kernel_ms / 1e3)
            results[form]["roofline_fp64_pipe"] = {
                "bound": "fp64", "achieved": achieved, "peak": fp64_rate, "unit": "FP64 instructions/s",
                "frac": achieved / fp64_rate, "instructions_per_node_cycle": FP64_INSTR_PER_NODE_CYCLE,
                "peak_kind": "measured FP64 FMA rate (sgml_measure_fma_rates, this run)"}
    # accuracy: each form at the benchmark tolerance against the FP64 form driven to 1e-13 (the
    # FP64 form equals the oracle cycle by cycle to 1e-12 in the parity tests)
    acc = {}
    u_form = {form: grids[form].get_solution(0) for form in forms}
    if "fp64" in grids:
        gf = grids["fp64"]
        gf.set_params(max_cycles=args.max_cycles + 200)
        st, cyc, rel = gf.solve_to_tol(1e-13)
        u_tight = gf.get_solution(0)
        acc = {"reference": f"FP64 form solved to rel. residual 1e-13 ({int(cyc[0])} cycles, status {st})",
               **{form: rel_l2(u_form[form], u_tight) for form in forms}}
        # the residual tolerance at which each form's solution is within 1e-10 of the reference
        # (the operator amplifies the relative residual ~14x in the relative L2 error here)
        matched = {}
        for form in forms:
            g = grids[form]
            g.set_params(max_cycles=args.max_cycles + 200)
            torch.cuda.synchronize()
            _, ms_m, cyc_m, rel_m, _ = time_solves(torch, g, stream, 1, 0, ACC_TOL)
            matched[form] = {"tol": ACC_TOL, "cycles": cyc_m, "rel_residual": rel_m, "ms_per_solve": ms_m,
                             "solved_nodes_per_s": M / (ms_m / 1e3), "rel_l2": rel_l2(g.get_solution(0), u_tight)}
            g.set_params(max_cycles=args.max_cycles)
        acc["at_matched_tolerance"] = matched
    # end to end through the C ABI with host buffers (pinned), copies and setup inside
    e2e = None
    if not args.no_e2e:
        form = forms[0]
        g = grids[form]
        f_h = torch.from_numpy(f).pin_memory().numpy()
        s_h = torch.from_numpy(sig).pin_memory().numpy()
        u_h = torch.empty(M, dtype=torch.float64).pin_memory().numpy().reshape(N, N, N)
        for _ in range(1):
            g.set_coeffs(0, s_h)
            g.set_source(0, f_h)
            g.solve_to_tol(TOL)
            g.get_solution(0, u_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g.set_coeffs(0, s_h)
            g.set_source(0, f_h)
            st, cyc, rel = g.solve_to_tol(TOL)
            g.get_solution(0, u_h)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        el = max_over_ranks(el, dev)
        e2e = {"value": world * M * args.steps / el, "unit": "nodes/s", "h2d_bytes_per_step": 2 * M * 8,
               "d2h_bytes_per_step": M * 8}
    for g in grids.values():
        g.close()
    del grids
    cpu, configs = None, None
    if rank == 0 and world == 1:
        if not args.no_cpu_baseline:
            cpu, u_orc = cpu_baseline_leg(args)
            acc["at_65cubed_vs_oracle"] = small_accuracy(args, stream, u_orc)
        if not args.no_configs:
            torch.cuda.empty_cache()
            configs = run_configs(args, stream, local, peak, peak_kind)
    if rank != 0:
        return
    main = results[forms[0]]
    line = {"metric": METRIC, "value": main["value"], "unit": "nodes/s", "n_gpus": world, "steps": main["steps"],
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if forms[0] == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": workload_name(n), "form": forms[0], "nodes": M, "cycles": main["cycles"],
                       "rel_residual": main["rel"], "l2": "inputs larger than L2 (working set > 1 GB per replica)",
                       "tile": f"{args.tile_x}x{512 // args.tile_x}",
                       "fused_pair_levels": args.pair_levels, "four_row_levels": args.quad_levels,
                       "launch": main["launch"],
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": main["roofline"], "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(round(main["launches_per_step"] * main["steps"])), "clocks": main["clocks"],
            "setup_ms": setup_ms, "rel_l2_vs_reference": acc,
            "fma_rates": {"fp64_per_s": fp64_rate, "fp32_per_s": fp32_rate}}
    if "fp64" in results and forms[0] != "fp64":
        fp = results["fp64"]
        line["fp64_form"] = {"value": fp["value"], "ms_per_step": fp["ms_per_step"], "cycles": fp["cycles"],
                             "rel_residual": fp["rel"], "steps": fp["steps"], "roofline": fp["roofline"],
                             "roofline_fp64_pipe": fp["roofline_fp64_pipe"], "clocks": fp["clocks"]}
        line["mixed_over_fp64"] = main["value"] / fp["value"]
        line["mixed_vs_fp64_rel_l2"] = rel_l2(u_form["mixed"], u_form["fp64"])
    if configs is not None:
        line["configs"] = configs
    print(json.dumps(line), flush=True)


def small_accuracy(args, stream, u_orc):
    """Both forms on the 65^3 instance of the recipe at the benchmark tolerance against the oracle's
    own solve at that tolerance, and against the FP64 form driven to 1e-13."""
    from paper_1703_07206_gb300 import inputs, sgml
    n = args.cpu_n
    d = inputs.dielectric_spheres_3d(n=n, seed=2000)
    out = {}
    u = {}
    for form, prec in (("mixed", sgml.MIXED), ("fp64", sgml.FP64)):
        g = sgml.Grid(3, [n], precision=prec, stream=stream)
        g.set_params(max_cycles=args.max_cycles + 200)
        sgml.problem_into_grid(g, 0, d)
        st, cyc, rel = g.solve_to_tol(TOL)
        u[form] = g.get_solution(0)
        if form == "fp64":
            st2, cyc2, _ = g.solve_to_tol(1e-13)
            u["tight"] = g.get_solution(0)
        g.close()
    for form in ("mixed", "fp64"):
        out[form] = rel_l2(u[form], u_orc)
        out[form + "_vs_fp64_1e-13"] = rel_l2(u[form], u["tight"])
    out["oracle_vs_fp64_1e-13"] = rel_l2(u_orc, u["tight"])
    out["reference"] = (f"the oracle's solution of the {2 ** n + 1}^3 instance at rel. residual {TOL:g} (and the "
                        f"GPU FP64 form at 1e-13)")
    return out


def run_configs(args, stream, local, peak, peak_kind):
    """Secondary lines: the other workloads of the benchmark set, each timed on its own (CUDA events
    on the grid's stream, inputs resident on the device, warm-up solves first)."""
    import torch
    from paper_1703_07206_gb300 import inputs, sgml
    dev = f"cuda:{local}"
    out = {}
    steps = max(1, min(args.steps, args.config_steps))

    def solve_line(probs, prec, tol, bytes_node_cycle, label, n_steps=steps, warmup=1):
        dim = probs[0]["dim"]
        g = sgml.Grid(dim, [q["n"] for q in probs], precision=prec, stream=stream)
        g.set_params(max_cycles=args.max_cycles)
        for b, q in enumerate(probs):
            g.set_bc(b, q["faces"], q["values"])
            g.set_coeffs(b, torch.from_numpy(np.ascontiguousarray(q["sigma"])).to(dev) if q["sigma"] is not None
                         else None, None, q.get("a_scalar", 0.0))
            g.set_source(b, torch.from_numpy(np.ascontiguousarray(q["f"])).to(dev))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.launch_info()
        torch.cuda.synchronize()
        setup = (time.perf_counter() - t0) * 1e3
        nodes = sum(int(np.prod(q["f"].shape)) for q in probs)
        with ClockSampler(local) as clk:
            total_ms, kernel_ms, cycles, rel, launches = time_solves(torch, g, stream, n_steps, warmup, tol)
        g.close()
        return {"workload": label, "form": "mixed" if prec == sgml.MIXED else "fp64", "nodes": nodes,
                "tol": tol, "cycles": cycles, "rel_residual": rel, "ms_per_solve": kernel_ms,
                "solved_nodes_per_s": nodes / (kernel_ms / 1e3), "setup_ms": setup, "steps": n_steps,
                "launches_per_solve": launches / n_steps,
                "roofline": hbm_roofline(bytes_node_cycle[ "mixed" if prec == sgml.MIXED else "fp64"], nodes, cycles,
                                         kernel_ms, peak, peak_kind),
                "clocks": clk.summary()}

    # 2-D Poisson 129^2, sin(pi x) sin(pi y), Dirichlet 0, tolerance 1e-12 (the plain method)
    p1 = [inputs.poisson_sine_2d(7)]
    out["poisson_129sq"] = {f: solve_line(p1, prec, 1e-12, BYTES_2D_CONST,
                                          "2-D Poisson 129^2, -Lap u = 2 pi^2 sin(pi x) sin(pi y), Dirichlet 0",
                                          n_steps=max(steps, 10), warmup=3)
                            for f, prec in (("fp64", sgml.FP64), ("mixed", sgml.MIXED))}
    # 3 x 513^3 trefoil vector Poisson (Sec. 3.3), both forms, one batch of three components
    p3 = inputs.trefoil_vorticity_3d(n=9)
    out["trefoil_3x513cubed"] = {f: solve_line(p3, prec, TOL, BYTES_3D_CONST,
                                               "3-D vector Poisson -Lap psi_i = omega_i, 3 x 513^3, trefoil tube")
                                 for f, prec in (("mixed", sgml.MIXED), ("fp64", sgml.FP64))}
    del p3
    torch.cuda.empty_cache()
    # 256 uneven 2-D Helmholtz problems in one persistent launch per solve (mixed form)
    p4 = inputs.helmholtz_batch_2d()
    out["helmholtz_batch_256"] = solve_line(p4, sgml.MIXED, TOL, BYTES_2D_CONST,
                                            "256 x 2-D -Lap u + k^2 u = f, sides 65..1025, D/N sides, one launch")
    del p4
    # 16 x 129^3 adjoint: forward solve + adjoint solve + gradient (autograd), mixed form (FP64 outer step)
    out["adjoint_16x129cubed"] = adjoint_line(args, stream, local, peak, peak_kind, steps)
    return out


def adjoint_line(args, stream, local, peak, peak_kind, steps):
    import torch
    from paper_1703_07206_gb300 import inputs, sgml
    from paper_1703_07206_gb300.autograd import SGMLSolve
    dev = f"cuda:{local}"
    probs = inputs.lognormal_dielectric_batch_3d(count=16, n=7, seed=5000)
    n = probs[0]["n"]
    M = (2 ** n + 1) ** 3
    # targets: solutions with the perturbed eps (one batched solve, outside the timed region)
    gt = sgml.Grid(3, [n] * 16, precision=sgml.MIXED, stream=stream)
    gt.set_params(max_cycles=args.max_cycles)
    gt.set_coeffs(-1, torch.from_numpy(np.stack([q["eps_target"] for q in probs])).to(dev))
    f_all = torch.from_numpy(np.stack([q["f"] for q in probs])).to(dev)
    gt.set_source(-1, f_all)
    st, cyc_t, _ = gt.solve_to_tol(TOL)
    ut = torch.empty_like(f_all)
    for b in range(16):
        gt.get_solution(b, ut[b])
    gt.close()
    grid = sgml.Grid(3, [n] * 16, precision=sgml.MIXED, stream=stream)
    grid.set_params(max_cycles=args.max_cycles)
    sig0 = torch.from_numpy(np.stack([q["sigma"] for q in probs])).to(dev)

    def step():
        f = f_all.clone().requires_grad_(True)
        s = sig0.clone().requires_grad_(True)
        u = SGMLSolve.apply(f, s, grid, TOL, True)
        J = 0.5 * ((u - ut) ** 2).sum()
        J.backward()
        return f.grad, s.grad

    with torch.cuda.stream(stream):
        step()
        torch.cuda.synchronize()
        launches0 = grid.launch_count()
        with ClockSampler(local) as clk:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                step()
            b.record(stream)
            torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
    launches = (grid.launch_count() - launches0) / steps
    cyc_adj = max(grid.get_stats(b)[0] for b in range(16))
    grid.close()
    nodes = 16 * M
    return {"workload": "16 x 3-D dielectric 129^3, log-normal eps, J = 1/2 ||u - u_t||^2: forward solve, "
                        "adjoint solve, dJ/deps and dJ/df (autograd)",
            "form": "mixed (FP32 cycle, FP64 outer step)", "nodes": nodes, "tol": TOL,
            "ms_per_forward_backward": ms, "nodes_per_s_forward_backward": nodes / (ms / 1e3),
            "launches_per_step": launches, "adjoint_solve_cycles": int(cyc_adj),
            "target_solve_cycles": int(np.max(cyc_t)), "steps": steps,
            "clocks": clk.summary()}


def schedule_labels(g):
    """Labels of the cycle's phases, from the library's own phase table (restriction passes, then
    the zig-zag visits of Algorithm 3 with their transitions; fused sweep pairs count as one)."""
    names = {0: lambda l: f"restrict ->{l}", 1: lambda l: f"sweep L{l}", 2: lambda l: f"prolong {l + 1}->{l}",
             3: lambda l: f"inject {l - 1}->{l}", 4: lambda l: "mean rows", 5: lambda l: "mean reduce",
             6: lambda l: "mean apply"}
    return [names[op](level) for op, level, _, _ in g.get_phases()]


def run_trace(args, g, n):
    """Per-phase time inside the persistent kernel, averaged over the traced cycles."""
    g.set_trace(args.trace_cycles)
    g.set_params(max_cycles=args.max_cycles)
    g.solve_to_tol(TOL)
    t = g.get_trace()
    lab = ["-", "residual", "check"] + schedule_labels(g)
    mean = t[1:].mean(axis=0) if len(t) > 1 else t.mean(axis=0)
    groups = {}
    for name, v in zip(lab, mean):
        key = name.split(" ")[0] + (" L0" if name.endswith("L0") or name.endswith("->0") else
                                    (" L1" if name.endswith("L1") or name.endswith("->1") else ""))
        groups[key] = groups.get(key, 0.0) + v
    rows = [{"phase": k, "us_per_cycle": round(v, 1)} for k, v in sorted(groups.items(), key=lambda kv: -kv[1])]
    print(json.dumps({"trace": True, "n": n, "cycles_traced": int(len(t)), "us_per_cycle_total": round(float(mean.sum()), 1),
                      "groups": rows, "per_phase_us": [round(float(x), 1) for x in mean]}))


def run_ncu_case(args):
    """Small case for ncu: one run_cycle launch of `--ncu-cycles` cycles on the workload."""
    import torch
    from paper_1703_07206_gb300 import build, inputs, sgml
    build.build()
    torch.cuda.set_device(0)
    if args.ncu_workload == "curl":  # v = curl psi (Eq. 14) of a random (2^n + 1)^3 potential: two launches
        N = 2 ** args.n + 1
        psi = torch.from_numpy(np.random.default_rng(7).standard_normal((3, N, N, N))).cuda()
        for _ in range(2):
            v = sgml.curl(psi)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": True, "workload": "curl", "n": args.n, "checksum": float(v.abs().sum())}))
        return
    if args.ncu_workload == "batch":  # the 256 uneven 2-D Helmholtz problems
        probs = inputs.helmholtz_batch_2d()
    else:
        probs = [inputs.dielectric_spheres_3d(n=args.n, seed=2000)]
    prec = sgml.MIXED if args.form in ("mixed", "both") else sgml.FP64
    g = sgml.Grid(probs[0]["dim"], [q["n"] for q in probs], precision=prec)
    g.set_params(max_cycles=args.max_cycles)
    g.set_launch(0, 1, 1 if args.phased else 0, args.tile_x, args.slab_z)
    g.set_fusion(args.pair_levels)
    g.set_quad(args.quad_levels)
    for b, q in enumerate(probs):
        sgml.problem_into_grid(g, b, q)
    g.run_cycle(1)  # warm-up launch (and setup)
    if args.trace:
        run_trace(args, g, args.n)
        g.close()
        return
    if args.ncu_solve:
        g.set_params(max_cycles=args.max_cycles)
        g.solve_to_tol(TOL)
    else:
        g.run_cycle(args.ncu_cycles)
    torch.cuda.synchronize()
    c, rel, st = g.get_stats(0)
    print(json.dumps({"ncu_case": True, "workload": args.ncu_workload, "n": args.n, "form": args.form, "cycles": c,
                      "rel": rel, "status": st, "phases": len(g.get_phases())}))
    g.close()


args_global = None


def run_next_rows(args):
    """Timings of the widened rows (not the headline): the capacitor of Sec. 3.4, the all-Neumann
    Helmholtz problem of Eq. 10, the per-level diagnostic residual, and the post-processing
    kernels of Secs. 3.2-3.3 (curl, streamlines, grid motion).  Inputs are synthetic and resident on
    the device; each figure is the mean of `--steps` calls after `--warmup` untimed ones, timed
    with CUDA events on the current stream.  Prints one JSON line."""
    import torch
    from paper_1703_07206_gb300 import inputs, sgml
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    peak, peak_kind = load_peaks()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps, out

    def solve_row(probs, tol, diag=0):
        dim = probs[0]["dim"]
        g = sgml.Grid(dim, [d["n"] for d in probs], precision=sgml.MIXED, stream=stream.cuda_stream)
        g.set_params(max_cycles=args.max_cycles)
        for b, d in enumerate(probs):
            sgml.problem_into_grid(g, b, d)
        if diag:
            g.set_diagnostics(diag)

        def one():
            st, cyc, rel = g.solve_to_tol(tol)
            if st != sgml.OK:
                raise RuntimeError(f"solve failed: status {st}")
            return int(np.max(cyc)), float(np.max(rel))

        ms, (cyc, rel) = timed(one)
        nodes = sum(int(np.prod(d["f"].shape)) for d in probs)
        return {"nodes": nodes, "cycles": cyc, "rel_residual": rel, "ms_per_solve": round(ms, 3),
                "solved_nodes_per_s": nodes / (ms * 1e-3)}

    out = {"metric": "next-row timings", "data": "synthetic", "steps": args.steps, "warmup": args.warmup}
    out["capacitor_129cubed"] = solve_row([inputs.capacitor_3d(n=7, sign=+1.0)], TOL)
    out["eq10_neumann_helmholtz_1025sq"] = solve_row([inputs.neumann_helmholtz_2d(n=10, a=0.1)], TOL)
    out["eq10_neumann_helmholtz_65sq"] = solve_row([inputs.neumann_helmholtz_2d(n=6, a=0.1)], TOL)
    d129 = inputs.dielectric_spheres_3d(n=7)
    base = solve_row([d129], TOL)
    diag = solve_row([d129], TOL, diag=args.max_cycles + 1)
    out["diagnostics_129cubed"] = {"ms_off": base["ms_per_solve"], "ms_on": diag["ms_per_solve"],
                                   "overhead": diag["ms_per_solve"] / base["ms_per_solve"] - 1.0}
    out["trefoil_3x129cubed"] = solve_row(inputs.trefoil_vorticity_3d(n=7), TOL)
    # post-processing kernels on synthetic fields
    rng = np.random.default_rng(7)
    N = 257
    psi = torch.from_numpy(rng.standard_normal((3, N, N, N))).to(dev)
    ms, _ = timed(lambda: sgml.curl(psi, stream=stream))
    bytes_per_call = 48.0 * N ** 3  # three potentials read, three velocity components written
    out["curl_257cubed"] = {"ms": round(ms, 3), "achieved_gbs": bytes_per_call / (ms * 1e-3) / 1e9,
                            "peak_gbs": peak, "peak_kind": peak_kind,
                            "frac": bytes_per_call / (ms * 1e-3) / 1e9 / peak, "bytes_per_node": 48}
    del psi
    Nv = 129
    v = torch.from_numpy(0.2 * rng.standard_normal((3, Nv, Nv, Nv))).to(dev)
    seeds = torch.from_numpy(rng.uniform(0.2, 0.8, size=(4096, 3))).to(dev)
    ms, _ = timed(lambda: sgml.streamlines(v, seeds, 1e-3, 1000, stream=stream))
    out["streamlines_129cubed"] = {"ms": round(ms, 3), "seeds": 4096, "steps": 1000,
                                   "rk4_steps_per_s": 4096 * 1000 / (ms * 1e-3)}
    del v, seeds
    for name, dim, n, steps in (("grid_motion_1025sq", 2, 10, 100), ("grid_motion_129cubed", 3, 7, 20)):
        M = (2 ** n + 1) ** dim
        shape = (2 ** n + 1,) * dim
        u = torch.from_numpy(0.05 * rng.standard_normal(shape)).to(dev)
        f = torch.from_numpy(0.5 + rng.uniform(size=shape)).to(dev)
        ms, _ = timed(lambda: sgml.grid_motion(u, f, steps, stream=stream))
        out[name] = {"ms": round(ms, 3), "nodes": M, "euler_steps": steps, "node_steps_per_s": M * steps / (ms * 1e-3)}
    print(json.dumps(out))


def main():
    global args_global
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--form", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--n", type=int, default=8, help="N = 2^n + 1 nodes per side (8: 257^3)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--max-cycles", type=int, default=400)
    ap.add_argument("--cpu-n", type=int, default=6, help="cpu_baseline: oracle solve at 2^n + 1 (all cores) and at 2^(n-1) + 1 (one thread)")
    ap.add_argument("--ref-n", type=int, default=5, help="reference arm: oracle solve of the 2^n + 1 instance per step")
    ap.add_argument("--no-configs", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--config-steps", type=int, default=2, help="timed solves per secondary workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ncu-case", action="store_true")
    ap.add_argument("--ncu-cycles", type=int, default=2)
    ap.add_argument("--ncu-solve", action="store_true", help="ncu case: one full solve instead of --ncu-cycles")
    ap.add_argument("--ncu-workload", default="dielectric", choices=["dielectric", "batch", "curl"],
                    help="ncu case: the 3-D dielectric workload (--n), the 256-problem 2-D Helmholtz batch, "
                         "or two curl launches on a random (2^n + 1)^3 potential")
    ap.add_argument("--phased", action="store_true")
    ap.add_argument("--tile-x", type=int, default=64, choices=[32, 64], help="column tiles 32 x 16 or 64 x 8")
    ap.add_argument("--slab-z", type=int, default=None,
                    help="z-slab height of the work partition (0: contiguous runs; default: the library's)")
    ap.add_argument("--pair-levels", type=int, default=0, help="levels whose sweeps run in fused pairs (0: none)")
    ap.add_argument("--quad-levels", type=int, default=0, help="levels whose sweeps run four rows per thread")
    ap.add_argument("--trace", action="store_true", help="with --ncu-case: per-phase times from the kernel's trace")
    ap.add_argument("--trace-cycles", type=int, default=64)
    ap.add_argument("--next-rows", action="store_true",
                    help="time the widened rows (capacitor, Eq. 10, diagnostics, curl, streamlines, grid motion)")
    args = ap.parse_args()
    args_global = args
    if args.warmup < 3 and args.impl == "gb300" and not args.ncu_case:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.ncu_case:
        run_ncu_case(args)
    elif args.next_rows:
        run_next_rows(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
