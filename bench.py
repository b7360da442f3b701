#!/usr/bin/env python
"""Benchmark: pAIR source iteration for upwind-DG S_N transport on one GB300.

Metric: DOF*directions solved per second per source iteration, every
direction's AIR solve reaching a relative FP64 residual of 1e-8.

Workload (default): unit cube, 32^3 hexahedra, trilinear Q1 upwind DG
(262,144 DOFs per direction), level-symmetric S4 (24 directions) in one
batch, sigma_t ~ U[0.5, 2] per element (SplitMix64 seed 1), sigma_s = 0.8
sigma_t, q = 1, vacuum boundaries.  Synthetic, seeded inputs.

One timed step = one complete source-iteration solve from phi = 0, every row of
the path in every step: DG assembly and block scaling of all directions, AIR
setup of every hierarchy (strength, PMIS, one-point P, lAIR, Galerkin RAP),
then source iterations to ||phi^{n+1} - phi^n|| <= 1e-8 ||phi^{n+1}||, each
iteration building the right-hand sides, solving every direction from psi = 0
to a 1e-8 relative FP64 residual (FP32 V-cycles under FP64 iterative
refinement) and forming the scalar-flux quadrature sum.  The value is
DOF*directions*iterations / step time, so the setup is amortised over the
solve's iterations; the mode that rebuilds every hierarchy for every iteration
(the paper's memory mode) is measured beside it.  Each step moves many GB, far
more than the 129 MB L2, so no explicit flush is needed between steps.

--impl reference times the CPU oracle (the plain C implementation the tests
check against) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF*directions solved/s per source iteration (AIR to 1e-8 FP64 residual)"
UNIT = "DOF*dir/s"
WORKLOADS = {
    "hex32_s4": "unit cube 32^3 hex Q1 upwind DG (262,144 DOFs/dir), S4 level-symmetric (24 dirs) in one batch, "
                "sigma_t~U[0.5,2] seed 1, sigma_s=0.8 sigma_t, q=1, vacuum",
    "hex8_s2": "unit cube 8^3 hex Q1 upwind DG (4,096 DOFs/dir), S2 (8 dirs), sigma_t=1, sigma_s=0.5, q=1, vacuum",
    "hex24_s4_adj": "unit cube 24^3 hex Q1 (110,592 DOFs/dir), S4 (24 dirs), sigma_t~U[0.5,2], sigma_s=0.7 sigma_t, "
                    "q=1 in central 8^3",
    "hex64_s8": "unit cube 64^3 hex Q1 (2,097,152 DOFs/dir), S8 (80 dirs) in HBM-admitted batches, "
                "sigma_t~logU[0.1,100], sigma_s=0.95 sigma_t, q=1",
    "tet40_s8": "unit cube 40^3 cubes x 6 Kuhn tets jittered 0.2h (1,536,000 P1 DOFs/dir), S8 (80 dirs), sigma_t "
                "checkerboard {1,100} over 4^3 regions, sigma_s=0.9 sigma_t, q=1 where sigma_t=1, distance-2 AIR",
    "tet16_s8": "the tet40_s8 construction on 16^3 cubes x 6 tets (98,304 P1 DOFs/dir), S8 (80 dirs), distance-2 "
                "AIR (a small case of the same setup kernels, for profiling)",
}
# workloads whose scattering ratio needs hundreds of SI iterations: a step runs a
# fixed number of iterations instead of the whole solve
FIXED_SI = {"hex64_s8": 2, "tet40_s8": 2, "tet16_s8": 2}
DISTANCE = {"tet40_s8": 2, "tet16_s8": 2}
# coarsest level (max_coarse rows, Jacobi sweeps) of the large workloads: the first
# level with at most 40,000 rows per direction, 3 sweeps (V-cycle counts unchanged
# against the library's 100 rows / 20 sweeps, measured with the oracle); the small
# meshes keep the library's, which a 40,000-row bound would reduce to one level
COARSEST = {"hex32_s4": (40000, 3), "hex64_s8": (40000, 3), "tet40_s8": (40000, 3)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over all ranks (the job's time is the slowest rank's)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def oracle_direction_times(prob, m, air_kw):
    """Oracle times for one direction: assembly + AIR setup, and one solve of
    the first SI iteration's right-hand side to 1e-8 (seconds)."""
    import numpy as np
    from oracle import oracle as O
    tet = hasattr(prob, "tets")
    t0 = time.perf_counter()
    if tet:
        r, c, v = O.tet_assemble(prob, prob.omega[m])
    else:
        r, c, v = O.hex_assemble(prob.n, prob.omega[m], prob.sigma_t)
    H = O.Hierarchy(r, c, v, O.default_params(**air_kw))
    t1 = time.perf_counter()
    src = np.repeat(prob.q, 4 if tet else 8) / (4 * np.pi)
    b = O.tet_rhs(prob, prob.omega[m], src) if tet else O.hex_rhs(prob.n, prob.omega[m], prob.sigma_t, src)
    H.solve(b, tol=1e-8, maxit=500)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def cpu_baseline_oracle(prob, si_iters, air_kw, max_seconds: float = 20.0):
    """The CPU oracle, as it stands, single-threaded on the host, on a bounded
    sample of the workload's directions; per-SI-iteration throughput with the
    setup amortised over the same number of SI iterations as the GPU solve."""
    from oracle import oracle as O
    O.build()
    done, ts, tv = 0, 0.0, 0.0
    while done < prob.M:
        a, b = oracle_direction_times(prob, done, air_kw)
        ts, tv, done = ts + a, tv + b, done + 1
        if ts + tv >= max_seconds:
            break
    per_dir_iter = ts / done / max(si_iters, 1) + tv / done
    out = {"value": prob.N / per_dir_iter, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{done} of {prob.M} directions: oracle assembly + AIR setup ({ts:.1f} s) and one 1e-8 solve "
                     f"each ({tv:.1f} s), setup amortised over {si_iters} SI iterations, single-threaded"}
    out["all_cores"] = cpu_oracle_all_cores(prob, si_iters, air_kw)
    out["oracle_sweep"] = cpu_oracle_sweep(prob)
    return out


def cpu_oracle_all_cores(prob, si_iters, air_kw):
    """The same oracle work with the directions spread over every host core (the
    directions are independent; the oracle's C calls release the GIL, so plain
    threads run them in parallel): one direction per core, wall time measured."""
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 1
    nd = min(prob.M, cores)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        res = list(ex.map(lambda m: oracle_direction_times(prob, m, air_kw), range(nd)))
    wall = time.perf_counter() - t0
    ts = sum(a for a, _ in res)
    tv = sum(b for _, b in res)
    # the wall time covers nd directions' setup + one solve each; amortise the setup
    # share of it over the SI iterations as in the single-thread figure
    share_setup = ts / (ts + tv)
    per_iter_wall = wall * (share_setup / max(si_iters, 1) + (1 - share_setup))
    return {"value": prob.N * nd / per_iter_wall, "unit": UNIT, "cores": cores,
            "sample": f"{nd} directions, one per thread, wall {wall:.1f} s (sum of per-direction times "
                      f"{ts + tv:.1f} s)"}


def cpu_oracle_sweep(prob):
    """The oracle's exact sweep (topological block forward substitution) per
    direction, single-threaded: the solver pAIR replaces (DOF*dir/s per SI iteration)."""
    import numpy as np
    from oracle import oracle as O
    tet = hasattr(prob, "tets")
    t = 0.0
    nd = min(prob.M, 4)
    for m in range(nd):
        if tet:
            r, c, v = O.tet_assemble(prob, prob.omega[m])
            src = np.repeat(prob.q, 4) / (4 * np.pi)
            b = O.tet_rhs(prob, prob.omega[m], src)
        else:
            r, c, v = O.hex_assemble(prob.n, prob.omega[m], prob.sigma_t)
            src = np.repeat(prob.q, 8) / (4 * np.pi)
            b = O.hex_rhs(prob.n, prob.omega[m], prob.sigma_t, src)
        t0 = time.perf_counter()
        if tet:
            O.sweep_scc(r, c, v, b, 4)
        else:
            O.sweep(r, c, v, b)
        t += time.perf_counter() - t0
    return {"value": prob.N * nd / t, "unit": UNIT, "cores": 1,
            "sample": f"exact sweep of {nd} directions (assembly excluded), single-threaded"}


def bench_config(args, world):
    """The workload configuration both arms print (the reference arm's own step is
    described in its cpu_baseline.sample)."""
    fixed = args.si_fixed if args.si_fixed is not None else FIXED_SI.get(args.config, 0)
    return {"workload": args.config + ": " + WORKLOADS[args.config],
            "step": ("one complete SI solve from phi=0 (assembly + AIR setup + SI iterations to 1e-8, every "
                     "direction solved from psi=0 to 1e-8 relative FP64 residual each iteration); value = "
                     "DOF*dir*iterations/step time") if not fixed else
                    (f"assembly + AIR setup + {fixed} SI iterations from phi=0 (every direction solved from "
                     "psi=0 to 1e-8 relative FP64 residual each iteration); value = DOF*dir*iterations/step "
                     "time (setup included); solve_only_value excludes the setup"),
            "air": {"R": "nAIR degree 1" if args.nair else f"lAIR distance {args.distance}",
                    "theta": args.theta, "eps_R": 0.01, "phi_R": args.phi_R, "phi_A": args.phi_A,
                    "relax": "F-F-C Jacobi", "coarsening": "PMIS", "max_coarse": coarsest(args)[0],
                    "coarse_sweeps": coarsest(args)[1]},
            "l2": "working set per step >> 129 MB L2 (no flush needed)",
            "parallelism": (f"angular decomposition over {world} GPUs (directions split, scalar flux all-reduced "
                            "every SI iteration)") if world > 1 else (
                               "1 GPU, all directions in one batch" if args.concurrent == 1 else
                               f"1 GPU, directions in {args.concurrent or 'the library default number of'} "
                               "concurrent groups"),
            "kernel_timing": f"CUDA events in the cycles of every {args.timing_every}th SI iteration",
            "precision": ("FP32 hierarchy/V-cycle, double-float refinement" if args.precision == 2 else
                          "FP32 hierarchy/V-cycle, FP64 refinement" if args.precision else "FP64")}


def coarsest(args, name=None):
    """(max_coarse, coarse_sweeps) of a workload: the command line's, else COARSEST's,
    else the library's defaults."""
    mc, cs = COARSEST.get(name or args.config, (100, 20))
    return (mc if args.max_coarse is None else args.max_coarse,
            cs if args.coarse_sweeps is None else args.coarse_sweeps)


def air_settings(args, distance=None, name=None):
    """The AIR parameters of the timed runs (both arms) of a workload (default: the
    command line's)."""
    mc, cs = coarsest(args, name)
    return dict(theta=args.theta, phi_R=args.phi_R, phi_A=args.phi_A,
                distance=args.distance if distance is None else distance, nair=args.nair,
                max_coarse=mc, coarse_sweeps=cs)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1910_11463_gb300 import inputs as I
    prob = I.config(args.config)
    # each step: one direction of the workload through the oracle (bounded CPU
    # sample); setup amortised over the SI iterations the workload needs
    from oracle import oracle as O
    O.build()
    akw = air_settings(args)
    fixed = args.si_fixed if args.si_fixed is not None else FIXED_SI.get(args.config, 0)
    si_iters = fixed or args.si_iters
    times = []
    for k in range(args.warmup + args.steps):
        a, b = oracle_direction_times(prob, k % prob.M, akw)
        if k >= args.warmup:
            times.append(a / si_iters + b)
    t = sum(times) / len(times)
    value = prob.N / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed directions (after {args.warmup} warm-up), "
                                       "single-threaded C oracle; a step = one direction of the workload: "
                                       "oracle assembly + AIR setup (amortised over "
                                       f"{si_iters} SI iterations) + one 1e-8 solve"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def kernel_table(infos, steps, ms, tet, precision):
    """Per kernel group of the timed steps: CUDA-event time inside the steps,
    algorithmic bytes counted by the library, launches (units), share of the step.
    The library times the cycles of every k-th SI iteration (si_params.timing), with
    the direction groups one after another: per-launch figures come from those
    cycles, and a group's share of the step scales their time by the iterations
    solved over the iterations timed."""
    def tot(key):
        return sum(i[key] for i in infos)
    scale = tot("si_iters") / max(tot("timed_iters"), 1)
    kern = {
        ("k_res0_csr" if tet else "k_res0_bsr_dd" if precision == 2 else "k_res0_bsr"): (
            ("FP64 outer residual, level 0 CSR" if tet else
             "outer residual in double-float pairs (FP32 pipe), level 0 block form" if precision == 2 else
             "FP64 outer residual, level 0 block form"),
            tot("t_res0_ms"), tot("n_res0"), tot("gb_res0")),
        ("k_relax_f+k_relax_c level 0" if tet else "k_relax0_split" if precision else "k_relax_bsr"): (
            "FP32 F-F-C Jacobi, level 0 " + ("CF-split CSR; one unit = one V-cycle's three sweeps" if tet
                                             else "CF-split block copy; one unit = one V-cycle's three sweeps"
                                             if precision else "block form; one unit = one V-cycle's sweeps"),
            tot("t_relax0_ms"), tot("n_relax0"), tot("gb_relax0")),
        "k_relax_f+k_relax_c": ("FP32 F-F-C Jacobi, levels >= 1 (CF-split SELL copies), and the grid-wide "
                                "coarsest-level Jacobi sweeps; one unit = every coarse level's sweeps of one "
                                "V-cycle", tot("t_relaxc_ms"), tot("n_relaxc"), tot("gb_relaxc")),
    }
    if tot("n_xfer") > 0:
        kern["k_restrict+k_prolong"] = (
            "grid transfers: every level's restriction b_l+1 = R_l b_l (SELL copy of Z) and one-point "
            "prolongation; one unit = one V-cycle's", tot("t_xfer_ms"), tot("n_xfer"), tot("gb_xfer"))
    if tot("n_res32") > 0:
        kern["k_res32_csr" if tet else "k_res32_bsr"] = (
            "FP32 inner residual r - A d of a refinement step, level 0 " + ("CSR" if tet else "block form"),
            tot("t_res32_ms"), tot("n_res32"), tot("gb_res32"))
    rl = {}
    for name, (what, t_ms, n_l, gb) in kern.items():
        rl[name] = {"what": what, "achieved_gbs": gb / (t_ms * 1e-3) if t_ms > 0 else None, "launches": n_l,
                    "ms_per_launch": t_ms / max(n_l, 1), "gb_per_launch": gb / max(n_l, 1),
                    "share_of_step": t_ms * scale / steps / ms, "timed_iterations": tot("timed_iters"),
                    "solved_iterations": tot("si_iters")}
    return rl


def measure_workload(name, args, pair, I, torch, steps=2, warmup=1, fp64=False):
    """One more workload on the current build, timed like the headline (CUDA events
    on the launching stream around `steps` steps after `warmup` untimed ones): a
    step is assembly + AIR setup of every direction + the workload's SI iterations,
    every direction solved from psi = 0 to a 1e-8 relative residual each iteration."""
    prob = I.config(name)
    dev = torch.device("cuda", torch.cuda.current_device())
    st, ss, qq = (torch.as_tensor(a, device=dev) for a in (prob.sigma_t, prob.sigma_s, prob.q))
    N, M = prob.N, prob.M
    tet = hasattr(prob, "tets")
    geom = pair.TetMesh(prob.verts, prob.tets, prob.nbr) if tet else prob.n
    fixed = FIXED_SI.get(name, 0)
    distance = DISTANCE.get(name, 1)
    kw = air_settings(args, distance, name)
    air = pair.default_air_params(precision=args.precision, **kw)
    si = (pair.default_si_params(tol=1e-8, max_iters=fixed, fixed_iters=1, inner_tol=1e-8, inner_maxit=200,
                                 use_graphs=args.graphs, concurrent=args.concurrent,
                                 timing=min(args.timing_every, fixed)) if fixed
          else pair.default_si_params(tol=1e-8, max_iters=1000, inner_tol=1e-8, inner_maxit=200,
                                      use_graphs=args.graphs, concurrent=args.concurrent,
                                      timing=args.timing_every))
    zero = torch.zeros(N, dtype=torch.float64, device=dev)

    def solve(a, s_):
        out, _, info = pair.si_solve(geom, prob.omega, prob.w, st, ss, qq, air=a, si=s_, phi0=zero)
        return out, info

    for _ in range(warmup):
        solve(air, si)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        phi, info = solve(air, si)
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    last = infos[-1]
    iters = last["si_iters"]
    t_setup = sum(i["t_setup_ms"] for i in infos) / steps
    t_solve = sum(i["t_solve_ms"] for i in infos) / steps
    rl = kernel_table(infos, steps, ms, tet, args.precision)
    peak, peak_kind = measured_peaks()
    dom = max(rl, key=lambda k: rl[k]["share_of_step"])
    entry = {"workload": name + ": " + WORKLOADS[name], "value": N * M * iters / (ms * 1e-3), "unit": UNIT,
             "ms_per_step": ms, "steps": steps, "warmup": warmup,
             "step": (f"assembly + AIR setup + {fixed} SI iterations from phi=0" if fixed else
                      "one complete SI solve from phi=0") + " (every direction from psi=0 to a 1e-8 relative "
                     "residual each iteration); value = DOF*dir*iterations/step time",
             "air": {"R": "nAIR degree 1" if args.nair else f"lAIR distance {distance}", "theta": args.theta,
                     "eps_R": 0.01, "phi_A": args.phi_A, "phi_R": args.phi_R, "max_coarse": kw["max_coarse"],
                     "coarse_sweeps": kw["coarse_sweeps"]},
             "si_iterations": iters, "setup_ms": t_setup, "solve_ms": t_solve,
             "solve_only_value": N * M * iters / (t_solve * 1e-3) if t_solve > 0 else None,
             "setup_phase_ms": dict(zip(("strength+pmis", "p+lair", "rap", "assembly+other"),
                                        [sum(i["t_setup_phase_ms"][k] for i in infos) / steps for k in range(4)])),
             "batches": last["batches"], "rebuilt_every_iteration": bool(last["rebuilt"]),
             "vcycles_per_direction_per_iteration": last["vcycles"] / M / max(iters, 1),
             "outer_residuals_per_direction_per_iteration": last["outer_residuals"] / M / max(iters, 1),
             "levels": last["levels_max"], "op_complexity": last["op_complexity"],
             "max_inner_resid": last["max_inner_resid"],
             "roofline": {"bound": "hbm", "kernel": dom, "achieved": rl[dom]["achieved_gbs"], "peak": peak,
                          "unit": "GB/s", "frac": (rl[dom]["achieved_gbs"] / peak) if rl[dom]["achieved_gbs"] else None,
                          "peak_source": f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (copy test)", "kernels": rl}}
    if fp64:
        air64 = pair.default_air_params(precision=0, **kw)
        si64 = pair.default_si_params(tol=1e-8, max_iters=fixed or 1000, fixed_iters=int(bool(fixed)),
                                      inner_tol=1e-8, inner_maxit=200, batch=1, use_graphs=0,
                                      concurrent=1)
        torch.cuda.synchronize()
        e0.record(stream)
        phi64, i64 = solve(air64, si64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        v64 = N * M * i64["si_iters"] / (ms64 * 1e-3)
        entry["fp64_one_direction"] = {"value": v64, "ms_per_step": ms64, "setup_ms": i64["t_setup_ms"],
                                       "speedup_of_fp32_refined_batched": entry["value"] / v64,
                                       "phi_rel_diff_fp32_refined_vs_fp64":
                                           (torch.linalg.norm(phi64 - phi) / torch.linalg.norm(phi64)).item()}
    return entry


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__ as g
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    g.build()
    from paper_1910_11463_gb300 import inputs as I
    from paper_1910_11463_gb300 import pair

    prob = I.config(args.config)
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.as_tensor(prob.sigma_t, device=dev)
    ss = torch.as_tensor(prob.sigma_s, device=dev)
    qq = torch.as_tensor(prob.q, device=dev)
    N, M = prob.N, prob.M
    geom = pair.TetMesh(prob.verts, prob.tets, prob.nbr) if hasattr(prob, "tets") else prob.n
    fixed = args.si_fixed if args.si_fixed is not None else FIXED_SI.get(args.config, 0)
    tuned = air_settings(args)
    air = pair.default_air_params(precision=args.precision, **tuned)
    if fixed:
        si = pair.default_si_params(tol=1e-8, max_iters=fixed, fixed_iters=1, inner_tol=1e-8, inner_maxit=200,
                                    use_graphs=args.graphs, concurrent=args.concurrent,
                                    timing=min(args.timing_every, fixed))
    else:
        si = pair.default_si_params(tol=1e-8, max_iters=1000, inner_tol=1e-8, inner_maxit=200,
                                    use_graphs=args.graphs, concurrent=args.concurrent, timing=args.timing_every)
    si_one = pair.default_si_params(tol=1e-8, max_iters=1, inner_tol=1e-8, inner_maxit=200,
                                    use_graphs=args.graphs, concurrent=args.concurrent)
    zero = torch.zeros(N, dtype=torch.float64, device=dev)

    from paper_1910_11463_gb300 import angle

    def solve(air_p, si_p, phi0):
        if world > 1:   # parallel in angle: this rank's directions, scalar flux all-reduced each iteration
            out, _, info, _ = angle.si_solve_angle(geom, prob.omega, prob.w, st, ss, qq, rank, world,
                                                   air=air_p, si=si_p, phi0=phi0)
        else:
            out, _, info = pair.si_solve(geom, prob.omega, prob.w, st, ss, qq, air=air_p, si=si_p, phi0=phi0)
        return out, info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        solve(air, si, zero)

    infos = []
    clocks = ClockSampler(torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = pair.kernel_launches()
    clocks.start()
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        phi, info = solve(air, si, zero)
        infos.append(info)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = pair.kernel_launches() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    iters = infos[-1]["si_iters"]
    # one problem whose directions are split over the ranks: the job solves N x M
    # DOF*directions per SI iteration whatever the number of ranks
    value = N * M * iters / (ms * 1e-3)

    def tot(key):
        return sum(i[key] for i in infos)
    t_setup, t_solve = tot("t_setup_ms") / args.steps, tot("t_solve_ms") / args.steps
    phases = [sum(i["t_setup_phase_ms"][k] for i in infos) / args.steps for k in range(4)]
    peak, peak_kind = measured_peaks()
    tet = hasattr(prob, "tets")
    rl = kernel_table(infos, args.steps, ms, tet, args.precision)
    dom = max(rl, key=lambda k: rl[k]["share_of_step"])
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tj = json.load(f)
        entry = tj.get(dom)
        # counters apply to the workload they were captured on, with the same kernel source
        if (entry and entry.get("workload") == args.config
                and entry.get("source_sha") == pair.kernel_source_sha(entry.get("source", "cycle.cu"))):
            traffic = entry["bytes_per_launch"] * (rl[dom]["gb_per_launch"] / entry["gb_per_launch_at_capture"])
    achieved = rl[dom]["achieved_gbs"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic, "kernel": dom,
                "peak_source": f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (copy test)",
                "algorithmic_bytes": "counted in the library from the hierarchy: per launch (level-0 kernels) or per V-cycle (all coarse levels' F, F and C sweeps and the coarsest level's Jacobi sweeps)",
                "kernels": rl}

    # the paper's memory mode: every hierarchy rebuilt for every iteration
    reb = []
    for k in range(3):
        barrier()
        e0.record(stream)
        solve(air, si_one, phi)
        e1.record(stream)
        barrier()
        reb.append(e0.elapsed_time(e1))
    ms_reb = sorted(reb)[1]
    rebuild = {"value": N * M / (ms_reb * 1e-3), "ms_per_iteration": ms_reb,
               "note": "assembly + AIR setup + one SI iteration per step (median of 3)"}

    # e2e: the same steps through the C ABI with HOST buffers (pinned): si_solve
    # itself copies sigma_t, sigma_s, q and the initial phi in and phi back out,
    # inside the timed region
    h_st = torch.as_tensor(prob.sigma_t).pin_memory()
    h_ss = torch.as_tensor(prob.sigma_s).pin_memory()
    h_q = torch.as_tensor(prob.q).pin_memory()
    h_phi = torch.zeros(N, dtype=torch.float64).pin_memory()
    om_e, w_e, red_e = prob.omega, prob.w, None
    if world > 1:
        m0, m1 = angle.direction_block(M, world, rank)
        om_e, w_e, red_e = prob.omega[m0:m1], prob.w[m0:m1], angle.allreduce_sum()
    e2e_steps = args.steps
    barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        h_phi.zero_()   # the step's initial guess
        info_e = pair.si_solve_host(geom, om_e, w_e, h_st, h_ss, h_q, h_phi, air=air, si=si, phi_reduce=red_e)
    e1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world, dev)
    e2e = {"value": N * M * info_e["si_iters"] / (ms_e2e * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": 3 * prob.E * 8 + N * 8, "d2h_bytes_per_step": N * 8, "ms_per_step": ms_e2e,
           "steps": e2e_steps, "phi_rel_diff_vs_device_api": (torch.linalg.norm(h_phi.to(dev) - phi)
                                                              / torch.linalg.norm(phi)).item()}

    # comparator: plain FP64 pAIR, one direction at a time, no graphs (same GPU, same AIR parameters)
    fp64 = None
    if not args.no_fp64_baseline:
        air64 = pair.default_air_params(precision=0, **tuned)
        si64 = pair.default_si_params(tol=1e-8, max_iters=fixed or 1000, fixed_iters=int(bool(fixed)),
                                      inner_tol=1e-8, inner_maxit=200, batch=1, use_graphs=0,
                                      concurrent=1)
        barrier()
        e0.record(stream)
        phi64, i64 = solve(air64, si64, zero)
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1)
        err = (torch.linalg.norm(phi64 - phi) / torch.linalg.norm(phi64)).item()
        fp64 = {"value": N * M * i64["si_iters"] / (ms64 * 1e-3), "ms_per_step": ms64, "si_iters": i64["si_iters"],
                "setup_ms": i64["t_setup_ms"], "solve_ms": i64["t_solve_ms"],
                "speedup_of_fp32_refined_batched": value / world / (N * M * i64["si_iters"] / (ms64 * 1e-3)),
                "phi_rel_diff_fp32_refined_vs_fp64": err}
    # comparator: the same source iteration with every direction solved exactly by the
    # GPU sweep (the solver AIR replaces): upwind wavefronts on hexes, the level
    # schedule with cyclic components on tets
    gsweep = None
    if not args.no_variants:
        si_sw = pair.default_si_params(tol=si.tol, max_iters=si.max_iters, fixed_iters=si.fixed_iters, solver=1)
        solve(air, si_sw, zero)
        barrier()
        e0.record(stream)
        for _ in range(2):
            phis, isw = solve(air, si_sw, zero)
        e1.record(stream)
        barrier()
        mss = e0.elapsed_time(e1) / 2
        gsweep = {"value": N * M * isw["si_iters"] / (mss * 1e-3), "ms_per_step": mss, "si_iters": isw["si_iters"],
                  "setup_ms": isw["t_setup_ms"], "solve_ms": isw["t_solve_ms"],
                  "phi_rel_diff_vs_air": (torch.linalg.norm(phis - phi) / torch.linalg.norm(phis)).item(),
                  "note": ("level schedule (one launch per upwind level, cyclic components as dense blocks), "
                           "all directions of the batch per launch" if hasattr(prob, "tets") else
                           "3n-2 upwind wavefronts per solve, all directions of the batch per launch")}
    # variant: the outer residual and iterate in double-float pairs on the FP32 pipe
    # instead of FP64 (hex block form; same hierarchy, same stopping test)
    dd = None
    if args.precision == 1 and not hasattr(prob, "tets") and not args.no_variants:
        air2 = pair.default_air_params(precision=2, **tuned)
        solve(air2, si, zero)
        barrier()
        e0.record(stream)
        for _ in range(2):
            phi2, i2 = solve(air2, si, zero)
        e1.record(stream)
        barrier()
        ms2 = e0.elapsed_time(e1) / 2
        dd = {"value": N * M * i2["si_iters"] / (ms2 * 1e-3), "ms_per_step": ms2, "si_iters": i2["si_iters"],
              "vcycles_per_direction_per_iteration": i2["vcycles"] / M / max(i2["si_iters"], 1),
              "max_inner_resid": i2["max_inner_resid"],
              "phi_rel_diff_vs_fp64_refinement": (torch.linalg.norm(phi2 - phi) / torch.linalg.norm(phi)).item(),
              "residual_gbs": i2["gb_res0"] / (i2["t_res0_ms"] * 1e-3) if i2["t_res0_ms"] > 0 else None}
    # variant: R from degree-1 nAIR with the R filter phi_R = 0.1 (the paper's
    # best-scaling configuration), everything else as the headline
    nair = None
    if not args.nair and not args.no_variants:
        kw = dict(tuned)
        kw.update(nair=1, phi_R=0.1)
        air3 = pair.default_air_params(precision=args.precision, **kw)
        solve(air3, si, zero)
        barrier()
        e0.record(stream)
        for _ in range(2):
            phi3, i3 = solve(air3, si, zero)
        e1.record(stream)
        barrier()
        ms3 = e0.elapsed_time(e1) / 2
        nair = {"value": N * M * i3["si_iters"] / (ms3 * 1e-3), "ms_per_step": ms3, "si_iters": i3["si_iters"],
                "setup_ms": i3["t_setup_ms"], "solve_ms": i3["t_solve_ms"],
                "vcycles_per_direction_per_iteration": i3["vcycles"] / M / max(i3["si_iters"], 1),
                "max_inner_resid": i3["max_inner_resid"],
                "phi_rel_diff_vs_headline": (torch.linalg.norm(phi3 - phi) / torch.linalg.norm(phi)).item()}
    # variant: the same solve without kernel-timing events (si_params.timing = 0), as
    # one batch and as the library's default concurrent direction groups
    untimed = None
    if not args.no_variants:
        untimed = {}
        for label, K in (("one_batch", 1), ("concurrent_groups_default", 0)):
            si_u = pair.default_si_params(tol=si.tol, max_iters=si.max_iters, fixed_iters=si.fixed_iters,
                                          inner_tol=si.inner_tol, inner_maxit=si.inner_maxit,
                                          use_graphs=si.use_graphs, concurrent=K, timing=0)
            solve(air, si_u, zero)
            barrier()
            e0.record(stream)
            for _ in range(2):
                phi_u, i_u = solve(air, si_u, zero)
            e1.record(stream)
            barrier()
            ms_u = max_over_ranks(e0.elapsed_time(e1) / 2, world, dev)
            untimed[label] = {"value": N * M * i_u["si_iters"] / (ms_u * 1e-3), "ms_per_step": ms_u,
                              "si_iters": i_u["si_iters"], "batches": i_u["batches"],
                              "phi_rel_diff_vs_headline":
                                  (torch.linalg.norm(phi_u - phi) / torch.linalg.norm(phi)).item()}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    last = infos[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": ("f32 V-cycle + f32-pair residual/iterate + f64 setup"
                                       if args.precision == 2 and not hasattr(prob, "tets")
                                       else "f32 V-cycle + f64 residual/setup" if args.precision else "f64"),
        "data": "synthetic",
        "config": bench_config(args, world),
        "si_iterations": iters, "setup_ms": t_setup, "solve_ms": t_solve,
        "solve_only_value": N * M * iters * world / (t_solve * 1e-3) if t_solve > 0 else None,
        "setup_phase_ms": {"strength+pmis": phases[0], "p+lair": phases[1], "rap": phases[2],
                           "assembly+other": phases[3]},
        "rebuild_every_iteration": rebuild,
        "vcycles_per_direction_per_iteration": last["vcycles"] / M / max(iters, 1),
        "outer_residuals_per_direction_per_iteration": last["outer_residuals"] / M / max(iters, 1),
        "coarse_relax_ms_per_cycle_by_level": [
            sum(i["t_relaxc_level_ms"][k] for i in infos) / max(sum(i["n_relaxc"] for i in infos), 1)
            for k in range(8)],
        "levels": last["levels_max"],
        "op_complexity": last["op_complexity"], "max_inner_resid": last["max_inner_resid"],
        "roofline": roofline, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
        "fp64_one_direction": fp64,
        "gpu_sweep": gsweep,
        "variants": {"double_float_refinement": dd, "nair_degree1_phiR_0.1": nair, "without_kernel_timing": untimed},
    }
    # the other synthetic meshes on the same build: unstructured tets (distance-2
    # lAIR) and the 64^3 scale run, each with its per-kernel roofline
    if world == 1 and args.config == "hex32_s4" and not args.no_workloads:
        line["workloads"] = {w: measure_workload(w, args, pair, I, torch, fp64=(w == "tet40_s8"))
                             for w in ("tet40_s8", "hex64_s8")}
    if world == 1 or rank == 0:
        line["cpu_baseline"] = (cpu_baseline_oracle(prob, iters, tuned, max_seconds=args.cpu_seconds)
                                if not args.no_cpu else None)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="hex32_s4", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2],
                    help="0 FP64; 1 FP32 V-cycle under FP64 refinement (default); 2 FP32 V-cycle under "
                         "double-float refinement (hex block form)")
    ap.add_argument("--timing-every", dest="timing_every", type=int, default=9,
                    help="kernel timings in SI iterations k, 2k, ... (si_params.timing)")
    ap.add_argument("--concurrent", type=int, default=1,
                    help="direction groups solved at the same time on their own streams (0: library default; "
                         "1: one batch, so the timed kernels are whole-batch launches)")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="1: V-cycles launched as CUDA graphs (default); 0: launched directly")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the tet40_s8 and hex64_s8 entries printed beside the hex32_s4 headline")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the variants (double-float refinement, nAIR with phi_R = 0.1)")
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--phi-R", dest="phi_R", type=float, default=0.0)
    ap.add_argument("--phi-A", dest="phi_A", type=float, default=0.05)
    ap.add_argument("--max-coarse", dest="max_coarse", type=int, default=None,
                    help="a level with at most this many rows per direction is the coarsest (default: 40000 for "
                         "hex32_s4, hex64_s8 and tet40_s8, else the library's 100)")
    ap.add_argument("--coarse-sweeps", dest="coarse_sweeps", type=int, default=None,
                    help="Jacobi sweeps from zero on the coarsest level (default: 3 for those workloads, else the "
                         "library's 20)")
    ap.add_argument("--nair", type=int, default=0, choices=[0, 1],
                    help="1: R from degree-1 nAIR (Neumann series) instead of lAIR local solves")
    ap.add_argument("--distance", type=int, default=None, choices=[1, 2],
                    help="lAIR distance (default: 2 for tet40_s8, else 1)")
    ap.add_argument("--si-fixed", dest="si_fixed", type=int, default=None,
                    help="run exactly this many SI iterations per step (default: 2 for hex64_s8 and tet40_s8, "
                         "0 = solve to 1e-8 for the others)")
    ap.add_argument("--eps-study", action="store_true",
                    help="eps_R of the R pattern vs convergence, setup and solve time, distance 1 and 2")
    ap.add_argument("--mms-study", action="store_true",
                    help="error against the manufactured solution vs V-cycles per SI iteration, 8^3/16^3/32^3")
    ap.add_argument("--one-iteration", action="store_true",
                    help="profiling aid: assembly + setup + one SI iteration of the workload, no timing line")
    ap.add_argument("--si-iters", type=int, default=18,
                    help="SI iterations the setup is amortised over in the reference arm (hex32_s4 needs 18)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)   # timing rule: at least three untimed warm-up steps
    if args.distance is None:
        args.distance = DISTANCE.get(args.config, 1)
    if args.impl == "reference":
        return run_reference(args)
    if args.one_iteration:
        return run_one_iteration(args)
    if args.mms_study:
        return run_mms_study(args)
    if args.eps_study:
        return run_eps_study(args)
    return run_ours(args)


def run_eps_study(args):
    """Sec. 4.1.1 study: the strength threshold eps_R of the R pattern against
    convergence, setup and solve time, for distance-1 and distance-2 lAIR, on the
    bench workload (complete SI solve from phi = 0, every direction to 1e-8).
    The effective convergence factor of a direction solve is 1e-8^(1/cycles).
    Prints one JSON line."""
    import torch
    import __graft_entry__ as g
    torch.cuda.set_device(0)
    g.build()
    from paper_1910_11463_gb300 import inputs as I
    from paper_1910_11463_gb300 import pair
    prob = I.config(args.config)
    st = torch.as_tensor(prob.sigma_t, device="cuda")
    ss = torch.as_tensor(prob.sigma_s, device="cuda")
    qq = torch.as_tensor(prob.q, device="cuda")
    si = pair.default_si_params(tol=1e-8, max_iters=1000, inner_tol=1e-8, inner_maxit=200)
    rows = []
    for distance in (1, 2):
        for eps in (0.001, 0.01, 0.1, 0.25):
            air = pair.default_air_params(precision=args.precision, eps_R=eps, **air_settings(args, distance))
            for _ in range(2):   # the first run also tunes the new shapes
                phi, _, info = pair.si_solve(prob.n, prob.omega, prob.w, st, ss, qq, air=air, si=si)
            torch.cuda.synchronize()
            cyc = info["vcycles"] / prob.M / max(info["si_iters"], 1)
            rows.append({"distance": distance, "eps_R": eps, "setup_ms": info["t_setup_ms"],
                         "solve_ms": info["t_solve_ms"], "si_iters": info["si_iters"],
                         "vcycles_per_solve": cyc, "conv_factor": 1e-8 ** (1.0 / cyc) if cyc > 0 else None,
                         "op_complexity": info["op_complexity"], "levels": info["levels_max"]})
    print(json.dumps({"study": "eps_R of the R pattern (Sec. 4.1.1)", "workload": args.config,
                      "theta": args.theta, "phi_A": args.phi_A, "rows": rows}))
    return 0


def run_mms_study(args):
    """Sec. 3 study: error of the scalar flux against the manufactured solution of
    the appendix when every direction gets a fixed number of V-cycles from zero per
    SI iteration, on three meshes; 0 cycles = each solve to a 1e-10 residual (the
    converged error).
    Prints one JSON line."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    torch.cuda.set_device(0)
    g.build()
    from paper_1910_11463_gb300 import inputs as I
    from paper_1910_11463_gb300 import pair
    air = pair.default_air_params(precision=args.precision, theta=args.theta, phi_R=args.phi_R, phi_A=args.phi_A,
                                  nair=args.nair)
    rows = []
    for n in (8, 16, 32):
        prob, q_ang, phi_exact = I.mms_hex(n, order=4)
        pe = torch.as_tensor(phi_exact, device="cuda")
        for cyc in (1, 2, 3, 4, 6, 8, 0):
            # SI to a 1e-8 change (far below the discretisation errors measured here)
            si = pair.default_si_params(tol=1e-8, max_iters=300, fixed_iters=1, inner_tol=1e-10,
                                        inner_maxit=200, inner_cycles=cyc)
            phi, _, info = pair.si_solve_problem(prob, air=air, si=si, q_ang=q_ang)
            err = (torch.linalg.norm(phi - pe) / torch.linalg.norm(pe)).item()
            rows.append({"n": n, "h": 1.0 / n, "cycles": cyc if cyc else "to 1e-10", "rel_l2_error": err,
                         "si_iters": info["si_iters"], "si_change": info["si_change"],
                         "final_inner_resid": info["max_inner_resid"],
                         "solve_ms": info["t_solve_ms"]})
    print(json.dumps({"study": "MMS error vs fixed V-cycles per SI iteration (Sec. 3)", "quadrature": "S4",
                      "sigma_t": 1.0, "sigma_s": 0.5, "air": "lAIR" if not args.nair else "nAIR",
                      "precision": args.precision, "rows": rows}))
    return 0


def run_one_iteration(args):
    """One SI iteration of the workload (the launch sequence an ncu capture of the
    V-cycle kernels needs, without the bench's repetitions)."""
    import torch
    import __graft_entry__ as g
    torch.cuda.set_device(0)
    g.build()
    from paper_1910_11463_gb300 import inputs as I
    from paper_1910_11463_gb300 import pair
    prob = I.config(args.config)
    air = pair.default_air_params(precision=args.precision, **air_settings(args))
    si = pair.default_si_params(tol=1e-8, max_iters=1, inner_tol=1e-8, inner_maxit=200,
                                use_graphs=args.graphs, concurrent=args.concurrent, timing=0)
    phi, _, info = pair.si_solve_problem(prob, air=air, si=si)
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.config, "setup_ms": info["t_setup_ms"], "solve_ms": info["t_solve_ms"],
                      "vcycles": info["vcycles"], "levels": info["levels_max"]}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
