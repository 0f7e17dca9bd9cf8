#!/usr/bin/env python
"""Benchmark of the staggered DG time step on one GB300 (or N replicas).

A "step" is one full time step of the scheme (projections, SSP-RK3
convection, implicit viscous CG per component, pressure CG, velocity update,
gauge) on the 2D 256 x 256, N = 7 perturbed Taylor-Green workload.

Headline value: pressure-CG throughput in GDOF/s = (pressure DOF x operator
applications) / device time of the pressure solves, in the mixed
FP32-iteration / FP64-reliable-update mode at rtol 1e-12.  ms_per_step is the
whole step.  The plain-FP64 step and the mixed-vs-FP64 error of one step from
the same state are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

# the oracle (CPU baseline) is timed single-threaded
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pressure-CG GDOF/s & s/time-step, mixed vs FP64 at <=1e-10 rel err; % HBM peak"
WORKLOAD = "tg2d_256x256_N7"
CPU_SAMPLE_CELLS = (32, 32)      # oracle sample: same degree / parameters, 32 x 32 cells
FLUSH_BYTES = 512 << 20          # > 129 MB L2
# fused CG operator of the default iteration form (FP32): read r, p_old, x;
# write p, Ap, x (x += alpha p_old of the previous iteration rides along)
BYTES_PER_DOF_FUSED_F32 = 24


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed plain-FP64 steps (after one warm-up)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tg3d-steps", type=int, default=20,
                    help="timed steps of the 3D 48^3, N = 4 workload in each precision (after one warm-up); "
                         "0 skips it")
    ap.add_argument("--batch-steps", type=int, default=1,
                    help="timed steps of the 48-problem batch (after one warm-up); 0 skips it")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def ncu_traffic(workload=WORKLOAD):
    """DRAM bytes per launch of the fused FP32 operator on `workload` from a
    committed ncu summary (null when absent)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d.get(workload, {}).get("fused_apply_f32_bytes")


def reduce_over_ranks(dist, step_ms, solve_ms, work, device):
    """Whole-job numbers of independent replicas: the slowest rank's times
    (max) and the work of all ranks (sum).  dist None: a single process."""
    if dist is None:
        return step_ms, solve_ms, work
    import torch
    t = torch.tensor([step_ms, solve_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(w)
    return float(t[0]), float(t[1]), float(w[0])


# ----------------------------------------------------------------- oracle timing
def oracle_sample_pressure_solve(cells=CPU_SAMPLE_CELLS):
    """Time the oracle's pressure CG on a bounded sample of the workload: the
    same degree, viscosity, theta, dt and perturbation on `cells` cells.
    The right-hand side comes from the oracle's own projections, convection
    and viscous solves (not timed).  Returns (GDOF/s, seconds, dof, applies)."""
    from oracle import Grid, Oracle, cg
    import sdg_inputs as si
    from paper_1602_05806_gb300.workloads import WORKLOADS, cfl_number, convection_substeps
    w = WORKLOADS[WORKLOAD]
    L = (2 * math.pi,) * 2
    o = Oracle(Grid(2, cells, L), w["N"], w["nu"], w["theta"], w["dt"])
    m = w["modes"]
    modes = si.stream_modes(m["seed"], m["nmodes"], m["kmax"], m["amplitude"])
    U = []
    for d in range(2):
        x, y = o.coords(d)
        U.append(si.taylor_green_2d(x, y)[d] + si.perturbation_velocity(modes, x, y)[d])
    cfl = cfl_number(2, cells, L, w["N"], w["dt"], [float(np.abs(u).max()) for u in U])
    o.nsub = convection_substeps(cfl) if cfl >= 1.0 else 1
    x, y = o.coords(None)
    P = si.taylor_green_2d(x, y)[2]
    P = P - o.physical_mean(P)
    V = [o.dual_to_main(U[d], d) for d in range(2)]
    F = o.rk3(V)
    Vh = [cg(o.viscous_apply, o.mass_all(F[c]), F[c], 1e-12).x for c in range(2)]
    Us = [o.main_to_dual(Vh[d], d) for d in range(2)]
    b = o.pressure_rhs(Us, P)
    b = b - b.mean()
    t0 = time.perf_counter()
    res = cg(o.pressure_apply, b, P, 1e-12, maxit=1000000)
    dt = time.perf_counter() - t0
    applies = res.iters + 1
    return o.ndof * applies / dt / 1e9, dt, o.ndof, applies


def _oracle_worker(cells):
    """One oracle sample solve in a pool process: (DOF x applications, seconds)."""
    _, secs, dof, applies = oracle_sample_pressure_solve(tuple(cells))
    return dof * applies, secs


def host_cpu():
    """(logical cores, CPU model name) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def oracle_all_cores(cells, rounds=1, procs=None):
    """The oracle on every host core: `procs` single-threaded processes (spawn
    start method) each solve the same sample, `rounds` times; throughput =
    all their work / wall time.  Returns (GDOF/s, wall seconds per round,
    processes, DOF x applications per round)."""
    import multiprocessing as mp
    procs = procs or (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_worker, [(4, 4)] * procs)  # imports and first calls, untimed
        work, t0 = 0.0, time.perf_counter()
        for _ in range(rounds):
            work += sum(w for w, _ in pool.map(_oracle_worker, [cells] * procs))
        wall = time.perf_counter() - t0
    return work / wall / 1e9, wall / rounds, procs, work / rounds


# ----------------------------------------------------------------- reference arm
REF_SAMPLE_CELLS = (24, 24)      # reference arm: one pool round per step, ~5 s


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores, model = host_cpu()
    # warm-up: tiny oracle solves in the pool (numpy has no compile step)
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    secs, work = [], 0.0
    with ctx.Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_worker, [(4, 4)] * cores)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            work += sum(w for w, _ in pool.map(_oracle_worker, [REF_SAMPLE_CELLS] * cores))
            secs.append(time.perf_counter() - t0)
    value = work / sum(secs) / 1e9
    n1 = 8
    dof = REF_SAMPLE_CELLS[0] * REF_SAMPLE_CELLS[1] * n1 * n1
    sample = (f"oracle pressure CG (numpy FP64, rtol 1e-12) on {REF_SAMPLE_CELLS[0]}x{REF_SAMPLE_CELLS[1]} "
              f"cells of the {WORKLOAD} workload ({dof} DOF), one single-threaded solve per host core per "
              f"step ({cores} processes, spawn pool; CPU: {model})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_cells": list(REF_SAMPLE_CELLS)},
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1602_05806_gb300 import build as _build
    if rank == 0:
        _build.build()
    barrier()
    from paper_1602_05806_gb300 import sdg
    from paper_1602_05806_gb300.workloads import workload_state

    w, U0, P0 = workload_state(WORKLOAD)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    h = sdg.Handle(2, w["n"], w["L"], w["N"], w["nu"], w["theta"], w["dt"])
    h.set_convection_substeps(w["nsub"])
    ndof = h.ndof
    h.set_options(sdg.SDG_MIXED, 1e-12, 1e-12)
    h.set_state([dev(u) for u in U0], dev(P0))
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # ---- warm-up (mixed)
    for _ in range(args.warmup):
        info = h.step(1)
        assert info["status"] == sdg.SDG_OK, info

    # ---- timed mixed steps (no per-launch instrumentation inside)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    barrier()
    sampler.start()
    p_ms = 0.0
    p_applies = 0
    launches = 0
    p_iters = []
    p_true, p_floor = [], []
    for k in range(args.steps):
        flush.fill_(float(k))  # evict L2 between steps (outside the step's events)
        ev[k][0].record(stream)
        info = h.step(1)
        ev[k][1].record(stream)
        assert info["status"] == sdg.SDG_OK, info
        p_ms += info["pressure_ms"]
        p_applies += info["pressure_applies"]
        launches += info["kernel_launches"]
        p_iters.append(info["pressure"]["iters"])
        p_true.append(info["pressure"]["true_res"])
        p_floor.append(info["pressure"]["floor_res"])
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]

    # ---- one more step with CUDA events around every launch of the fused
    # FP32 operator (on the launch stream), for its roofline
    h.set_profiling(True)
    flush.fill_(-1.0)
    info = h.step(1)
    assert info["status"] == sdg.SDG_OK, info
    cnt = h.counters()
    h.set_profiling(False)

    tot_step_ms = sum(step_ms)
    # max over ranks of the times, sum of the work
    tot_step_ms, p_ms_max, work = reduce_over_ranks(dist, tot_step_ms, p_ms, float(ndof * p_applies), "cuda")
    value = work / (p_ms_max * 1e-3) / 1e9

    # ---- dominant kernel: fused FP32 CG operator (roofline)
    peaks, peak_src = measured_peaks()
    n32 = cnt["apply_launches"][1]
    avg_ms = cnt["apply_ms"][1] / n32 if n32 else float("nan")
    bytes_per_launch = BYTES_PER_DOF_FUSED_F32 * ndof
    achieved_gbs = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    flops_per_dof = (6 * (w["N"] + 1) + 2) * 2
    achieved_tflops = flops_per_dof * ndof / (avg_ms * 1e-3) / 1e12
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # FMA lanes x 2 flop x clock
    frac_hbm = achieved_gbs / hbm_peak
    frac_alu = achieved_tflops / fp32_peak
    traffic = ncu_traffic()
    if frac_hbm >= frac_alu:
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": frac_hbm, "traffic": traffic}
    else:
        roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": frac_alu, "traffic": traffic}
    roofline.update({"kernel": "k_apply<float,2,8> (fused CG operator: x += alpha p_old, p = r + beta p_old, "
                               "A p, p.Ap; timed in one extra step with events around each launch)",
                     "avg_launch_us": avg_ms * 1e3, "launches_timed": n32,
                     "peak_source": peak_src + (" (hbm_gbs)" if roofline["bound"] == "hbm"
                                                else " (152 SM x 128 FP32 lanes x 2 x sm_max_mhz)"),
                     "hbm_frac": frac_hbm, "alu_frac": frac_alu,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "flops_per_launch": flops_per_dof * ndof})

    # ---- plain FP64 step and mixed-vs-FP64 error from the same state
    fp64 = None
    accuracy = None
    if args.fp64_steps > 0:
        Us = [torch.empty_like(dev(U0[0])) for _ in range(2)]
        Ps = torch.empty_like(Us[0])
        h.get_state(Us, Ps)
        h.set_options(sdg.SDG_FP64, 1e-12, 1e-12)
        h.step(1)  # warm-up
        h.get_state(Us, Ps)  # state S
        f_ms, f_pms, f_app, f_it = [], 0.0, 0, []
        for k in range(args.fp64_steps):
            if k == 0:
                S = ([u.clone() for u in Us], Ps.clone())
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            info = h.step(1)
            b.record(stream)
            torch.cuda.synchronize()
            assert info["status"] == sdg.SDG_OK, info
            f_ms.append(a.elapsed_time(b))
            f_pms += info["pressure_ms"]
            f_app += info["pressure_applies"]
            f_it.append(info["pressure"]["iters"])
            f_true = info["pressure"]["true_res"]
            f_floor = info["pressure"]["floor_res"]
            if k == 0:
                U64 = [torch.empty_like(Us[0]) for _ in range(2)]
                P64 = torch.empty_like(Us[0])
                h.get_state(U64, P64)
        fp64 = {"gdofs": ndof * f_app / (f_pms * 1e-3) / 1e9, "ms_per_step": statistics.mean(f_ms),
                "pressure_iters": f_it, "steps": args.fp64_steps, "warmup": 1,
                "pressure_true_res": f_true, "pressure_floor_res": f_floor}
        # the same step in mixed precision from state S
        h.set_options(sdg.SDG_MIXED, 1e-12, 1e-12)
        h.set_state(S[0], S[1])
        m_info = h.step(1)
        Um = [torch.empty_like(Us[0]) for _ in range(2)]
        Pm = torch.empty_like(Us[0])
        h.get_state(Um, Pm)
        relerr = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        accuracy = {"mixed_vs_fp64_rel_l2": {"u": relerr(Um[0], U64[0]), "v": relerr(Um[1], U64[1]),
                                             "p": relerr(Pm, P64)},
                    "pressure_true_res": {"mixed": m_info["pressure"]["true_res"], "fp64": f_true},
                    "pressure_floor_res": m_info["pressure"]["floor_res"],
                    "speedup_mixed_over_fp64_step": statistics.mean(f_ms) / (tot_step_ms / args.steps),
                    "note": ("both solves stop on the true FP64 residual <= max(rtol, 3 floor_res), floor_res "
                             "the residual that rounding the solution to FP64 leaves")}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        hostU = [torch.empty(U0[0].shape, dtype=torch.float64).pin_memory() for _ in range(2)]
        hostP = torch.empty(P0.shape, dtype=torch.float64).pin_memory()
        h.get_state(hostU, hostP)
        torch.cuda.synchronize()
        t_tot, app = 0.0, 0
        for k in range(args.e2e_steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.set_state(hostU, hostP)         # H2D of the step's input state
            info = h.step(1)
            h.get_state(hostU, hostP)         # D2H of the step's result
            t_tot += time.perf_counter() - t0
            app += info["pressure_applies"]
        e2e = {"value": ndof * app / t_tot / 1e9, "unit": "GDOF/s",
               "h2d_bytes_per_step": 3 * ndof * 8, "d2h_bytes_per_step": 3 * ndof * 8,
               "ms_per_step": 1000 * t_tot / args.e2e_steps}

    # ---- 3D workload: 48^3 cells, N = 4 (block hepta-diagonal pressure system):
    # the same steps from the same state in mixed precision and in FP64,
    # kinetic energy after every step, and the roofline of the 3D operator
    tg3d = None
    if args.tg3d_steps > 0:
        w3, U3, P3 = workload_state("tg3d_48_N4")
        h3 = sdg.Handle(3, w3["n"], w3["L"], w3["N"], w3["nu"], w3["theta"], w3["dt"])
        h3.set_convection_substeps(w3["nsub"])
        res3, K3 = {}, {}
        for prec, name in ((sdg.SDG_MIXED, "mixed"), (sdg.SDG_FP64, "fp64")):
            h3.set_options(prec, 1e-12, 1e-12)
            h3.set_state([dev(u) for u in U3], dev(P3))
            assert h3.step(1)["status"] == sdg.SDG_OK  # warm-up
            h3.set_state([dev(u) for u in U3], dev(P3))
            ms, pms, app, its, ks, trs, launches3 = 0.0, 0.0, 0, [], [], [], 0
            for k in range(args.tg3d_steps):
                flush.fill_(0.25 + k)
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                inf = h3.step(1)
                e.record(stream)
                torch.cuda.synchronize()
                assert inf["status"] == sdg.SDG_OK, inf
                ms += a.elapsed_time(e)
                pms += inf["pressure_ms"]
                app += inf["pressure_applies"]
                launches3 += inf["kernel_launches"]
                its.append(inf["pressure"]["iters"])
                trs.append(inf["pressure"]["true_res"])
                ks.append(h3.diagnostics()[0])  # outside the step's events
            K3[name] = ks
            res3[name] = {"ms_per_step": ms / args.tg3d_steps,
                          "pressure_gdofs": h3.ndof * app / (pms * 1e-3) / 1e9, "pressure_iters": its,
                          "pressure_true_res_max": max(trs), "kinetic_energy": [ks[0], ks[-1]],
                          "gpu_launches": launches3}
        # roofline of the fused FP32 3D operator: one more mixed step with events
        # around each of its launches
        h3.set_options(sdg.SDG_MIXED, 1e-12, 1e-12)
        h3.set_profiling(True)
        flush.fill_(-2.0)
        assert h3.step(1)["status"] == sdg.SDG_OK
        c3 = h3.counters()
        h3.set_profiling(False)
        n3 = c3["apply_launches"][1]
        avg3 = c3["apply_ms"][1] / n3 if n3 else float("nan")
        b3 = BYTES_PER_DOF_FUSED_F32 * h3.ndof
        ach3 = b3 / (avg3 * 1e-3) / 1e9
        hbm_peak3 = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
        dK = max(abs(a - b) / abs(b) for a, b in zip(K3["mixed"], K3["fp64"]))
        tg3d = {"workload": "tg3d_48_N4 (3D TG, 48^3 cells, N 4, nu 1/1600, dt 1e-3, rtol 1e-12)",
                "dof": h3.ndof, "steps": args.tg3d_steps, "warmup": 1, **res3,
                "kinetic_energy_mixed_vs_fp64_max_rel": dK,
                "roofline": {"bound": "hbm", "achieved": ach3, "peak": hbm_peak3, "unit": "GB/s",
                             "frac": ach3 / hbm_peak3, "traffic": ncu_traffic("tg3d_48_N4"),
                             "kernel": "k_apply3m<float,5> (fused z-marching CG operator: x += alpha p_old, "
                                       "p = r + beta p_old, A p, p.Ap; events around each launch "
                                       "in one extra mixed step)",
                             "avg_launch_us": avg3 * 1e3, "launches_timed": n3,
                             "algorithmic_bytes_per_launch": b3}}
        h3.close()

    # ---- batched workload: 48 independent problems stepped concurrently
    batch = None
    if args.batch_steps > 0:
        from paper_1602_05806_gb300.workloads import batch_workload
        bw, problems, states = batch_workload()
        bt = sdg.Batch(problems, bw["theta"], bw["dt"])
        for i, (U, P) in enumerate(states):
            m = bt.members[i]
            m.set_options(sdg.SDG_MIXED, 1e-12, 1e-12)
            m.set_convection_substeps(bw["nsub"][i])
            m.set_state([dev(u) for u in U], dev(P))
        okc = (sdg.SDG_OK, sdg.SDG_ERR_NOT_CONVERGED)
        rc, _ = bt.step(1, ok=okc)  # warm-up
        flush.fill_(0.5)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        rc, infos = bt.step(args.batch_steps, stream=stream, ok=okc)
        e.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(e)
        work = sum(m.ndof * inf["pressure_applies"] for m, inf in zip(bt.members, infos))
        short = [(i, bt.members[i].N, inf["pressure"]["true_res"]) for i, inf in enumerate(infos)
                 if inf["pressure"]["status"] != sdg.SDG_OK]
        batch = {"workload": "batch48_seed2 (2D, 16^2..128^2 cells, N 2..11, mixed, rtol 1e-12)",
                 "problems": len(bt), "dof_total": sum(m.ndof for m in bt.members),
                 "steps": args.batch_steps, "warmup": 1, "ms_per_step": ms / args.batch_steps,
                 "pressure_gdof_applies_per_s": work / (ms * 1e-3) / 1e9,
                 "pressure_iters_max": max(inf["pressure"]["iters"] for inf in infos),
                 "pressure_true_res_max": max(inf["pressure"]["true_res"] for inf in infos),
                 "members_short_of_rtol": [{"member": i, "N": N, "true_res": r} for i, N, r in short],
                 "threads": "min(48, 16, cores) host threads, one stream per member"}
        bt.close()

    # ---- CPU baseline (rank 0, N = 1): the oracle on one core and on all of them
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v1, s1, dof, applies = oracle_sample_pressure_solve()
        vall, wall, procs, _ = oracle_all_cores(CPU_SAMPLE_CELLS)
        cores, model = host_cpu()
        cpu = {"value": vall, "unit": "GDOF/s", "cores": procs, "kind": "oracle",
               "single_core": {"value": v1, "cores": 1, "seconds": s1},
               "cpu_model": model,
               "sample": (f"oracle pressure CG (numpy FP64, rtol 1e-12) on {CPU_SAMPLE_CELLS[0]}x"
                          f"{CPU_SAMPLE_CELLS[1]} cells of the workload: {dof} DOF, {applies} operator "
                          f"applications; value: {procs} single-threaded processes (one per host core, spawn "
                          f"pool) solving it at once, {wall:.1f} s wall; single_core: one process, {s1:.1f} s")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_step_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "dim": 2, "cells": list(w["n"]), "N": w["N"],
                           "dof": ndof, "nu": w["nu"], "theta": w["theta"], "dt": w["dt"],
                           "cfl": round(w["cfl"], 3), "convection_substeps": w["nsub"],
                           "rtol": 1e-12, "precision": "FP32 CG, FP64 reliable updates",
                           "l2": "512 MB buffer written between timed steps (outside the step events)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "pressure_iters_per_step": p_iters, "pressure_ms_total": p_ms,
                "pressure_true_res_max": max(p_true), "pressure_floor_res": max(p_floor),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "fp64": fp64, "accuracy": accuracy, "tg3d": tg3d, "batch": batch}
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
