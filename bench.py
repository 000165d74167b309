#!/usr/bin/env python
"""Benchmark: implicit Euler heat steps of the tensor B-spline operator at 928^3.

Workload (the paper's ~0.8 G-node scale, synthetic): 928^3 = 799,178,752 unknowns on the unit
cube, cubic B-splines, zero Dirichlet faces, dt = 5e-4, initial coefficients = 64 seeded sine
modes (k in {1..16}^3, amplitudes N(0,1)/|k|^2), one implicit Euler step per benchmark step,
solved to a 1e-8 true relative residual by CG with FP32 operator sweeps and iterative
refinement (FP64-accurate true residual -- double-float arithmetic on the FP32 pipes, FP64
input and output -- FP64 update and CG scalars).

value = operator throughput inside the solve: unknowns x operator applications / time, summed
over ranks, where every application of the full operator counts (inner FP32 CG iterations and
the true residuals; the mass-only right-hand side is not counted). Each rank solves its own
problem (weak scaling, no collective on the data path).

--impl reference runs the FP64 CPU oracle (the test-suite's reference implementation) on a
bounded slab of the same workload, in the same unit.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "operator GDoF/s (% HBM peak) at 928³; time-to-1e-8 residual, FCG-net vs CG"
N_GRID, DEGREE, DT, TOL, SEED, NMODES, KMAX = 928, 3, 5e-4, 1e-8, 3, 64, 16
WORKLOAD = "heat3d_928cube_cubic_f32sweeps_f64refinement"


# DRAM bytes per unknown of one launch of each single-pass CG kernel (dram__bytes_read.sum +
# dram__bytes_write.sum over the unknowns of the launch), measured on the 512^3 profiling case
# (`--profile-case cg512`) and scaled to the benchmark grid by its unknowns; valid only while the
# kernels' sources hash to CG_TRAFFIC_SOURCES_SHA256 (None: no capture of the current sources).
# 512^3 capture (--metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum):
# k_op_tma<float,3,CG> 2.915 + 1.569 GB, k_ws<3,WS_CG> with chunked items 2.191 + 1.559 GB and
# with whole-column items 2.151 + 1.559 GB per launch.
CG_TRAFFIC_BYTES_PER_UNKNOWN = {"classic": 33.41, "ws": 27.94, "ws_columns": 27.64}
# Algorithmic bytes per unknown of one single-pass FP32 CG iteration.
CG_BYTES_PER_UNKNOWN = 28.0
CG_TRAFFIC_SOURCES_SHA256 = "fbb43515eb447f8e6870b37431ce25ee7b4f83b8ab0fc17502205d2a888f04fb"
CG_KERNEL_SOURCES = ("op_tma.cuh", "op_ws.cuh", "tma_impl.cuh", "tma_util.cuh", "bsk_device.cuh",
                     "tma_f32.cu", "ws_f32.cu")


def cg_kernel_sources_sha256() -> str:
    import hashlib
    d = hashlib.sha256()
    for name in CG_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1904_03057_gb300", "csrc", name), "rb") as f:
            d.update(f.read())
    return d.hexdigest()


def max_over_ranks(value: float, dist, device="cuda") -> float:
    """The largest value over all ranks (the job's wall time is its slowest rank's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gdofs(world: int, dofs_per_rank: int, op_apps_per_rank: float, seconds: float) -> float:
    """Weak scaling: every rank solves its own problem of the same size; the job's throughput is
    all ranks' unknowns x operator applications over the slowest rank's time."""
    return world * dofs_per_rank * op_apps_per_rank / seconds / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples (200 ms) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev, self.lines, self.proc = dev, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, maximum SM clock and the throttle reasons seen in `FIELDS` lines
        (csv, no header, no units); lines that do not parse are skipped."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                clk, clk_max = float(parts[0]), float(parts[1])
            except ValueError:
                continue
            sm.append(clk)
            mx.append(clk_max)
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_sample(reps: int = 3, planes: int = 16):
    """FP64 oracle operator (Fig. FiltAlg separable chains, OpenMP) on a 928 x 928 x planes slab
    of the workload's field; returns (GDoF/s, cores, seconds, description)."""
    import numpy as np
    import torch

    import oracle
    from paper_1904_03057_gb300 import inputs
    h = 1.0 / (N_GRID + 1)
    modes = inputs.random_sine_modes(SEED, NMODES, KMAX)
    full = inputs.sine_mode_field(N_GRID, N_GRID, planes, modes, h=h, dtype=torch.float64)
    x = full.numpy()
    p = oracle.Problem(N_GRID, N_GRID, planes, DEGREE, h, dt=DT)
    oracle.op_separable(p, x)  # warm-up (page faults, thread start)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.op_separable(p, x)
    dt_s = time.perf_counter() - t0
    dofs = N_GRID * N_GRID * planes * reps
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"{reps} FP64 oracle operator applications on a 928x928x{planes} slab "
            f"({N_GRID * N_GRID * planes} unknowns) of the 928^3 workload")
    return dofs / dt_s / 1e9, cores, dt_s, desc


def cpu_model() -> str:
    """The host CPU's name as /proc/cpuinfo gives it (x86 "model name", Arm implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model", "CPU part"):
        for ln in info.splitlines():
            if ln.startswith(key):
                val = ln.split(":", 1)[1].strip()
                if key == "CPU part":
                    impl = next((x.split(":", 1)[1].strip() for x in info.splitlines()
                                 if x.startswith("CPU implementer")), "?")
                    return f"Arm CPU implementer {impl}, part {val}"
                return val
    return "unknown"


def cpu_baseline_by_config(line) -> dict:
    """The FP64 oracle timed on the host cores for every workload the line reports, next to the
    GPU figure. Config 1 is solved whole; the others take the oracle's measured time per
    operator application (a separable FP64 sweep over the whole grid, every core) times the
    operator applications the GPU run needed, and are labelled extrapolated. About 10 s of CPU
    work in all."""
    import numpy as np
    import torch

    import oracle
    from paper_1904_03057_gb300 import inputs

    def t_op(p, x):
        oracle.op_separable(p, x)                 # warm-up (pages, threads)
        t0 = time.perf_counter()
        oracle.op_separable(p, x)
        return time.perf_counter() - t0

    out = {"cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "cpu": cpu_model()}
    # config 1: 32^3, cubic, sin sin sin, dt = 1e-3, 10 steps, tol 1e-10, FP64 -- whole solve
    c1 = line.get("c1_32cube_fp64")
    if c1:
        N = 32
        h = 1.0 / (N + 1)
        p = oracle.Problem(N, N, N, DEGREE, h, dt=1e-3)
        u0 = inputs.sine_mode_field(N, N, N, [((1, 1, 1), 1.0)]).numpy()
        t0 = time.perf_counter()
        oracle.heat(p, u0, None, 10, tol=1e-10)
        out["c1_32cube_10_steps"] = {"oracle_ms": 1e3 * (time.perf_counter() - t0), "gpu_ms": c1["ms"],
                                     "kind": "measured"}
    # config 2: 256^3 sphere, FP64 CG, 50 steps
    c2 = line.get("mixed_precision_sphere256")
    if c2:
        N = 256
        h = 1.0 / (N + 1)
        mask = inputs.sphere_mask(N, N, N, (0.5, 0.5, 0.5), 0.45, h=h).numpy()
        p = oracle.Problem(N, N, N, DEGREE, h, dt=1e-3, mask=mask)
        t = t_op(p, np.random.default_rng(0).standard_normal(p.shape) * mask)
        apps = c2["f64"]["iterations_per_step"] + 2   # CG iterations + right-hand side + residual
        out["c2_256_sphere_50_steps"] = {
            "oracle_ms": 1e3 * t * apps * 50, "gpu_ms_fp64": c2["f64"]["ms_per_step"] * 50,
            "gpu_ms_f32_ir": c2["f32_ir"]["ms_per_step"] * 50, "oracle_ms_per_operator": 1e3 * t,
            "kind": "extrapolated (oracle operator time x the FP64 run's applications)"}
    # config 3: 928^3 heat step (the line's headline), from the slab sample of the same field
    v, cores, secs, desc = cpu_oracle_sample(reps=1)
    apps = line["config"]["op_applications_per_step"]
    out["c3_928_heat_step"] = {"oracle_ms": 1e3 * N_GRID ** 3 * apps / (v * 1e9), "gpu_ms": line["ms_per_step"],
                               "oracle_gdofs": v, "kind": "extrapolated (" + desc + ")"}
    # config 4: the 64 boxes, from one box solved whole
    c4 = line.get("batch_64_boxes")
    if c4:
        specs = inputs.batch_problems(seed=4)
        s = sorted(specs, key=lambda q: q.nx * q.ny * q.nz)[len(specs) // 2]   # the median box
        p = oracle.Problem(s.nx, s.ny, s.nz, s.degree, s.h, dt=1e-3)
        qf = inputs.gaussian_source(s.nx, s.ny, s.nz, s.centers, 0.03, h=s.h).numpy()
        t0 = time.perf_counter()
        _, its, _, _ = oracle.heat(p, np.zeros(p.shape), qf, 1, tol=1e-8)
        dt_s = time.perf_counter() - t0
        rate = s.nx * s.ny * s.nz * (int(np.sum(its)) + 2) / dt_s          # unknowns x applications / s
        apps_b = c4["batched_gdofs"] * 1e9 * c4["batched_ms"] * 1e-3
        out["c4_64_boxes"] = {"oracle_ms": 1e3 * apps_b / rate, "gpu_ms_batched": c4["batched_ms"],
                              "gpu_ms_sequential": c4["sequential_ms"],
                              "kind": f"extrapolated (box {s.nx}x{s.ny}x{s.nz} n={s.degree} solved whole: "
                                      f"{rate / 1e9:.3f} GDoF/s)"}
    # config 5: 512^3 union of spheres, plain FP64 CG to 1e-8
    c5 = line.get("fcg_race")
    if c5:
        N = 512
        h = 1.0 / (N + 1)
        centers, radii = inputs.random_spheres(5, 40, 0.05, 0.2)
        mask = inputs.union_of_spheres_mask(N, N, N, centers, radii, h=h).numpy()
        p = oracle.Problem(N, N, N, DEGREE, h, dt=1e-3, mask=mask)
        t = t_op(p, np.random.default_rng(0).standard_normal(p.shape) * mask)
        apps = c5["fp64_cg"]["iterations"] + 2
        out["c5_512_spheres_to_1e-8"] = {
            "oracle_ms": 1e3 * t * apps, "gpu_ms_fp64_cg": c5["fp64_cg"]["ms"],
            "gpu_ms_f32_ir_cg": c5["f32_ir_cg"]["ms"], "gpu_ms_fcg_net_ir": c5["fcg_net_ir"]["ms"],
            "oracle_ms_per_operator": 1e3 * t,
            "kind": "extrapolated (oracle operator time x the FP64 CG run's applications)"}
    del torch
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_sample(reps=1)
    vals, total = [], 0.0
    for _ in range(args.steps):
        v, cores, secs, desc = cpu_oracle_sample(reps=1)
        vals.append(v)
        total += secs
    value = len(vals) / sum(1.0 / v for v in vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": desc,
                                        "runs_on": "host CPU cores (FP64 oracle); rank 0 only"},
        "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _timed_ms(fn):
    """Device time of fn() on the current stream (CUDA events, synchronised on both sides)."""
    import torch
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def batch_64_boxes():
    """64 independent boxes (dims U{48..160} per axis, degrees 2..5, 8 Gaussian
    sources each, dt = 1e-3), one implicit Euler step of every box to a 1e-8 true residual:
    the batched persistent solver (autotuned decomposition) against the same problems solved one
    after another through single handles. Throughput counts unknowns x operator applications."""
    import torch

    from paper_1904_03057_gb300 import api, inputs
    dt, tol = 1e-3, 1e-8
    specs = inputs.batch_problems(seed=4)
    qs = [inputs.gaussian_source(s.nx, s.ny, s.nz, s.centers, 0.03, h=s.h, device="cuda") for s in specs]
    B = api.BatchHandle(specs, dt)
    tune = B.autotune(3)
    dofs = [s.nx * s.ny * s.nz for s in specs]
    # each degree group's tuned pass against HBM: 32 algorithmic bytes per unknown per
    # single-pass CG iteration (read r, q, p, x; write r, q, p, x in FP32)
    peak, peak_kind = peaks()
    tune["hbm_peak"] = {"gbs": peak, "kind": peak_kind}
    for g in tune["groups"]:
        unknowns = sum(d for d, s in zip(dofs, specs) if s.degree == g["degree"])
        gbs = 32.0 * unknowns / (g["ms"] * 1e-3) / 1e9 if g["ms"] > 0 else None
        g["unknowns"] = unknowns
        g["hbm_gbs"] = gbs
        g["hbm_frac"] = gbs / peak if (gbs and peak) else None

    def fresh():
        return [torch.zeros((s.nz, s.ny, s.nx), dtype=torch.float64, device="cuda") for s in specs]

    B.heat_step(fresh(), qs, 1, tol=tol)                 # warm-up (graphs)
    us = fresh()
    ms_b, reps_b = _timed_ms(lambda: B.heat_step(us, qs, 1, tol=tol))
    apps_b = sum(d * (r["iterations"] + r["outer_iterations"] + 1) for d, r in zip(dofs, reps_b))
    B.close()
    hs = [api.Handle(s.nx, s.ny, s.nz, s.degree, s.h, dt, precision="f32_ir") for s in specs]
    for H, q, u in zip(hs, qs, fresh()):                 # warm-up
        H.heat_step(u, q, 1, tol=tol)
    us2 = fresh()
    ms_s, reps_s = _timed_ms(lambda: [H.heat_step(u, q, 1, tol=tol) for H, q, u in zip(hs, qs, us2)])
    apps_s = sum(d * (r["iterations"] + r["outer_iterations"] + 1) for d, r in zip(dofs, reps_s))
    diff = max((torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item() for a, b in zip(us, us2))
    for H in hs:
        H.close()
    return {"workload": "64 boxes, dims U{48..160}^3, degrees 2-5, one heat step, tol 1e-8",
            "unknowns": sum(dofs), "batched_ms": ms_b, "sequential_ms": ms_s,
            "speedup_batched_vs_sequential": ms_s / ms_b,
            "batched_gdofs": apps_b / (ms_b * 1e-3) / 1e9, "sequential_gdofs": apps_s / (ms_s * 1e-3) / 1e9,
            "max_rel_residual": max(r["rel_residual"] for r in reps_b),
            "max_rel_diff_batched_vs_sequential": diff, "autotune": tune}


def mixed_precision_sphere256(steps: int = 50):
    """256^3, sphere mask r = 0.45 at the centre, 32 Gaussian sources (sigma 0.03,
    centres U[0.2,0.8]^3, seed 2), u0 = 0, dt = 1e-3, `steps` implicit Euler steps to a 1e-8 true
    residual, FP64 CG against FP32 CG with FP64-accurate refinement: time per step, iterations,
    and the relative difference of the final fields."""
    import torch

    from paper_1904_03057_gb300 import api, inputs
    N, dt, tol = 256, 1e-3, 1e-8
    h = 1.0 / (N + 1)
    mask = inputs.sphere_mask(N, N, N, (0.5, 0.5, 0.5), 0.45, h=h, device="cuda")
    q = inputs.gaussian_source(N, N, N, inputs.gaussian_centers(2, 32), sigma=0.03, h=h, mask=mask,
                               device="cuda")
    out = {"workload": f"256^3 sphere r=0.45, 32 Gaussian sources, dt=1e-3, {steps} steps, tol 1e-8",
           "active_unknowns": int(mask.sum().item())}
    us = {}
    for prec in ("f64", "f32_ir"):
        H = api.Handle(N, N, N, DEGREE, h, dt, mask=mask, precision=prec)
        H.heat_step(torch.zeros((N, N, N), dtype=torch.float64, device="cuda"), q, 1, tol=tol)   # warm-up
        u = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
        ms, rep = _timed_ms(lambda: H.heat_step(u, q, steps, tol=tol))
        out[prec] = {"ms_per_step": ms / steps, "iterations_per_step": rep["iterations"] / steps,
                     "last_rel_residual": rep["rel_residual"]}
        us[prec] = u
        H.close()
    out["speedup_f32_ir_vs_f64"] = out["f64"]["ms_per_step"] / out["f32_ir"]["ms_per_step"]
    out["rel_diff_f32_ir_vs_f64"] = (torch.linalg.vector_norm(us["f32_ir"] - us["f64"])
                                     / torch.linalg.vector_norm(us["f64"])).item()
    return out


def fcg_race():
    """The 512^3 union-of-40-spheres race: one implicit Euler step from u = 0 with a
    Gaussian source, dt = 1e-3, each solver from x = 0 to a 1e-8 true relative residual: plain
    FP64 CG, FP32 CG with FP64 refinement, and flexible CG preconditioned by the trained linear
    network inside FP64 refinement. The network is trained first (32^3 crops at the same h and
    dt; its time is reported separately); solves are timed with CUDA events after a warm-up."""
    import torch

    from paper_1904_03057_gb300 import api, inputs, learned
    N, dt, tol = 512, 1e-3, 1e-8
    h = 1.0 / (N + 1)
    t0 = time.perf_counter()
    problems = learned.make_problems(40, crop=32, h=h, dt=dt, seed=2, noise_fraction=0.25)
    pairs = learned.make_pairs(440, crop=32, h=h, dt=dt, problems=problems,
                               ks=(0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32))
    tr = api.Net(32, 32, 32, activation="linear")
    tr.set_params(learned.init_params(0, h=h, dt=dt))
    learned.train_on_policy(tr, pairs, problems[:12], rounds=3)
    params = tr.get_params()
    tr.close()
    del pairs, problems
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    centers, radii = inputs.random_spheres(5, 40, 0.05, 0.2)
    mask = inputs.union_of_spheres_mask(N, N, N, centers, radii, h=h, device="cuda")
    q = inputs.gaussian_source(N, N, N, inputs.gaussian_centers(5, 32), sigma=0.03, h=h, mask=mask,
                               device="cuda")
    H64 = api.Handle(N, N, N, DEGREE, h, dt, mask=mask, precision="f64")
    b = H64.mass_apply(q) * dt          # (M + dt K) u1 = M (u0 + dt q), u0 = 0
    del q
    stream = torch.cuda.current_stream()

    def timed(fn):
        x = torch.zeros_like(b)
        fn(x, 1e-3)                      # warm-up: graphs, work vectors
        x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = fn(x, tol)
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms": e0.elapsed_time(e1), "iterations": rep["iterations"],
                "outer_iterations": rep["outer_iterations"], "rel_residual": rep["rel_residual"],
                "status": rep["status"], "fallback_iter": rep["fallback_iter"]}

    out = {"workload": "union40spheres_512cube_cubic_dt1e-3_one_step", "tol": tol,
           "active_unknowns": int(mask.sum().item())}
    out["fp64_cg"] = timed(lambda x, t: H64.cg_solve(b, x, tol=t))
    H64.close()
    H32 = api.Handle(N, N, N, DEGREE, h, dt, mask=mask, precision="f32_ir")
    out["f32_ir_cg"] = timed(lambda x, t: H32.cg_solve(b, x, tol=t))
    out["fcg_plain_ir"] = timed(lambda x, t: H32.fcg_solve(b, x, None, tol=t))
    net = api.Net(N, N, N, activation="linear")
    net.set_params(params)
    out["fcg_net_ir"] = timed(lambda x, t: H32.fcg_solve(b, x, net, tol=t))
    net.close()
    H32.close()
    out["training_s"] = train_s
    out["speedup_fcg_net_vs_fp64_cg"] = out["fp64_cg"]["ms"] / out["fcg_net_ir"]["ms"]
    out["iterations_fcg_net_vs_fcg_plain"] = (out["fcg_net_ir"]["iterations"]
                                              / max(out["fcg_plain_ir"]["iterations"], 1))
    return out


# Per-SM FP32 lanes and SM count of a GB300 (152 SMs x 128 FP32 lanes, one FMA = 2 flops per
# lane per clock): the ALU roofline of the variable-coefficient kernel at the sampled maximum SM
# clock.
FP32_LANES = 152 * 128


def variable_coefficients():
    """The variable-coefficient operator A(d, m) (D and mu_a as B-spline fields) on the grids
    the paper times its on-the-fly operator on (240 x 240 x 960, degrees 1-3, FP32 and FP64;
    522^3 cubic FP32), with inclusion fields D (contrast up to 25) and mu_a; one application per
    timing, inputs larger than L2. Also one implicit Euler step (m = 1 + dt mu_a) solved to a
    1e-8 true residual by FP32 CG inside FP64 refinement on a 256^3 sphere."""
    import torch

    from paper_1904_03057_gb300 import api, inputs
    out = {"operator": [], "note": "flop counts per node from bsk_op_flops: algorithmic = per-cell "
                                   "Gauss quadrature with sum factorisation, executed = with the "
                                   "halo cells each block recomputes"}
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    cases = [(n, (240, 240, 960), p) for p in ("f32", "f64") for n in (1, 2, 3)]
    cases.append((3, (522, 522, 522), "f32"))
    for n, (nx, ny, nz), prec in cases:
        h = 1.0 / (max(nx, ny, nz) + 1)
        H = api.Handle(nx, ny, nz, n, h, 5e-4, precision=prec)
        d = inputs.inclusion_coefficients(nx, ny, nz, seed=7, h=h, device="cuda")
        m = 1.0 + 0.5 * inputs.inclusion_coefficients(nx, ny, nz, seed=8, h=h, base=0.3, device="cuda")
        H.set_coefficients(d, m)
        del d, m
        ms = H.time_kernel(api.KERNEL_OP, reps=2 if prec == "f64" else 5)
        alg, exe = H.op_flops()
        nodes = nx * ny * nz
        out["operator"].append({
            "grid": f"{nx}x{ny}x{nz}", "degree": n, "precision": prec, "ms": ms,
            "gnodes_per_s": nodes / (ms * 1e-3) / 1e9,
            "flop_per_node": {"algorithmic": alg, "executed": exe},
            "tflops": {"algorithmic": nodes * alg / (ms * 1e-3) / 1e12,
                       "executed": nodes * exe / (ms * 1e-3) / 1e12}})
        H.close()
        torch.cuda.empty_cache()
    # one implicit Euler step with variable coefficients, time to a 1e-8 true residual
    N = 256
    h = 1.0 / (N + 1)
    dt = 5e-4
    mask = inputs.sphere_mask(N, N, N, radius=0.45, h=h, device="cuda")
    H = api.Handle(N, N, N, 3, h, dt, mask=mask, precision="f32_ir")
    d = inputs.inclusion_coefficients(N, N, N, seed=7, h=h, device="cuda")
    mu = 10.0 * inputs.inclusion_coefficients(N, N, N, seed=8, h=h, base=0.3, device="cuda")
    H.set_coefficients(d, 1.0 + dt * mu)
    del d, mu
    u = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
    q = inputs.gaussian_source(N, N, N, inputs.gaussian_centers(2, 32), sigma=0.03, h=h,
                               mask=mask, device="cuda")
    u0 = u.clone()
    H.heat_step(u.clone(), q, 1, tol=1e-8)   # warm-up (graph capture)
    ms, rep = _timed_ms(lambda: H.heat_step(u, q, 1, tol=1e-8))
    out["heat_step_256_sphere"] = {"ms": ms, "cg_iterations": rep["iterations"],
                                   "refinement_steps": rep["outer_iterations"],
                                   "true_rel_residual": rep["rel_residual"],
                                   "coefficients": "D inclusions (0.2-5 in background 1), "
                                                   "m = 1 + dt mu_a"}
    # the same step with Jacobi-preconditioned CG (the diagonal probed once, timed apart)
    ms_probe, _ = _timed_ms(lambda: H.set_preconditioner("jacobi"))
    H.heat_step(u0.clone(), q, 1, tol=1e-8)
    ms_j, rep_j = _timed_ms(lambda: H.heat_step(u0, q, 1, tol=1e-8))
    out["heat_step_256_sphere_jacobi"] = {"ms": ms_j, "cg_iterations": rep_j["iterations"],
                                          "refinement_steps": rep_j["outer_iterations"],
                                          "true_rel_residual": rep_j["rel_residual"],
                                          "diagonal_probe_ms": ms_probe}
    del u0
    H.close()
    del u, q, mask
    torch.cuda.empty_cache()
    clocks = sampler.stop()
    top = next(r for r in out["operator"] if r["degree"] == 3 and r["precision"] == "f32"
               and r["grid"] == "240x240x960")
    mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = FP32_LANES * 2 * mhz * 1e6 / 1e12
    ach = top["tflops"]["algorithmic"]
    out["roofline"] = {"kernel": "k_op_var<float,3,OP> on 240x240x960", "bound": "alu",
                       "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                       "executed_frac": top["tflops"]["executed"] / peak, "traffic": None,
                       "note": "peak = 152 SMs x 128 FP32 lanes x 2 flop x the sampled maximum "
                               "SM clock; achieved = algorithmic flops / kernel time"}
    out["clocks"] = clocks
    # the paper's own times for one application on the same grids (other hardware, context):
    # Table tblPerformance (24-core CPU) and Table tblGpu (one GPU, 522^3)
    out["paper_seconds"] = {"240x240x960 f32 n=1,2,3": [0.87, 3.65, 9.87],
                            "240x240x960 f64 n=1,2,3": [1.07, 6.93, 15.11],
                            "522x522x522 f32 n=3": 21.079}
    return out


def robin_large_run(iters: int = 200):
    """A synthetic analogue of the paper's large run (section 3): 600 x 600 x 2400 unknowns
    (0.86 G), linear B-splines, Robin boundary penalty, FP64 Jacobi-preconditioned CG, started
    from a 120 x 120 x 480 solution prolonged to the fine grid. The steady problem here is
    M + K + pen E (perfusion-like mass term, unit conductivity) with 8 Gaussian heat sources
    (seed 6); pen = 1e3. Reports the time per PCG iteration, and the residual after a fixed
    number of iterations from zero and from the prolonged coarse solution (the paper ran a
    fixed 1000 iterations, in 4 h 4 min on its 24-core CPU)."""
    import numpy as np
    import torch

    from paper_1904_03057_gb300 import api, inputs
    n, pen, dt = 1, 1.0e3, 1.0
    nt_f, nt_c = (600, 600, 2400), (120, 120, 480)
    hf = 1.0 / (nt_f[2] - 1)            # box [0, 1] along z: (N + 1) h = 1 with N = nt - 2
    hc = 1.0 / (nt_c[2] - 1)
    # the coarse grid covers the same box: (nt_c - 1) hc = (nt_f - 1) hf per axis
    hcs = tuple((f - 1) * hf / (c - 1) for f, c in zip(nt_f, nt_c))
    out = {"grid": "600x600x2400", "coarse": "120x120x480", "degree": n, "penalty": pen,
           "precision": "FP64", "iterations": iters}
    Hc = api.Handle(*nt_c, n, hcs, dt, precision="f64")
    Hf = api.Handle(*nt_f, n, hf, dt, precision="f64")
    for H in (Hc, Hf):
        H.set_boundary("robin", pen)
        H.set_preconditioner("jacobi")
    rng = np.random.default_rng(6)
    cs = [tuple(rng.uniform(0.2, 0.8, size=3) * np.array([(c - 1) * hf for c in nt_f])) for _ in range(8)]

    def load(H, nt, h3):
        # a Gaussian field sampled at the B-spline centres (generator nodes are offset by one
        # step for the linear Robin basis), loaded with the grid's mass matrix
        q = inputs.gaussian_source(*nt, [(c[0] + h3[0], c[1] + h3[1], c[2] + h3[2]) for c in cs],
                                   sigma=0.03, h=h3, device="cuda")
        b = H.mass_apply(q)
        del q
        return b
    bc = load(Hc, nt_c, hcs)
    xc = torch.zeros(bc.shape, dtype=torch.float64, device="cuda")
    ms_c, rep_c = _timed_ms(lambda: Hc.cg_solve(bc, xc, tol=1e-8, max_iter=20000))
    bf = load(Hf, nt_f, (hf, hf, hf))
    ms_p, x0 = _timed_ms(lambda: api.prolong(Hf, Hc, xc))
    res = {}
    for name, start in (("from_zero", None), ("from_coarse", x0)):
        x = torch.zeros_like(bf) if start is None else start
        ms, rep = _timed_ms(lambda: Hf.cg_solve(bf, x, tol=1e-14, max_iter=iters))
        res[name] = {"ms": ms, "iterations": rep["iterations"], "rel_residual": rep["rel_residual"]}
        del x
    ms_it = res["from_zero"]["ms"] / max(res["from_zero"]["iterations"], 1)
    nodes = nt_f[0] * nt_f[1] * nt_f[2]
    # dominant kernel: the fused FP64 CG pass (Jacobi p update, A p with the Robin rows, x
    # update, p.Ap), timed alone; algorithmic work 7 band convolutions of 2n + 1 taps per unknown
    ms_cgp = Hf.time_kernel(api.KERNEL_CG_FUSED, reps=3)
    ms_upd = Hf.time_kernel(api.KERNEL_CG_UPDATE, reps=3)
    flops = 14.0 * (2 * n + 1) * nodes
    # TFLOP/s, nominal GB300 FP64: 152 SMs x 2 DFMA per clock x 2 flop x 2.07 GHz (ncu reports a
    # DFMA peak of 304 per cycle for the whole GPU); no measured FP64 peak is recorded
    fp64_peak = 1.25
    out["kernel_ms"] = {"cg_fused_f64": ms_cgp, "cg_update_f64": ms_upd}
    out["roofline"] = {"kernel": "k_op_generic<double,1,CGP,RB> (Robin, Jacobi)", "bound": "fp64",
                       "achieved": flops / (ms_cgp * 1e-3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                       "frac": flops / (ms_cgp * 1e-3) / 1e12 / fp64_peak, "traffic": None,
                       "hbm_gbs": 56.0 * nodes / (ms_cgp * 1e-3) / 1e9,
                       "note": "algorithmic 14 (2n + 1) flop per unknown; peak = nominal FP64 rate "
                               "(152 SMs x 2 DFMA/clock x 2 flop x 2.07 GHz); "
                               "hbm_gbs = 56 B/unknown (r, p, 1/diag A read; p, q written; x read and written)"}
    Hf.close()
    torch.cuda.empty_cache()
    # the same problem and start with FP32 inner PCG inside FP64 refinement (the library's
    # mixed-precision path), for the same number of inner iterations
    Hm = api.Handle(*nt_f, n, hf, dt, precision="f32_ir")
    Hm.set_boundary("robin", pen)
    Hm.set_preconditioner("jacobi")
    xm = x0.clone()
    ms_m, rep_m = _timed_ms(lambda: Hm.cg_solve(bf, xm, tol=1e-14, max_iter=iters, inner_tol=1e-6))
    res["from_coarse_f32_inner_f64_refinement"] = {"ms": ms_m, "iterations": rep_m["iterations"],
                                                   "refinement_steps": rep_m["outer_iterations"],
                                                   "rel_residual": rep_m["rel_residual"]}
    Hm.close()
    del xm
    out.update({"coarse_solve": {"ms": ms_c, "iterations": rep_c["iterations"],
                                 "rel_residual": rep_c["rel_residual"]},
                "prolong_ms": ms_p, "fine": res, "ms_per_pcg_iteration": ms_it,
                "gdofs_per_pcg_iteration": nodes / (ms_it * 1e-3) / 1e9,
                "projected_1000_iterations_s": ms_it * 1000 / 1e3,
                "paper_1000_iterations_s": 4 * 3600 + 4 * 60})
    Hc.close()
    del bf, bc, xc, x0
    torch.cuda.empty_cache()
    return out


def profile_case(name: str, cg_kernel: str = "auto"):
    """Small cases for the profiler: `cg512` runs 12 single-pass FP32 CG iterations of the
    benchmark's operator at 512^3 (537 MB per vector, a 3.8 GB handle) and then times that pass
    alone; `op384` applies the FP32 cubic operator of the benchmark
    (unmasked box, dt = 5e-4) to the benchmark's kind of field at 384^3 (226 MB per vector, larger
    than L2) four times; `var240` runs the variable-coefficient operator (cubic, FP32,
    240 x 240 x 960, the inclusion fields of `variable_coefficients`) three times; `robin200` runs
    10 iterations of the FP64 Jacobi-preconditioned Robin CG of `robin_large_run` on 200 x 200 x
    800 unknowns (256 MB per vector), then times its fused CG pass alone; `batch64` runs the 64-box
    batched measurement (autotuned tiles and z-chunks) and prints it; `net512` applies the learned
    preconditioner of `fcg_race` (linear network, Jacobi-scale start) to a masked residual at the
    race's 512^3 four times (about 2.4 GB on the device: r, z, mask and four activations)."""
    import torch

    from paper_1904_03057_gb300 import api, inputs
    if name == "batch64":
        print(json.dumps({"profile_case": name, **batch_64_boxes()}), flush=True)
        return
    if name == "cg512":
        N = 512
        h = 1.0 / (N + 1)
        H = api.Handle(N, N, N, DEGREE, h, DT, precision="f32")
        kern = H.select_cg_kernel(cg_kernel)
        modes = inputs.random_sine_modes(SEED, NMODES, KMAX)
        b = inputs.sine_mode_field(N, N, N, modes, device="cuda", dtype=torch.float64).float()
        x = torch.zeros_like(b)
        ms, rep = _timed_ms(lambda: H.cg_solve(b, x, tol=1e-30, max_iter=12, check_every=4))
        ms_cg = H.time_kernel(api.KERNEL_CG_FUSED, reps=5)
        print(json.dumps({"profile_case": name, "cg_kernel": kern, "solve_ms": ms,
                          "iterations": rep["iterations"], "cg_fused_ms": ms_cg}), flush=True)
        return
    if name == "op384":
        N = 384
        h = 1.0 / (N + 1)
        H = api.Handle(N, N, N, DEGREE, h, DT, precision="f32")
        modes = inputs.random_sine_modes(SEED, NMODES, KMAX)
        x = inputs.sine_mode_field(N, N, N, modes, device="cuda", dtype=torch.float64).float()
        y = torch.empty_like(x)
        ms = [_timed_ms(lambda: H.op_apply(x, y))[0] for _ in range(4)]
        print(json.dumps({"profile_case": name, "ms": ms, "max_abs_y": float(y.abs().max())}), flush=True)
        return
    if name == "net512":
        from paper_1904_03057_gb300 import learned
        N = 512
        h = 1.0 / (N + 1)
        centers, radii = inputs.random_spheres(5, 40, 0.05, 0.2)
        mask = inputs.union_of_spheres_mask(N, N, N, centers, radii, h=h, device="cuda")
        r = inputs.random_field((N, N, N), 9, device="cuda", dtype=torch.float32) * mask
        net = api.Net(N, N, N, activation="linear")
        net.set_params(learned.init_params(0, h=h, dt=1e-3))
        z = torch.empty_like(r)
        ms = [_timed_ms(lambda: net.forward(r, mask, z))[0] for _ in range(4)]
        print(json.dumps({"profile_case": name, "ms": ms, "max_abs_z": float(z.abs().max())}), flush=True)
        net.close()
        return
    if name == "robin200":
        import numpy as np
        nt = (200, 200, 800)
        h = 1.0 / (nt[2] - 1)
        H = api.Handle(*nt, 1, h, 1.0, precision="f64")
        H.set_boundary("robin", 1.0e3)
        H.set_preconditioner("jacobi")
        rng = np.random.default_rng(6)
        cs = [tuple(rng.uniform(0.2, 0.8, size=3) * np.array([(c - 1) * h for c in nt]) + h) for _ in range(8)]
        q = inputs.gaussian_source(*nt, cs, sigma=0.03, h=(h, h, h), device="cuda")
        b = H.mass_apply(q)
        x = torch.zeros_like(b)
        ms, rep = _timed_ms(lambda: H.cg_solve(b, x, tol=1e-14, max_iter=10))
        ms_cgp = H.time_kernel(api.KERNEL_CG_FUSED, reps=3)
        print(json.dumps({"profile_case": name, "solve_ms": ms, "iterations": rep["iterations"],
                          "cg_fused_ms": ms_cgp}), flush=True)
        return
    if name != "var240":
        raise ValueError(name)
    nx, ny, nz = 240, 240, 960
    h = 1.0 / 961
    H = api.Handle(nx, ny, nz, 3, h, 5e-4, precision="f32")
    d = inputs.inclusion_coefficients(nx, ny, nz, seed=7, h=h, device="cuda")
    m = 1.0 + 0.5 * inputs.inclusion_coefficients(nx, ny, nz, seed=8, h=h, base=0.3, device="cuda")
    H.set_coefficients(d, m)
    x = inputs.random_field((nz, ny, nx), 9, device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    ms = [_timed_ms(lambda: H.op_apply(x, y))[0] for _ in range(3)]
    print(json.dumps({"profile_case": name, "ms": ms, "max_abs_y": float(y.abs().max())}), flush=True)


def run_ours(args, rank, world, dist):
    import torch

    from paper_1904_03057_gb300 import api, inputs
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    N = args.grid
    h = 1.0 / (N + 1)
    dofs = N ** 3
    # the pinned host buffer of the end-to-end steps is allocated first and touched once. The
    # host link moves up to 190-210 GB/s, but the rate varies from box to box (device-to-host
    # ran at 12-19 GB/s on some); the measured rates are reported with the e2e figure.
    uh = None
    if not args.no_e2e:
        uh = torch.empty((N, N, N), dtype=torch.float64, pin_memory=True)
        uh.zero_()
    modes = inputs.random_sine_modes(SEED + rank, NMODES, KMAX)
    u = inputs.sine_mode_field(N, N, N, modes, device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream()
    H = api.Handle(N, N, N, DEGREE, h, DT, precision="f32_ir", stream=stream)
    cg_kernel = H.select_cg_kernel(args.cg_kernel if args.cg_kernel != "auto" else "current")
    opts = dict(tol=TOL, check_every=16)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        H.heat_step(u, None, 1, **opts)
    barrier()
    sampler = ClockSampler(dev)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = []
    e0.record(stream)
    for _ in range(args.steps):
        reps.append(H.heat_step(u, None, 1, **opts))
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1), dist)
    inner = sum(r["iterations"] for r in reps)
    outer = sum(r["outer_iterations"] for r in reps)
    op_apps = inner + outer + len(reps)          # inner CG + true residuals (one per outer + final)
    launches = sum(r["kernel_launches"] for r in reps)
    value = whole_job_gdofs(world, dofs, op_apps, elapsed_ms * 1e-3)
    ms_step = elapsed_ms / args.steps
    worst_res = max(r["rel_residual"] for r in reps)

    # end to end through the public API with host buffers: heat_step_host copies u from the
    # pinned host buffer to the device, steps it and copies it back, all inside the library
    e2e = None
    if not args.no_e2e:
        uh.copy_(u)
        barrier()
        e2e_steps = max(1, min(args.steps, 2))
        H.heat_step_host(uh, None, 1, **opts)          # untimed round trip (first-call set-up)
        barrier()
        t0 = time.perf_counter()
        e2e_apps = 0
        h2d_ms = d2h_ms = solve_ms = 0.0
        for k in range(e2e_steps):
            r = H.heat_step_host(uh, None, 1, **opts)
            e2e_apps += r["iterations"] + r["outer_iterations"] + 1
            h2d_ms += r["h2d_ms"] / e2e_steps
            d2h_ms += r["d2h_ms"] / e2e_steps
            solve_ms += (r["elapsed_ms"] - r["h2d_ms"] - r["d2h_ms"]) / e2e_steps
        t_e2e = max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": whole_job_gdofs(world, dofs, e2e_apps, t_e2e), "unit": "GDoF/s",
               "h2d_bytes_per_step": dofs * 8, "d2h_bytes_per_step": dofs * 8,
               "ms_per_step": 1e3 * t_e2e / e2e_steps, "h2d_ms": h2d_ms, "solve_ms": solve_ms,
               "d2h_ms": d2h_ms, "h2d_gbs": dofs * 8 / (h2d_ms * 1e-3) / 1e9,
               "d2h_gbs": dofs * 8 / (d2h_ms * 1e-3) / 1e9, "api": "heat_step_host (host buffers)"}
        del uh

    # dominant kernel: the fused CG iteration (one launch per inner iteration). Its average
    # duration inside the timed region comes from the CUDA events the library records on the
    # handle's stream around the CG-graph launches (iter_ms / iterations: an upper bound, it
    # includes the graph's inter-kernel gaps); time_kernel gives the same kernel timed alone.
    hbm, peak_kind = peaks()
    iter_ms = sum(r["iter_ms"] for r in reps)
    ms_fused_live = iter_ms / max(inner, 1)
    ms_fused = H.time_kernel(api.KERNEL_CG_FUSED, reps=10)
    # FP32 single-pass iteration: read p_{m-1}, q_{m-1}, p_{m-2}, x; write p_m, q_m, x (r is
    # rebuilt from the two p and never stored)
    bytes_fused = CG_BYTES_PER_UNKNOWN * dofs
    ms_op = H.time_kernel(api.KERNEL_OP, reps=10)
    bytes_op = 8.0 * dofs       # read x, write y (FP32)
    ms_res64 = H.time_kernel(api.KERNEL_RES64, reps=3)
    ms_resdf = H.time_kernel(api.KERNEL_RES_DF, reps=5)
    ms_upd = H.time_kernel(api.KERNEL_CG_UPDATE, reps=10)
    # B-spline transforms at the nodes of the same field (direct: interpolation by banded line
    # solves; indirect: the separable sampled-B-spline convolution), FP64 vectors
    cf = H.to_coeffs(u)
    uf = H.to_samples(cf)
    ms_direct, _ = _timed_ms(lambda: H.to_coeffs(u, cf))
    ms_indirect, _ = _timed_ms(lambda: H.to_samples(cf, uf))
    tr_err = (torch.max(torch.abs(uf - u)) / torch.max(torch.abs(u))).item()
    del cf, uf
    # BF16-storage operator variant (BSK_BF16S): its speed, and what BF16 storage costs in
    # accuracy against the FP64 operator of the same (unrounded) field
    Hb = api.Handle(N, N, N, DEGREE, h, DT, precision="bf16s", stream=stream)
    ub = u.to(torch.bfloat16)
    yb = Hb.op_apply(ub)
    torch.cuda.synchronize()
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    for _ in range(3):
        Hb.op_apply(ub, yb)
    eb1.record(stream)
    torch.cuda.synchronize()
    ms_bf16 = eb0.elapsed_time(eb1) / 3
    y64 = H.op_apply(u)
    bf16_err = (torch.linalg.vector_norm(yb.double() - y64) / torch.linalg.vector_norm(y64)).item()
    del y64, yb, ub
    Hb.close()
    ach = bytes_fused / (ms_fused_live * 1e-3) / 1e9
    traffic = None
    # the traffic figure of the plan actually in use: classic, or the warp-specialised pass with
    # chunked or whole-column items
    plan = H.cg_kernel_config()
    plan_key = "classic" if plan["kernel"] == "classic" else (
        "ws_columns" if plan["zchunk_planes"] >= N else "ws")
    per_unknown = CG_TRAFFIC_BYTES_PER_UNKNOWN.get(plan_key)
    if per_unknown is not None and cg_kernel_sources_sha256() == CG_TRAFFIC_SOURCES_SHA256:
        traffic = per_unknown * dofs

    line = {
        "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD if N == N_GRID else WORKLOAD.replace(str(N_GRID), str(N)),
            "grid": f"{N}^3", "unknowns": dofs, "degree": DEGREE, "dt": DT,
            "tol": TOL, "precision": "FP32 operator sweeps; true residual in double-float "
                                     "(FP64-accurate) on FP64 vectors; FP64 update and CG scalars",
            "l2": f"inputs larger than L2 ({4 * dofs / 1e9:.2f} GB FP32 / {8 * dofs / 1e9:.2f} GB FP64 vectors)",
            "cg_kernel": cg_kernel + " (chosen per handle by timing both single-pass CG kernels)"
                         if args.cg_kernel == "auto" else cg_kernel + " (forced)",
            "cg_kernel_config": H.cg_kernel_config(),
            "op_applications_per_step": op_apps / len(reps),
            "cg_iterations_per_step": inner / len(reps),
            "refinement_steps_per_step": outer / len(reps),
            "max_true_rel_residual": worst_res,
            "kernel_ms": {"cg_fused_f32_in_timed_region": ms_fused_live,
                          "cg_fused_f32_alone": ms_fused, "cg_update_f32": ms_upd, "op_f32": ms_op,
                          "residual_f64": ms_res64, "residual_double_float": ms_resdf},
            "cg_iteration_share_of_timed_region": iter_ms / elapsed_ms if world == 1 else None,
            "op_apply_gdofs": dofs / (ms_op * 1e-3) / 1e9,
            "op_apply_hbm_frac": bytes_op / (ms_op * 1e-3) / 1e9 / hbm,
            "transforms": {"direct_ms": ms_direct, "indirect_ms": ms_indirect,
                           "direct_gdofs": dofs / (ms_direct * 1e-3) / 1e9,
                           "indirect_gdofs": dofs / (ms_indirect * 1e-3) / 1e9,
                           "round_trip_max_rel_error": tr_err},
            "op_apply_bf16_storage": {"gdofs": dofs / (ms_bf16 * 1e-3) / 1e9, "ms": ms_bf16,
                                      "rel_l2_error_vs_fp64": bf16_err,
                                      "kernel": "general kernel, FP32 arithmetic, BF16 in/out"},
            "parallelism": f"{world} independent problems (one per GPU)",
        },
        "roofline": {"kernel": ("k_ws<3,WS_CG>" + (" (whole-column items)" if plan_key == "ws_columns" else "")
                                if cg_kernel == "ws" else "k_op_tma<float,3,CG>")
                               + ": one CG iteration (r rebuilt, p and x updates + A p + r.r, p.Ap, Ap.Ap)",
                     "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                     "frac": ach / hbm, "traffic": traffic,
                     "note": f"peak = {peak_kind} HBM copy bandwidth; algorithmic "
                             f"{CG_BYTES_PER_UNKNOWN:.0f} B/unknown (read p_m-1, q_m-1, p_m-2, x; write "
                             "p_m, q_m, x); duration = mean per iteration over the timed region (CUDA "
                             "events on the launching stream); traffic = DRAM bytes per unknown of the "
                             "same kernel captured at 512^3 (--profile-case cg512), times the unknowns",
                     "traffic_source": "profile case cg512 (512^3), scaled by unknowns"
                                       if traffic is not None else None},
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if e2e is not None:
        line["e2e"] = e2e
    H.close()
    del u
    torch.cuda.empty_cache()
    if rank == 0:
        # config 1 (32^3, sin sin sin, dt = 1e-3, 10 steps, tol 1e-10, FP64), for the CPU baseline
        hc = 1.0 / 33
        Hc = api.Handle(32, 32, 32, DEGREE, hc, 1e-3, precision="f64", stream=stream)
        u1 = inputs.sine_mode_field(32, 32, 32, [((1, 1, 1), 1.0)], device="cuda")
        Hc.heat_step(u1.clone(), None, 10, tol=1e-10)        # warm-up
        ms_c1, rep_c1 = _timed_ms(lambda: Hc.heat_step(u1, None, 10, tol=1e-10))
        line["c1_32cube_fp64"] = {"ms": ms_c1, "iterations": rep_c1["iterations"],
                                  "rel_residual": rep_c1["rel_residual"]}
        Hc.close()
    if rank == 0 and not args.no_fcg_race and args.grid == N_GRID:
        line["fcg_race"] = fcg_race()
    if rank == 0 and not args.no_extra_configs and args.grid == N_GRID:
        line["batch_64_boxes"] = batch_64_boxes()
        line["mixed_precision_sphere256"] = mixed_precision_sphere256()
        line["variable_coefficients"] = variable_coefficients()
        line["robin_large_run"] = robin_large_run()
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, secs, desc = cpu_oracle_sample()
        line["cpu_baseline"] = {"value": v, "unit": "GDoF/s", "cores": cores, "kind": "oracle",
                                "sample": desc, "cpu": cpu_model(),
                                "by_config": cpu_baseline_by_config(line)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the batched (64 boxes), the 256^3 mixed-precision, the "
                         "variable-coefficient and the Robin large-run measurements")
    ap.add_argument("--no-fcg-race", action="store_true",
                    help="skip the 512^3 union-of-spheres time-to-1e-8 race (learned FCG vs CG)")
    ap.add_argument("--grid", type=int, default=N_GRID,
                    help="grid edge (default: the benchmark workload; smaller grids are the "
                         "profiler's small case)")
    ap.add_argument("--cg-kernel", choices=["auto", "ws", "classic", "ws_chunked", "ws_columns"], default="auto",
                    help="single-pass CG kernel: chosen per handle by timing (default) or forced "
                         "(ws_chunked / ws_columns: the warp-specialised pass with z-chunks of <= 128 "
                         "planes or whole-column items)")
    ap.add_argument("--profile-case", choices=["op384", "cg512", "var240", "robin200", "batch64", "net512"], default=None,
                    help="run one small case for the profiler instead of the benchmark")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case, args.cg_kernel)
        return
    if args.grid < 16 or args.grid % 4:
        ap.error("--grid must be a multiple of 4 (16-byte FP32 rows for the TMA kernels), >= 16")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
