"""Benchmark: time to a 1e-6 relative FP64 residual, FP32-cycle-preconditioned FGMRES vs the plain
FP64 solve, and V-cycle HBM bandwidth, on one GB300.

Workload (default): the 2D heterogeneous configuration -- 2048 x 2048 cells, smooth random medium
(Vp 1.5-4.5, correlation length 64 cells), 10 points per minimum shear wavelength, point source at
depth 32, 5-level W(1,1) hierarchy with two coarsest sweeps, FGMRES(5) to 1e-6. One "step" is one
complete solve from a zero initial guess with the right-hand side resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl emg|reference] [--config c2|c1|c3]

--impl reference times the FP64 CPU oracle (oracle/) on the host cores instead: each step runs a
few FGMRES iterations on a crop of the same medium and extrapolates to the full solve.
Prints one JSON line on rank 0; the default (c2) line carries the other configurations as
sub-results under "configs".
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-6 rel. residual & V-cycle HBM GB/s: FP32-precond vs plain FP64, 1 GB300"
# Iteration count used to extrapolate the oracle's per-iteration time to a full solve in the
# reference arm (which runs no GPU code): iterations of the FP64 solve of each configuration with
# its own FGMRES restart (the FP64 GPU solve reproduces the oracle's count within +-1 in the
# parity tests).
REF_ITERS = {"c2": 230, "c1": 97, "c3": 193}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="emg", choices=["emg", "reference"])
    ap.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "c4", "c5"],
                    help="c4: the 64-instance batch of 2D solves (emg_solve_batch); c5: one misfit gradient of "
                         "the 3D inversion setting (forward and adjoint solves of 16 sources)")
    ap.add_argument("--instances", type=int, default=64, help="c4: number of instances")
    ap.add_argument("--grid", type=int, default=None,
                    help="cells per axis instead of the configuration's own (c1-c3; smaller cases for kernel captures)")
    ap.add_argument("--workers", type=int, default=0, help="c4: host worker threads (0: one per instance)")
    ap.add_argument("--restart", type=int, default=None, help="FGMRES restart length (default: the workload's)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed plain-FP64 solves (after 1 warm-up)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub-configs", action="store_true",
                    help="c2: leave out the other configurations' sub-results (c1, c2 seed 1, c3, c4, c5)")
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--damping", type=float, default=None)
    ap.add_argument("--cycle", default=None, choices=["V", "W", "K"])
    ap.add_argument("--coarse-sweeps", type=int, default=None)
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="run this many FGMRES iterations of the configured solve and exit without timing "
                         "(target for ncu launch lists and kernel captures)")
    ap.add_argument("--profile-precision", type=int, default=32, choices=[32, 64])
    return ap.parse_args()


def workload(name, args=None):
    from workloads import config_c1_homogeneous, config_c2_random2d, config_c3_layered3d
    make = {"c1": config_c1_homogeneous, "c2": config_c2_random2d, "c3": config_c3_layered3d}[name]
    grid = getattr(args, "grid", None) if args is not None else None
    w = make(grid) if grid else make()
    if args is not None:
        for k in ("levels", "alpha", "damping", "cycle", "coarse_sweeps", "restart"):
            v = getattr(args, k, None)
            if v is not None:
                setattr(w, k, v)
                if k == "alpha":
                    w.level_alpha = None
        args.restart = w.restart
    return w


# Sources of the dominant kernel (the finest-level one-pass 2D red-black sweep); the DRAM traffic
# recorded from an ncu capture is reported only while these files are unchanged.
HOT_KERNEL_SOURCES = ["paper_2307_03242_gb300/csrc/sweep2d_tile.cuh", "paper_2307_03242_gb300/csrc/vanka2d_fast.cuh",
                      "paper_2307_03242_gb300/csrc/kernels2d.cuh", "paper_2307_03242_gb300/csrc/stencil2d.cuh",
                      "paper_2307_03242_gb300/csrc/emg_types.cuh"]
HOT_KERNEL_PROFILE = "profiles/sweep_tile_c2_2048.txt"


def hot_kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in HOT_KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_profile(key, n):
    """A per-launch figure (DRAM bytes, FP32 flops) from the committed ncu summary of the dominant
    kernel, if it was captured on a finest grid of n cells and its sources still hash to the value
    recorded there; else None (DRAM traffic does not scale with the grid once it fits in L2)."""
    try:
        vals = {}
        with open(os.path.join(ROOT, HOT_KERNEL_PROFILE)) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("source_hash") != hot_kernel_hash():
            return None
        if tuple(int(v) for v in vals["grid"].split("x")) != tuple(n):
            return None
        return float(vals[key])
    except Exception:
        return None


def recorded_traffic(n):
    return recorded_profile("dram_bytes_per_launch", n)


# FP32 CUDA-core peak from the unit counts and the maximum clock: 152 SMs x 128 FP32 lanes x 2
# flop (FMA) x 2.07 GHz. (A measured FFMA loop reached 67.8 TFLOP/s on this part.)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_sample(w, iters=3, crop=512):
    """FP64 oracle on a crop of the same medium (same h, omega, shift, damping, absorbing layer):
    returns (seconds per FGMRES iteration scaled to the full grid, description, threads)."""
    import oracle
    from oracle.discretization import Problem
    d = w.dim
    c = min(crop if d == 2 else 64, min(w.n))
    sl = tuple(slice((n - c) // 2 if a < d - 1 else 0, ((n - c) // 2 if a < d - 1 else 0) + c)
               for a, n in reversed(list(enumerate(w.n))))
    n = (c,) * d
    lv = w.levels
    while c % (1 << (lv - 1)) or c >> (lv - 1) < 4:
        lv -= 1
    pb = Problem(n, w.h, w.omega, w.gamma, w.beta, w.lam[sl], w.mu[sl], w.rho[sl], abl_length=w.abl_cells * w.h,
                 abl_gamma_max=w.abl_gamma_max)
    if w.coarse == "kaczmarz":
        coarse = "kaczmarz"
    else:
        coarse = "dense" if (c >> (lv - 1)) ** d * (d + 1) <= 4096 and w.coarse == "dense" else "smooth"
    full = w.level_alphas()
    alphas = full[:lv - 1] + [full[-1]]  # the crop's coarsest level keeps the coarsest shift
    hier = oracle.Hierarchy(pb, lv, alphas, w.damping, nu_pre=w.nu_pre, nu_post=w.nu_post, coarse=coarse,
                            coarse_sweeps=max(w.coarse_sweeps, 1), coarse_damping=w.coarse_damping, cycle=w.cycle)
    H = oracle.assemble(pb, 0.0)
    b = np.zeros(H.shape[0], complex)
    b[oracle.active_mask(pb)] = 1.0
    t0, c0 = time.perf_counter(), time.process_time()
    _, its, _ = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b, tol=1e-30, restart=w.restart,
                              max_iter=iters)
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    dt = wall / its
    scale = float(np.prod(w.n)) / float(np.prod(n))
    desc = ("oracle FGMRES(%d)+%s(%d,%d) iterations on a %s crop of the same medium (%d levels), %d iterations "
            "timed, per-iteration time scaled by the cell ratio %.1f" % (w.restart, w.cycle, w.nu_pre, w.nu_post,
                                                                         "x".join(map(str, n)), lv, its, scale))
    # the threads the oracle actually kept busy (process CPU time over wall time): scipy.sparse
    # products run on one thread, the small dense block solves mostly so
    threads = max(1, int(round(cpu / wall)))
    desc += "; %.2f CPU-seconds per wall second on %d host cores" % (cpu / wall, os.cpu_count())
    return dt * scale, desc, threads


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.config not in REF_ITERS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm covers the single-solve "
                          "configurations c1-c3; %s has no single-solve iteration count" % args.config}))
        return
    w = workload(args.config, args)
    iters = REF_ITERS[args.config]
    vals = []
    for s in range(args.warmup + args.steps):
        per_it, desc, threads = oracle_sample(w, iters=2)
        if s >= args.warmup:
            vals.append(per_it * iters)
    v = float(np.mean(vals))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128", "data": "synthetic", "config": config_json(w, args),
           "cpu_baseline": {"value": v, "unit": "s", "cores": threads, "kind": "oracle",
                            "sample": desc + " x %d iterations (FP64 solve count)" % iters},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def max_over_ranks(value, device=None):
    """Replica timing: every rank solves its own copy of the workload (no data exchange); the
    job's time is the slowest rank's. Returns value unchanged when torch.distributed is not
    initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config_json(w, args):
    return {"workload": w.name, "grid": "x".join(map(str, w.n)), "levels": w.levels, "cycle": "%s(%d,%d)" % (
        w.cycle, w.nu_pre, w.nu_post), "coarse_sweeps": w.coarse_sweeps, "alpha": w.alpha, "damping": w.damping, "beta": round(w.beta, 6),
        "krylov": "FGMRES(%d)" % args.restart, "tol": w.tol, "coarsest": w.coarse if w.coarse != "kaczmarz" else
        "hybrid Kaczmarz-GMRES: FGMRES(5) on the Schur complement, 10 steps at 0.8 over 2^d-cell boxes, 0.1 drop",
        "shift_per_level": [round(v, 6) for v in w.level_alphas()],
        "l2": "inputs larger than L2 (vectors %d MB)" % int(16 * (w.dim + 1) * np.prod(w.n) / 2 ** 20),
        "parallelism": "replicas" if args.gpus > 1 else "single"}


def run_profile(args):
    """K FGMRES iterations of the configured solve, no timing (for ncu)."""
    import torch
    from paper_2307_03242_gb300 import emg
    w = workload(args.config, args)
    b = torch.from_numpy(w.rhs.astype(np.complex128)).cuda()
    s = emg.Solver(emg.params_from_workload(w, args.profile_precision), w.lam, w.mu, w.rho)
    x = torch.zeros_like(b)
    st = s.solve(b, x, tol=w.tol, max_iter=args.profile_iters, restart=args.restart)
    torch.cuda.synchronize()
    s.close()
    print(json.dumps({"profile_iters": st["iterations"], "rel_residual": st["rel_residual"], "workload": w.name}))


def dist_context():
    """(world, rank, local device index, device): one process per GPU under torchrun; the process
    group (NCCL) serves only the barrier and the max-over-ranks timing."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    return world, rank, local, torch.device("cuda", local)


def bench_single(args, w, steps, warmup, fp64_steps, cpu_baseline, e2e_steps=None):
    """One configuration solved K times from a zero guess (the JSON line of a single-solve
    workload): the FP32-cycle solve timed with CUDA events, the plain FP64 solve (fp64_steps > 0),
    the V-cycle alone, the end-to-end solve through host buffers and, on request, the oracle."""
    import torch
    import torch.distributed as dist
    from paper_2307_03242_gb300 import emg
    world, rank, local, dev = dist_context()
    e2e_steps = steps if e2e_steps is None else e2e_steps
    shape = (w.dim + 1,) + tuple(w.n[::-1])
    nvec = int(np.prod(shape))
    b = torch.from_numpy(w.rhs.astype(np.complex128)).to(dev)
    # the solver runs on a stream of its own, where its preconditioner cycle is replayed as a
    # captured CUDA graph; the timing events are recorded on that stream
    sst = torch.cuda.Stream(dev)
    s32 = emg.Solver(emg.params_from_workload(w, 32), w.lam, w.mu, w.rho, stream=sst)
    paths = [s32.sweep_path(l)[0] for l in range(w.levels)]
    x = torch.zeros_like(b)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def solve(s):
        x.zero_()
        return s.solve(b, x, tol=w.tol, max_iter=2000, restart=args.restart)

    for _ in range(warmup):
        st = solve(s32)
    s32.profile_read(emg.K_ALL)
    s32.profile(True)
    st = solve(s32)  # captures the timed cycle graphs (instrumentation events inside)
    for cls in (emg.K_SMOOTH, emg.K_RESTRICT, emg.K_PROLONG, emg.K_APPLY64, emg.K_KRYLOV, emg.K_ALL):
        s32.profile_read(cls)
    stream = sst
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        e0.record(stream)
        iters = []
        for _ in range(steps):
            st = solve(s32)
            iters.append(st["iterations"])
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1) / steps
    prof = s32.profile_read(emg.K_SMOOTH)
    breakdown = {name: s32.profile_read(cls) for name, cls in (("restrict", emg.K_RESTRICT), ("prolong", emg.K_PROLONG),
                                                               ("apply64", emg.K_APPLY64), ("krylov", emg.K_KRYLOV))}
    s32.profile(False)
    launches = s32.profile_read(emg.K_ALL)["launches"]
    # one more solve, untimed, with every level's kernels timed: the coarser levels' share
    s32.profile(True, coarse=True)
    solve(s32)
    coarse_ms = s32.profile_read(emg.K_COARSE)["ms"]
    for cls in (emg.K_SMOOTH, emg.K_RESTRICT, emg.K_PROLONG, emg.K_APPLY64, emg.K_KRYLOV, emg.K_ALL):
        s32.profile_read(cls)
    s32.profile(False)
    t32 = max_over_ranks(ms / 1e3, device=dev)
    res32 = st["rel_residual"]

    # V-cycle bandwidth (FP32 cycle on the finest level, zero initial guess)
    bc = torch.zeros(shape, dtype=torch.complex64, device=dev)
    bc.copy_(b)
    xc = torch.zeros_like(bc)
    for _ in range(3):
        s32.vcycle(bc, xc)
    barrier()
    nv = 20
    e0.record(stream)
    for _ in range(nv):
        s32.vcycle(bc, xc)
    e1.record(stream)
    barrier()
    vms = e0.elapsed_time(e1) / nv
    ncell = float(np.prod(w.n))
    # algorithmic bytes per finest cell of one cycle over all level visits (vcycle_bytes_per_cell)
    per_cell = vcycle_bytes_per_cell(w, 8, 4)
    v_gbs = per_cell * ncell / (vms * 1e-3) / 1e9

    # plain FP64 solve
    s32.close()
    t64, st64 = None, None
    if fp64_steps > 0:
        s64 = emg.Solver(emg.params_from_workload(w, 64), w.lam, w.mu, w.rho, stream=sst)
        st64 = solve(s64)
        barrier()
        e0.record(stream)
        for _ in range(fp64_steps):
            st64 = solve(s64)
        e1.record(stream)
        barrier()
        t64 = e0.elapsed_time(e1) / fp64_steps / 1e3
        s64.close()

    # end to end through the public API with host buffers (copies inside the timed region)
    s32 = emg.Solver(emg.params_from_workload(w, 32), w.lam, w.mu, w.rho, stream=sst)
    bh = torch.from_numpy(w.rhs.astype(np.complex128).ravel()).pin_memory().numpy()
    xh = torch.zeros(nvec, dtype=torch.complex128).pin_memory().numpy()
    s32.solve_host(bh, xh, tol=w.tol, max_iter=2000, restart=args.restart)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        xh[:] = 0
        sth = s32.solve_host(bh, xh, tol=w.tol, max_iter=2000, restart=args.restart)
    barrier()
    te2e = (time.perf_counter() - t0) / e2e_steps
    s32.close()

    peak, peak_kind = load_peaks()
    achieved = prof["bytes"] / (prof["ms"] * 1e-3) / 1e9 if prof["ms"] > 0 else None
    out = {"metric": METRIC, "value": t32, "unit": "s", "n_gpus": world, "steps": steps, "warmup": warmup,
           "ms_per_step": t32 * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "c64 cycle / c128 outer", "data": "synthetic", "config": config_json(w, args),
           "iterations": {"fp32_precond": int(np.median(iters)), "fp64_plain": st64["iterations"] if st64 else None},
           "rel_residual": {"fp32_precond": res32, "fp64_plain": st64["rel_residual"] if st64 else None},
           "fp64_plain": {"value": t64, "unit": "s", "steps": fp64_steps, "warmup": 1} if st64 else None,
           "speedup_vs_fp64": t64 / t32 if t64 else None,
           "vcycle": {"ms": vms, "gbs_algorithmic": v_gbs, "bytes_per_cell": per_cell,
                      "frac_of_hbm": v_gbs / peak},
           "roofline": dict(finest_sweep_kernel(w, paths), **{
                        "bound": "hbm", "achieved": achieved,
                        "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                        "frac": achieved / peak if achieved else None,
                        "traffic": recorded_traffic(w.n) if tiled_finest(w, paths) else None,
                        "launches": prof["launches"], "avg_launch_ms": prof["ms"] / max(prof["launches"], 1),
                        "bytes_per_launch": prof["bytes"] / max(prof["launches"], 1),
                        "fp32": fp32_fraction(prof, w.n) if tiled_finest(w, paths) else None}),
           "fine_level_ms_per_solve": dict({"smooth": prof["ms"] / steps},
                                           **{k: v["ms"] / steps for k, v in breakdown.items()}),
           "coarse_levels_ms_per_solve": coarse_ms,
           "e2e": {"value": te2e, "unit": "s", "h2d_bytes_per_step": 2 * nvec * 16, "d2h_bytes_per_step": nvec * 16},
           "gpu_launches": int(launches)}
    out["sweep_paths"] = [emg.SWEEP_NAMES[p] for p in paths]
    if rank == 0 and world == 1 and cpu_baseline:
        per_it, desc, threads = oracle_sample(w)
        out["cpu_baseline"] = {"value": per_it * out["iterations"]["fp32_precond"], "unit": "s", "cores": threads,
                               "kind": "oracle", "sample": desc + " x the FP32 solve's iteration count"}
    out["clocks"] = clk.summary()
    return out


def sub_configs(args):
    """The other configurations, each with its own timing, iterations, end-to-end figure and clock
    record, at fewer steps so that the default run stays short: the small 128^2 case (C1), a
    second medium of the 2048^2 configuration (seed 1, held out from the damping choice), the
    256^3 layered medium (C3), the 64-instance batch (C4) and the 128^3 misfit gradient (C5)."""
    import copy
    from workloads import config_c2_random2d
    out = {}
    a = copy.copy(args)
    a.restart = None
    w1 = workload("c1", a)
    out["c1"] = bench_single(a, w1, steps=3, warmup=1, fp64_steps=1, cpu_baseline=False, e2e_steps=3)
    a = copy.copy(args)
    a.restart = None
    w = config_c2_random2d(seed=1)
    a.restart = w.restart
    r = bench_single(a, w, steps=2, warmup=1, fp64_steps=0, cpu_baseline=False, e2e_steps=1)
    r["config"]["workload"] = "c2_random_2d_2048_seed1"
    out["c2_seed1"] = r
    a = copy.copy(args)
    a.restart = None
    w3 = workload("c3", a)
    out["c3"] = bench_single(a, w3, steps=1, warmup=1, fp64_steps=0, cpu_baseline=False, e2e_steps=1)
    a = copy.copy(args)
    out["c4"] = bench_batch(a, steps=1, warmup=1)
    a = copy.copy(args)
    a.grid = None
    out["c5"] = bench_gradient(a, steps=1, warmup=1)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_iters > 0:
        run_profile(args)
        return
    world, rank, local, dev = dist_context()
    if args.config == "c4":
        out = bench_batch(args, args.steps, args.warmup)
    elif args.config == "c5":
        out = bench_gradient(args, args.steps, args.warmup)
    else:
        w = workload(args.config, args)
        out = bench_single(args, w, args.steps, args.warmup, args.fp64_steps, not args.no_cpu_baseline)
        if args.config == "c2" and world == 1 and not args.no_sub_configs and args.grid is None:
            out["configs"] = sub_configs(args)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


BATCH_METRIC = "time to solve a batch of independent 2D systems to 1e-6 rel. residual (FP32 cycle, FP64 FGMRES), 1 GB300"


def bench_batch(args, steps, warmup):
    """The 2D batch (config_c4_batch): every (instance, source) system solved to 1e-6, all of them
    in one emg_solve_batch call per step (each instance on a stream of its own). Reported: the
    batch time (wall clock between device synchronisations, since the work spans every
    instance's stream and the host threads that drive them), the same systems solved one after
    another, and the finest-level half-sweep's bandwidth from per-launch CUDA events of that
    sequential pass."""
    import torch
    import torch.distributed as dist
    from paper_2307_03242_gb300 import emg
    from workloads import config_c4_batch
    world, rank, local, dev = dist_context()
    ws = config_c4_batch(args.instances)
    solvers, jobs = [], []
    for w in ws:
        s = emg.Solver(emg.params_from_workload(w, 32), w.lam, w.mu, w.rho, stream=torch.cuda.Stream(dev))
        solvers.append(s)
        for q in w.extra["sources"]:
            b = torch.from_numpy(q).to(dev)
            jobs.append((s, b, torch.zeros_like(b)))
    tol, restart = ws[0].tol, ws[0].restart
    mcells = sum(s.ncell for s, _, _ in jobs) / 1e6

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def batch():
        for _, _, x in jobs:
            x.zero_()
        return emg.solve_batch(jobs, tol=tol, max_iter=2000, restart=restart, workers=args.workers)

    for _ in range(warmup):
        res = batch()
    for s in solvers:
        s.profile_read(emg.K_ALL)
    barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(steps):
            res = batch()
        barrier()
        tb = (time.perf_counter() - t0) / steps
    launches = sum(s.profile_read(emg.K_ALL)["launches"] for s in solvers) // steps
    tb = max_over_ranks(tb, device=dev)
    # the same systems one after another, with per-launch instrumentation
    smooth = {"ms": 0.0, "launches": 0, "bytes": 0.0}
    barrier()
    t0 = time.perf_counter()
    seq = []
    for s, b, x in jobs:
        s.profile(True)
        x.zero_()
        seq.append(s.solve(b, x, tol=tol, max_iter=2000, restart=restart))
        p = s.profile_read(emg.K_SMOOTH)
        s.profile(False)
        for k in smooth:
            smooth[k] += p[k]
    barrier()
    tseq = time.perf_counter() - t0
    # end to end: right-hand sides from pinned host memory in, solutions out, inside the timing
    hb = [torch.from_numpy(q).pin_memory() for w in ws for q in w.extra["sources"]]
    hx = [torch.empty_like(h).pin_memory() for h in hb]
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        for h, (_, b, _) in zip(hb, jobs):
            b.copy_(h, non_blocking=True)
        batch()
        for h, (_, _, x) in zip(hx, jobs):
            h.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
    te2e = (time.perf_counter() - t0) / steps
    nbytes = int(sum(h.numel() for h in hb) * 16)
    its = [r["iterations"] for r in res]
    peak, peak_kind = load_peaks()
    achieved = smooth["bytes"] / (smooth["ms"] * 1e-3) / 1e9 if smooth["ms"] > 0 else None
    sizes = sorted(set(w.n[0] for w in ws))
    out = {"metric": BATCH_METRIC, "value": tb, "unit": "s", "n_gpus": world, "steps": steps,
           "warmup": warmup, "ms_per_step": tb * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "c64 cycle / c128 outer", "data": "synthetic",
           "config": {"workload": "c4_batch_%d" % len(ws), "instances": len(ws), "systems": len(jobs),
                      "grids": "%s (squares)" % "/".join(map(str, sizes)), "mcell_systems": round(mcells, 2),
                      "cycle": "W(2,2)", "levels": 5, "krylov": "FGMRES(%d)" % restart, "tol": tol,
                      "concurrency": "one stream and host worker per instance",
                      "timing": "wall clock between device synchronisations",
                      "l2": "inputs larger than L2 (%.0f MB of FP64 right-hand sides)" % (16 * mcells * 3),
                      "parallelism": "replicas" if world > 1 else "single"},
           "throughput_mcell_systems_per_s": mcells / tb,
           "iterations": {"min": int(min(its)), "median": int(np.median(its)), "max": int(max(its)),
                          "all_converged": all(r["converged"] for r in res)},
           "sequential": {"value": tseq, "unit": "s", "speedup_of_batch": tseq / tb},
           "roofline": {"kernel": "vanka half-sweep (finest level of every instance, FP32, sequential pass)",
                        "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                        "frac": achieved / peak if achieved else None, "traffic": None,
                        "launches": smooth["launches"]},
           "e2e": {"value": te2e, "unit": "s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
           "gpu_launches": int(launches)}
    out["clocks"] = clk.summary()
    out["sweep_paths"] = {str(n): [emg.SWEEP_NAMES[s.sweep_path(l)[0]] for l in range(s.params.levels)]
                          for n, s in sorted({w.n[0]: s for w, s in zip(ws, solvers)}.items())}
    for s in solvers:
        s.close()
    return out


GRADIENT_METRIC = "time per misfit gradient wrt (lambda, mu, rho): forward + adjoint solves of every source, 1 GB300"


def bench_gradient(args, steps, warmup):
    """One misfit gradient of the 3D inversion setting (config_c5_adjoint: 128^3, 16 sources, 64 x
    64 receivers): per step, a solver built from the current model, a forward solve per source,
    an adjoint solve per source and the material-derivative kernel (inversion.misfit + backward),
    timed with CUDA events on the current stream between synchronisations. The data come from
    the +5 % blob model (set-up, untimed). A second, instrumented pass reports the finest-level
    half-sweep bandwidth."""
    import torch
    import torch.distributed as dist
    from paper_2307_03242_gb300 import emg, inversion
    from workloads import config_c5_adjoint
    world, rank, local, dev = dist_context()
    n = args.grid or 128
    w = config_c5_adjoint(n)
    params = emg.params_from_workload(w, 32)
    shape = (w.dim + 1,) + tuple(w.n[::-1])
    rec = torch.tensor([int(np.ravel_multi_index((c,) + tuple(idx[::-1]), shape)) for c, idx in w.extra["receivers"]],
                       dtype=torch.int64, device=dev)
    sources = [torch.from_numpy(q).to(dev) for q in w.extra["sources"]]
    true = emg.Solver(params, *w.extra["true"])
    data = []
    for q in sources:
        u = torch.zeros_like(q)
        true.solve(q, u, tol=w.tol, max_iter=4000, restart=w.restart)
        data.append(u.reshape(-1)[rec].clone())
    true.close()
    model = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (w.lam, w.mu, w.rho)]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def gradient(m, stats=None, solver=None):
        leaves = [t.detach().clone().requires_grad_(True) for t in m]
        J = inversion.misfit(*leaves, params, sources, rec, data, tol=w.tol, solver=solver, stats=stats,
                             restart=w.restart)
        J.backward()
        return J, [t.grad for t in leaves]

    for _ in range(warmup):
        gradient(model)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    barrier()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(steps):
            J, g = gradient(model, stats)
        e1.record(stream)
        barrier()
    tg = max_over_ranks(e0.elapsed_time(e1) / steps / 1e3, device=dev)
    fwd = [st["iterations"] for st in stats if st["kind"] == "forward"]
    adj = [st["iterations"] for st in stats if st["kind"] == "adjoint"]
    # instrumented pass on a solver built once: finest-level half-sweep bandwidth, launch count
    s = emg.Solver(params, *model)
    s.profile(True)
    s.profile_read(emg.K_ALL)
    gradient(model, solver=s)
    prof = s.profile_read(emg.K_SMOOTH)
    launches = s.profile_read(emg.K_ALL)["launches"]
    s.profile(False)
    s.close()
    # end to end: the model from pinned host memory in, the three gradient fields out
    hm = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (w.lam, w.mu, w.rho)]
    hg = [torch.empty_like(h).pin_memory() for h in hm]
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        m = [h.to(dev, non_blocking=True) for h in hm]
        _, g = gradient(m)
        for h, gg in zip(hg, g):
            h.copy_(gg, non_blocking=True)
        torch.cuda.synchronize()
    te2e = (time.perf_counter() - t0) / steps
    nbytes = int(sum(h.numel() for h in hm) * 8)
    peak, peak_kind = load_peaks()
    achieved = prof["bytes"] / (prof["ms"] * 1e-3) / 1e9 if prof["ms"] > 0 else None
    out = {"metric": GRADIENT_METRIC, "value": tg, "unit": "s", "n_gpus": world, "steps": steps,
           "warmup": warmup, "ms_per_step": tg * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "c64 cycle / c128 outer", "data": "synthetic",
           "config": {"workload": "c5_adjoint_3d_%d" % n, "grid": "%dx%dx%d" % tuple(w.n), "sources": len(sources),
                      "receivers": int(rec.numel()), "cycle": "K(1,1)", "levels": w.levels,
                      "krylov": "FGMRES(%d)" % w.restart, "tol": w.tol,
                      "l2": "inputs larger than L2" if 16 * 4 * np.prod(w.n) > 129e6 else "inputs smaller than L2",
                      "parallelism": "replicas" if world > 1 else "single"},
           "iterations": {"forward_median": int(np.median(fwd)), "adjoint_median": int(np.median(adj)),
                          "forward_total": int(sum(fwd)) // steps, "adjoint_total": int(sum(adj)) // steps},
           "misfit": float(J.item()),
           "roofline": {"kernel": "vanka half-sweep (finest level, FP32, instrumented pass)", "bound": "hbm",
                        "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                        "frac": achieved / peak if achieved else None, "traffic": None,
                        "launches": prof["launches"]},
           "e2e": {"value": te2e, "unit": "s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
           "gpu_launches": int(launches)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_it, desc, threads = oracle_sample(w)
        total = out["iterations"]["forward_total"] + out["iterations"]["adjoint_total"]
        out["cpu_baseline"] = {"value": per_it * total, "unit": "s", "cores": threads, "kind": "oracle",
                               "sample": desc + " x the forward and adjoint iterations of one gradient"}
    out["clocks"] = clk.summary()
    return out


def tiled_finest(w, paths):
    """True when the finest level's sweeps run the one-pass tiled kernel (2D, FP32)."""
    from paper_2307_03242_gb300 import emg
    return w.dim == 2 and paths and paths[0] in (emg.SWEEP_TILE24, emg.SWEEP_TILE8, emg.SWEEP_TILE4)


def finest_sweep_kernel(w, paths):
    """Name and byte basis of the finest level's sweep kernel, the roofline's dominant kernel."""
    if tiled_finest(w, paths):
        return {"kernel": "one-pass red-black Vanka sweep k2t::sweep_tile (finest level, FP32)",
                "bytes_basis": "84 B per cell per sweep (3S + 3r), 60 B from a zero guess, + 6 B of coarse "
                               "correction in the first post-sweep"}
    if w.dim == 3:
        return {"kernel": "red-black Vanka half-sweep k3t::vanka_tile (finest level, FP32)",
                "bytes_basis": "100 B per cell per half-sweep (the colour's faces and pressures read and "
                               "written, b read, 3 material reals)"}
    return {"kernel": "red-black Vanka half-sweep k2::vanka_fast (finest level, FP32)",
            "bytes_basis": "76 B per cell per half-sweep"}


def fp32_fraction(prof, n):
    """The dominant kernel's FP32 rate: its flops per launch (ncu FADD + FMUL + 2 FFMA thread
    instructions of one launch, from the committed summary) over the live mean launch time."""
    flops = recorded_profile("fp32_flops_per_launch", n)
    if not flops or prof["ms"] <= 0:
        return None
    tf = flops / (prof["ms"] / max(prof["launches"], 1) * 1e-3) / 1e12
    return {"achieved_tflops": tf, "peak_tflops": FP32_PEAK_TFLOPS, "peak_kind": "derived (unit counts x max clock)",
            "frac": tf / FP32_PEAK_TFLOPS, "flops_per_launch": flops}


def vcycle_bytes_per_cell(w, cw, rw):
    """Algorithmic bytes per finest cell of one preconditioner cycle: the method's minimum traffic
    of each step (every input read once, every output written once, no stored matrix), with
    c = complex word, r = real word, S = (d+1)c per cell of a level:
      sweep (both colours)     3S + 3r (read x, b and mu, rho, 1/(lambda+mu); write x);
                               2S + 3r for a sweep from a zero guess (x is not read)
      residual + restriction   2S + 3r (read x, b, material) + S/2^d (write the coarse b)
      prolongation + correction into the first post-sweep: S/2^d (read the coarse e)
    Level l has 2^-dl of the finest cells. A V-cycle visits every level once; a W- or K-cycle
    visits level l <= L-2 2^l times (the first call of each pair from a zero guess) and the
    coarsest level 2^(L-2) times (from a zero guess)."""
    d = w.dim
    S = (d + 1) * cw
    sweep = 3 * S + 3 * rw
    g = 1 if w.cycle == "V" else 2
    tot = 0.0
    for l in range(w.levels):
        cells = 2.0 ** (-d * l)
        if l < w.levels - 1:
            visits = g ** l
            zero_visits = 1 if l == 0 else visits // g  # the finest cycle starts from zero, then one call per pair
            lvl = (w.nu_pre + w.nu_post) * sweep + (2 * S + 3 * rw + S / 2 ** d) + S / 2 ** d
            tot += cells * (visits * lvl - (zero_visits * S if w.nu_pre > 0 else 0.0))
        else:
            visits = g ** max(l - 1, 0)
            lvl = (w.coarse_sweeps * sweep - S) if w.coarse == "smooth" else 0.0
            tot += visits * cells * lvl
    return tot

if __name__ == "__main__":
    main()
